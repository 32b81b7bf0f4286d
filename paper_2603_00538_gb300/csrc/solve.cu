// Step 7 of Sec. 4: solve the target Galerkin system M u = b (Eq.
// cv_galerkin_system) from u = 0 (or, in the mixed mode on request, from the
// u the caller holds), stopping at ||b - M u||_2 <= tol ||b||_2 (the paper
// does not name its solver). Two kernels:
//   k_pcg       Jacobi-preconditioned CG in FP64 (cg_mode FP64, and the
//               allocation-free entry point, which takes any SPD CSR matrix);
//   k_mixed_cg  mixed-precision iterative refinement (default; see below).
//
// One cooperative (co-resident) kernel runs the whole iteration: no host round
// trip per step. Each k_pcg iteration has two grid barriers:
//   A: w = M z (SpMV), then for the own row p = z + beta p and
//      q = w + beta q (= M p by linearity, one FP64 FMA per nonzero instead of
//      two), and the partial dot p.q;
//   B: u += a p, r -= a q, z = D^-1 r, partial dots r.r and r.z.
// FP64 throughput is the scarce resource on this GPU, so the iteration is
// written to minimise FP64 operations per row.
// Dot products are reduced deterministically: per-block partials, then every
// block sums all partials in the same fixed order, so all blocks take the
// same convergence decision. The barrier wait is bounded (error flag on
// timeout; the kernel then returns).
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>
#include "internal.hpp"
#include "util.cuh"

namespace sft {

constexpr int kSolveThreads = 256;

struct PcgCtl {
  GridBarrier bar;
  int32_t err;
  int32_t iters[kMaxFields];
  double rel[kMaxFields];
  int32_t conv[kMaxFields];
};

// sum the per-block partials [nblocks][nrhs][2] -> tot[nrhs][2], identical
// in all blocks: thread t sums blocks t, t + 256, ... in order, then warps
// reduce with a fixed shuffle tree and thread k adds the 8 warp sums in order
__device__ __forceinline__ void reduce_partials(const double* part, int nblocks, int nrhs, double* sh_tot) {
  __shared__ double shw[kSolveThreads / 32][kMaxFields * 2];
  double acc[kMaxFields * 2];
#pragma unroll
  for (int k = 0; k < kMaxFields * 2; ++k) acc[k] = 0.0;
  for (int bidx = threadIdx.x; bidx < nblocks; bidx += blockDim.x) {
    const double* pb = part + (int64_t)bidx * nrhs * 2;
#pragma unroll
    for (int k = 0; k < kMaxFields * 2; ++k)
      if (k < nrhs * 2) acc[k] += __ldcg(pb + k);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < kMaxFields * 2; ++k) {
    if (k >= nrhs * 2) break;
    const double w = warp_sum<double>(acc[k]);
    if (lane == 0) shw[warp][k] = w;
  }
  __syncthreads();
  if (threadIdx.x < nrhs * 2) {
    double t = 0.0;
    for (int w = 0; w < kSolveThreads / 32; ++w) t += shw[w][threadIdx.x];
    sh_tot[threadIdx.x] = t;
  }
  __syncthreads();
}

__device__ __forceinline__ void block_partials(double v[kMaxFields][2], int nrhs, double* part) {
  __shared__ double sh[kSolveThreads / 32][kMaxFields][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int f = 0; f < nrhs; ++f)
    for (int c = 0; c < 2; ++c) {
      const double w = warp_sum<double>(v[f][c]);
      if (lane == 0) sh[warp][f][c] = w;
    }
  __syncthreads();
  if (threadIdx.x < nrhs * 2) {
    const int f = threadIdx.x >> 1, c = threadIdx.x & 1;
    double s = 0.0;
    for (int w = 0; w < kSolveThreads / 32; ++w) s += sh[w][f][c];
    part[((int64_t)blockIdx.x * nrhs + f) * 2 + c] = s;
  }
  __syncthreads();
}

template <int TPR>
__global__ void __launch_bounds__(kSolveThreads) k_pcg(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                       const double* __restrict__ val, const double* __restrict__ dinv,
                                                       int64_t n, int nrhs, const double* __restrict__ b,
                                                       double* __restrict__ x, double* r, double* z, double* p,
                                                       double* q, double* part, PcgCtl* ctl, double tol,
                                                       int max_iter, uint64_t wait_ns) {
  __shared__ double tot[kMaxFields * 2];
  __shared__ double bnorm[kMaxFields], rz[kMaxFields], beta[kMaxFields], alpha[kMaxFields];
  __shared__ int conv[kMaxFields];
  const unsigned nb = gridDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  double v[kMaxFields][2];

  // init: x = 0, r = b, z = D^-1 r, p_old = 0
  for (int f = 0; f < kMaxFields; ++f) v[f][0] = v[f][1] = 0.0;
  for (int64_t i = tid; i < n; i += nthreads) {
    const double di = dinv[i];
    for (int f = 0; f < nrhs; ++f) {
      const int64_t k = (int64_t)f * n + i;
      const double bi = b[k];
      x[k] = 0.0;
      r[k] = bi;
      z[k] = di * bi;
      p[k] = 0.0;
      q[k] = 0.0;
      v[f][0] += bi * bi;
      v[f][1] += bi * di * bi;
    }
  }
  block_partials(v, nrhs, part);
  if (!grid_sync(&ctl->bar, nb, &ctl->err, wait_ns)) return;
  reduce_partials(part, nb, nrhs, tot);
  if (threadIdx.x == 0) {
    for (int f = 0; f < nrhs; ++f) {
      bnorm[f] = sqrt(tot[f * 2]);
      rz[f] = tot[f * 2 + 1];
      beta[f] = 0.0;
      conv[f] = bnorm[f] == 0.0;
    }
  }
  __syncthreads();

  int it = 0;
  constexpr int kRowsPerWarp = 32 / TPR;
  const int lane = threadIdx.x & 31;
  const int lane_in_row = lane % TPR;
  const int64_t warp_id = tid >> 5, nwarps = nthreads >> 5;
  for (;;) {
    bool all = true;
    for (int f = 0; f < nrhs; ++f) all = all && conv[f];
    if (all || it >= max_iter) break;
    // phase A (warp-uniform loop: each warp owns 32/TPR consecutive rows)
    for (int f = 0; f < kMaxFields; ++f) v[f][0] = v[f][1] = 0.0;
    for (int64_t base = warp_id * kRowsPerWarp; base < n; base += nwarps * kRowsPerWarp) {
      const int64_t row = base + lane / TPR;
      const bool valid = row < n;
      int32_t q0 = 0, q1 = 0;
      if (valid) {
        q0 = __ldg(rp + row);
        q1 = __ldg(rp + row + 1);
      }
      for (int f = 0; f < nrhs; ++f) {
        if (conv[f]) continue;
        const double* zf = z + (int64_t)f * n;
        double s = 0.0;
        // z was written by other blocks before the grid barrier; the barrier's
        // acquire fence makes those writes visible to ordinary (L1-cached)
        // loads, so neighbouring rows share the gathered lines in L1
        for (int32_t k = q0 + lane_in_row; k < q1; k += TPR) s += __ldg(val + k) * zf[__ldg(col + k)];
        if constexpr (TPR > 1) {
#pragma unroll
          for (int o = TPR / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, TPR);
        }
        if (valid && lane_in_row == 0) {
          const double bt = beta[f];
          const int64_t k = (int64_t)f * n + row;
          const double pn = __ldcg(zf + row) + bt * __ldcg(p + k);
          const double qn = s + bt * __ldcg(q + k);
          p[k] = pn;
          q[k] = qn;
          v[f][0] += pn * qn;
        }
      }
    }
    block_partials(v, nrhs, part);
    if (!grid_sync(&ctl->bar, nb, &ctl->err, wait_ns)) return;
    reduce_partials(part, nb, nrhs, tot);
    if (threadIdx.x == 0)
      for (int f = 0; f < nrhs; ++f) alpha[f] = conv[f] ? 0.0 : rz[f] / tot[f * 2];
    __syncthreads();
    // phase B
    for (int f = 0; f < kMaxFields; ++f) v[f][0] = v[f][1] = 0.0;
    for (int64_t i = tid; i < n; i += nthreads) {
      const double di = dinv[i];
      for (int f = 0; f < nrhs; ++f) {
        if (conv[f]) continue;
        const int64_t k = (int64_t)f * n + i;
        const double a = alpha[f];
        x[k] = __ldcg(x + k) + a * __ldcg(p + k);
        const double ri = __ldcg(r + k) - a * __ldcg(q + k);
        r[k] = ri;
        const double zi = di * ri;
        z[k] = zi;
        v[f][0] += ri * ri;
        v[f][1] += ri * zi;
      }
    }
    block_partials(v, nrhs, part);
    if (!grid_sync(&ctl->bar, nb, &ctl->err, wait_ns)) return;
    reduce_partials(part, nb, nrhs, tot);
    ++it;
    if (threadIdx.x == 0) {
      for (int f = 0; f < nrhs; ++f) {
        if (conv[f]) continue;
        const double rn = sqrt(tot[f * 2]);
        ctl->iters[f] = it;  // identical in every block
        ctl->rel[f] = rn / bnorm[f];
        if (rn <= tol * bnorm[f]) conv[f] = 1;
        beta[f] = tot[f * 2 + 1] / rz[f];
        rz[f] = tot[f * 2 + 1];
      }
    }
    __syncthreads();
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int f = 0; f < nrhs; ++f) {
      ctl->conv[f] = conv[f];
      if (bnorm[f] == 0.0) { ctl->iters[f] = 0; ctl->rel[f] = 0.0; }
    }
  }
}

// ---------------------------------------------------------------------------
// Mixed-precision iterative refinement (cg_mode MIXED).
//
// With S = diag(M)^-1/2 the scaled matrix A = S M S has unit diagonal. For P1
// elements the element mass matrix against its own diagonal has eigenvalues
// in [1/2, 2] (triangles) or [1/2, 5/2] (tetrahedra), and the assembled
// matrix inherits the union of the element bounds, so cond(A) <= 4 or 5 on
// any mesh: an FP32 solve on A converges like Jacobi-PCG in FP64 on M, and
// its attainable accuracy (~ eps32 cond(A)) is far below the per-cycle target.
// One refinement cycle:
//   R (FP64)  r = b - M x, t = S r, ||r||_2 (the stopping test) and ||t||_2;
//   I         c = t / ||t||_2 rounded to FP32 (unit norm), y = 0;
//   inner (FP32) on A y = c to ||c - A y||_2 <= eta, eta about the reduction
//             the stopping test still needs (between 1e-5 and 1/4): the
//             Chebyshev iteration over the spectrum interval (the step count
//             the interval fixes for eta; util.cuh), or CG until its
//             recurrence residual reaches eta when built with
//             SFT_MIX_CHEBYSHEV=0;
//   U (FP64)  x += ||t||_2 S y   (so the new residual is ||t|| S^-1 (c - A y)).
// A warm start takes x as given (||b|| is then reduced separately first) and
// skips nothing else: the first R phase checks whether x already converged.
// The FP64 pipe does one SpMV per cycle (2 to 3 cycles) instead of one per
// iteration. Every block takes every decision from the same fixed-order
// reductions; the stopping test uses the true FP64 residual.
// smallest inner reduction asked of one FP32 solve (measured: 1e-5 gives
// 0.71 / 0.68 ms on the 1.0 M-row 2D / 0.5 M-row 3D systems, 3e-6 and 1e-6
// 0.74 / 0.71 ms: deeper FP32 solves cost more iterations than the extra
// refinement cycle they save)
#ifndef SFT_MIX_ETA_FLOOR
#define SFT_MIX_ETA_FLOOR 1e-5f
#endif
constexpr float kEtaFloor = SFT_MIX_ETA_FLOOR;
#ifndef SFT_MIX_ROWS_PER_THREAD
#define SFT_MIX_ROWS_PER_THREAD 3
#endif


struct MixCtl {
  GridBarrier bar;
  int32_t err;
  int32_t cycles;
  int32_t iters[kMaxFields];
  double rel[kMaxFields];
  int32_t conv[kMaxFields];
};

template <int NR>
__device__ __forceinline__ void block_partials_d(const double (&v)[NR][2], int nrhs, double* part) {
  __shared__ double sh[kSolveThreads / 32][NR][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int f = 0; f < NR; ++f) {
    if (f >= nrhs) break;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const double w = warp_sum<double>(v[f][c]);
      if (lane == 0) sh[warp][f][c] = w;
    }
  }
  __syncthreads();
  if (threadIdx.x < nrhs * 2) {
    const int f = threadIdx.x >> 1, c = threadIdx.x & 1;
    double s = 0.0;
    for (int w = 0; w < kSolveThreads / 32; ++w) s += sh[w][f][c];
    part[((int64_t)blockIdx.x * nrhs + f) * 2 + c] = s;
  }
  __syncthreads();
}

template <int NR>
__device__ __forceinline__ void block_partials_f(const float (&v)[NR], int nrhs, float* part) {
  __shared__ float sh[kSolveThreads / 32][NR];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int f = 0; f < NR; ++f) {
    if (f >= nrhs) break;
    const float w = warp_sum<float>(v[f]);
    if (lane == 0) sh[warp][f] = w;
  }
  __syncthreads();
  if (threadIdx.x < nrhs) {
    float s = 0.f;
    for (int w = 0; w < kSolveThreads / 32; ++w) s += sh[w][threadIdx.x];
    part[(int64_t)blockIdx.x * nrhs + threadIdx.x] = s;
  }
  __syncthreads();
}

// sum the FP32 partials [nblocks][nrhs] in a fixed order (identical in all blocks)
template <int NR>
__device__ __forceinline__ void reduce_partials_f(const float* part, int nblocks, int nrhs, float* sh_tot) {
  __shared__ float shw[kSolveThreads / 32][NR];
  float acc[NR];
#pragma unroll
  for (int f = 0; f < NR; ++f) acc[f] = 0.f;
  for (int bidx = threadIdx.x; bidx < nblocks; bidx += blockDim.x) {
    const float* pb = part + (int64_t)bidx * nrhs;
#pragma unroll
    for (int f = 0; f < NR; ++f)
      if (f < nrhs) acc[f] += __ldcg(pb + f);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int f = 0; f < NR; ++f) {
    if (f >= nrhs) break;
    const float w = warp_sum<float>(acc[f]);
    if (lane == 0) shw[warp][f] = w;
  }
  __syncthreads();
  if (threadIdx.x < nrhs) {
    float t = 0.f;
    for (int w = 0; w < kSolveThreads / 32; ++w) t += shw[w][threadIdx.x];
    sh_tot[threadIdx.x] = t;
  }
  __syncthreads();
}

// NR: compile-time bound on the number of right-hand sides (nrhs <= NR).
// Four resident blocks per SM (64 registers a thread): 0.69 ms on the 1.0 M-row
// 2D system against 0.78 ms with the compiler's own register choice (48 and
// spills). Interleaving 2, 4 or 8 of a thread's rows (overlapping their load
// chains) measured no better (0.69 / 0.71 / 0.91 ms).
template <int NR>
__global__ void __launch_bounds__(kSolveThreads, 4) k_mixed_cg(
    const int32_t* __restrict__ rp, const int32_t* __restrict__ col, const double* __restrict__ val,
    const float* __restrict__ aval, const double* __restrict__ sc, int64_t n, int nrhs,
    const double* __restrict__ b, double* x, double* t, float* r, float* p, float* q, float* y, double* partd,
    float* partf, MixCtl* ctl, double tol, int max_iter, int warm, uint64_t wait_ns, float lmax) {
  __shared__ double totd[kMaxFields * 2];
  __shared__ float totf[NR];
  __shared__ double bnorm[NR], prev[NR], sig[NR], isig[NR];
  __shared__ float eta2[NR], rr[NR], alpha[NR], beta[NR];
  __shared__ int live[NR], act[NR], conv[NR], ksteps[NR], stop;
  const ChebCoef ch = cheb_coef(lmax);
  const unsigned nb = gridDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int f = 0; f < NR; ++f) {
      live[f] = f < nrhs;
      act[f] = 0;
      conv[f] = 0;
    }
  }
  __syncthreads();
  int it = 0, cyc = 0;
  if (warm) {
    // warm start from the x given: ||b|| for the stopping test first
    double v[NR][2];
#pragma unroll
    for (int f = 0; f < NR; ++f) v[f][0] = v[f][1] = 0.0;
    for (int64_t i = tid; i < n; i += nthreads) {
#pragma unroll
      for (int f = 0; f < NR; ++f) {
        if (f >= nrhs) break;
        const double bi = b[(int64_t)f * n + i];
        v[f][0] += bi * bi;
      }
    }
    block_partials_d<NR>(v, nrhs, partd);
    if (!grid_sync(&ctl->bar, nb, &ctl->err, wait_ns)) return;
    reduce_partials(partd, nb, nrhs, totd);
    if (threadIdx.x == 0)
      for (int f = 0; f < nrhs; ++f) bnorm[f] = sqrt(totd[2 * f]);
    __syncthreads();
  }
  for (;; ++cyc) {
    // R: true residual in FP64 (x = 0 in the first cycle unless warm)
    double v[NR][2];
#pragma unroll
    for (int f = 0; f < NR; ++f) v[f][0] = v[f][1] = 0.0;
    for (int64_t i = tid; i < n; i += nthreads) {
      const double si = sc[i];
      int32_t k0 = 0, k1 = 0;
      if (cyc > 0 || warm) {
        k0 = __ldg(rp + i);
        k1 = __ldg(rp + i + 1);
      }
#pragma unroll
      for (int f = 0; f < NR; ++f) {
        if (f >= nrhs) break;
        if (!live[f]) continue;
        const int64_t o = (int64_t)f * n;
        double s = 0.0;
        // x was written by other blocks before the grid barrier (plain loads)
        for (int32_t k = k0; k < k1; ++k) s += __ldg(val + k) * x[o + __ldg(col + k)];
        if (cyc == 0 && !warm) x[o + i] = 0.0;
        const double ri = b[o + i] - s;
        const double ti = si * ri;
        t[o + i] = ti;
        v[f][0] += ri * ri;
        v[f][1] += ti * ti;
      }
    }
    block_partials_d<NR>(v, nrhs, partd);
    if (!grid_sync(&ctl->bar, nb, &ctl->err, wait_ns)) return;
    reduce_partials(partd, nb, nrhs, totd);
    if (threadIdx.x == 0) {
      bool any = false;
      for (int f = 0; f < nrhs; ++f) {
        act[f] = 0;
        if (!live[f]) continue;
        const double rn = sqrt(totd[2 * f]), tn = sqrt(totd[2 * f + 1]);
        if (cyc == 0 && !warm) bnorm[f] = rn;
        if (blockIdx.x == 0) {
          ctl->rel[f] = bnorm[f] > 0.0 ? rn / bnorm[f] : 0.0;
          ctl->iters[f] = it;
        }
        if (rn <= tol * bnorm[f]) {
          live[f] = 0;
          conv[f] = 1;
          continue;
        }
        // a cycle that did not halve the residual (FP64 rounding floor) or a
        // residual on rows without diagonal ends the field unconverged
        if ((cyc > 0 && rn > 0.5 * prev[f]) || !(tn > 0.0)) {
          live[f] = 0;
          continue;
        }
        prev[f] = rn;
        sig[f] = tn;
        isig[f] = 1.0 / tn;
        const double e = fmin(0.25, fmax((double)kEtaFloor, 0.1 * tol * bnorm[f] / rn));
        eta2[f] = (float)(e * e);
        ksteps[f] = cheb_steps(e, ch.s1);
        act[f] = 1;
        any = true;
      }
      stop = !any || it >= max_iter;
    }
    __syncthreads();
    if (stop) break;

    if constexpr (kMixCheb) {
      // I: c = t / ||t|| in FP32, r = c, y = 0, d = c / theta (in p)
      const float ith = 1.f / ch.theta;
      for (int64_t i = tid; i < n; i += nthreads) {
#pragma unroll
        for (int f = 0; f < NR; ++f) {
          if (f >= nrhs) break;
          if (!act[f]) continue;
          const int64_t k = (int64_t)f * n + i;
          const float ci = (float)(t[k] * isig[f]);
          r[k] = ci;
          y[k] = 0.f;
          p[k] = ci * ith;
        }
      }
      if (!grid_sync(&ctl->bar, nb, &ctl->err, wait_ns)) return;
      // Chebyshev steps; d alternates between p and q (the SpMV of a step
      // reads the d every block wrote in the step before)
      float rho = 1.f / ch.s1;
      const float idl = 2.f / ch.delta;
      auto steps_left = [&](int s) {  // fields that take step s
        unsigned mm = 0u;
#pragma unroll
        for (int f = 0; f < NR; ++f)
          if (f < nrhs && act[f] && s < ksteps[f]) mm |= 1u << f;
        return it < max_iter ? mm : 0u;
      };
      for (int s = 0;; ++s) {
        const unsigned m = steps_left(s);
        if (!m) break;
        const float rn1 = 1.f / (2.f * ch.s1 - rho);
        const float c1 = rn1 * rho, c2 = rn1 * idl;
        const float* dc = (s & 1) ? q : p;
        float* dn = (s & 1) ? p : q;
        for (int64_t i = tid; i < n; i += nthreads) {
          const int32_t k0 = __ldg(rp + i), k1 = __ldg(rp + i + 1);
#pragma unroll
          for (int f = 0; f < NR; ++f) {
            if (f >= nrhs) break;
            if (!((m >> f) & 1u)) continue;
            const int64_t o = (int64_t)f * n;
            const float* df = dc + o;
            float w = 0.f;
            // d was written by other blocks before the grid barrier (plain loads)
            for (int32_t k = k0; k < k1; ++k) w += __ldg(aval + k) * df[__ldg(col + k)];
            const float di = df[i];
            y[o + i] += di;
            const float ri = r[o + i] - w;
            r[o + i] = ri;
            dn[o + i] = c1 * di + c2 * ri;
          }
        }
        rho = rn1;
        ++it;
        // the next step's SpMV reads the d of other blocks; after the last
        // step U touches only the thread's own rows, so no barrier
        if (!steps_left(s + 1)) break;
        if (!grid_sync(&ctl->bar, nb, &ctl->err, wait_ns)) return;
      }
    } else {
      // I: unit-norm FP32 right-hand side, zero iterate and directions
      float vf[NR];
#pragma unroll
      for (int f = 0; f < NR; ++f) vf[f] = 0.f;
      for (int64_t i = tid; i < n; i += nthreads) {
#pragma unroll
        for (int f = 0; f < NR; ++f) {
          if (f >= nrhs) break;
          if (!act[f]) continue;
          const int64_t k = (int64_t)f * n + i;
          const float ci = (float)(t[k] * isig[f]);
          r[k] = ci;
          y[k] = 0.f;
          p[k] = 0.f;
          q[k] = 0.f;
          vf[f] += ci * ci;
        }
      }
      block_partials_f<NR>(vf, nrhs, partf);
      if (!grid_sync(&ctl->bar, nb, &ctl->err, wait_ns)) return;
      reduce_partials_f<NR>(partf, nb, nrhs, totf);
      if (threadIdx.x == 0)
        for (int f = 0; f < nrhs; ++f) {
          rr[f] = totf[f];
          beta[f] = 0.f;
        }
      __syncthreads();

      // CG in FP32 on A y = c
      for (;;) {
        bool any = false;
#pragma unroll
        for (int f = 0; f < NR; ++f)
          if (f < nrhs) any = any || act[f];
        if (!any || it >= max_iter) break;
        // phase A: w = A r, p = r + beta p, q = w + beta q (= A p), partial (p, q)
#pragma unroll
        for (int f = 0; f < NR; ++f) vf[f] = 0.f;
        for (int64_t i = tid; i < n; i += nthreads) {
          const int32_t k0 = __ldg(rp + i), k1 = __ldg(rp + i + 1);
#pragma unroll
          for (int f = 0; f < NR; ++f) {
            if (f >= nrhs) break;
            if (!act[f]) continue;
            const int64_t o = (int64_t)f * n;
            const float* rf = r + o;
            float s = 0.f;
            // r was written by other blocks before the grid barrier (plain loads)
            for (int32_t k = k0; k < k1; ++k) s += __ldg(aval + k) * rf[__ldg(col + k)];
            const float bt = beta[f];
            const int64_t k = o + i;
            const float pn = rf[i] + bt * p[k];
            const float qn = s + bt * q[k];
            p[k] = pn;
            q[k] = qn;
            vf[f] += pn * qn;
          }
        }
        block_partials_f<NR>(vf, nrhs, partf);
        if (!grid_sync(&ctl->bar, nb, &ctl->err, wait_ns)) return;
        reduce_partials_f<NR>(partf, nb, nrhs, totf);
        if (threadIdx.x == 0)
          for (int f = 0; f < nrhs; ++f) alpha[f] = act[f] ? rr[f] / totf[f] : 0.f;
        __syncthreads();
        // phase B: y += alpha p, r -= alpha q, partial (r, r)
#pragma unroll
        for (int f = 0; f < NR; ++f) vf[f] = 0.f;
        for (int64_t i = tid; i < n; i += nthreads) {
#pragma unroll
          for (int f = 0; f < NR; ++f) {
            if (f >= nrhs) break;
            if (!act[f]) continue;
            const int64_t k = (int64_t)f * n + i;
            const float a = alpha[f];
            y[k] += a * p[k];
            const float ri = r[k] - a * q[k];
            r[k] = ri;
            vf[f] += ri * ri;
          }
        }
        block_partials_f<NR>(vf, nrhs, partf);
        if (!grid_sync(&ctl->bar, nb, &ctl->err, wait_ns)) return;
        reduce_partials_f<NR>(partf, nb, nrhs, totf);
        ++it;
        if (threadIdx.x == 0)
          for (int f = 0; f < nrhs; ++f) {
            if (!act[f]) continue;
            const float rn = totf[f];
            beta[f] = rn / rr[f];
            rr[f] = rn;
            if (rn <= eta2[f]) act[f] = 0;
          }
        __syncthreads();
      }
    }

    // U: x += ||t|| S y for every field that ran this cycle
    for (int64_t i = tid; i < n; i += nthreads) {
      const double si = sc[i];
#pragma unroll
      for (int f = 0; f < NR; ++f) {
        if (f >= nrhs) break;
        if (!live[f]) continue;
        const int64_t k = (int64_t)f * n + i;
        x[k] += (sig[f] * si) * (double)y[k];
      }
    }
    if (!grid_sync(&ctl->bar, nb, &ctl->err, wait_ns)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    ctl->cycles = cyc;
    for (int f = 0; f < nrhs; ++f) ctl->conv[f] = conv[f];
  }
}

// S = diag(M)^-1/2 (0 on a row without diagonal) and the FP32 scaled values
__global__ void k_jacobi_sqrt(const double* __restrict__ dinv, int64_t n, double* __restrict__ sc) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    sc[i] = sqrt(dinv[i]);
}

__global__ void k_scaled_values(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ sc, int64_t n,
                                float* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double si = sc[i];
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k) out[k] = (float)(val[k] * si * sc[col[k]]);
  }
}

sft_status scaled_matrix(sft_target_s* t, cudaStream_t st) {
  if (t->val32s) return SFT_OK;
  const int64_t n = t->nv;
  SFT_CUDA(dalloc(&t->sc, (size_t)n, st));
  SFT_CUDA(dalloc(&t->val32s, (size_t)std::max<int64_t>(t->nnz, 1), st));
  const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 16));
  ::sft::note_launch(), k_jacobi_sqrt<<<nb, 256, 0, st>>>(t->dinv, n, t->sc);
  SFT_CUDA(cudaGetLastError());
  ::sft::note_launch(), k_scaled_values<<<nb, 256, 0, st>>>(t->row_ptr, t->col, t->val, t->sc, n, t->val32s);
  SFT_CUDA(cudaGetLastError());
  return SFT_OK;
}

static_assert(sizeof(MixCtl) <= sizeof(SolveLate::host), "status block larger than its host copy");

static void mix_result(const MixCtl& h, int nrhs, SolveResult* res) {
  for (int f = 0; f < nrhs; ++f) {
    res->iters = std::max(res->iters, (int)h.iters[f]);
    res->rel_resid = std::max(res->rel_resid, h.rel[f]);
    if (!h.conv[f]) res->converged = 0;
  }
}

sft_status finish_solve(const SolveLate& late, SolveResult* res) {
  if (!late.pending) return SFT_OK;
  MixCtl h;
  std::memcpy(&h, late.host, sizeof(MixCtl));
  if (h.err != 0) return fail(SFT_ERR_DEVICE_STATUS, "CG kernel: grid barrier wait expired");
  mix_result(h, late.nrhs, res);
  return SFT_OK;
}

template <int NR>
static sft_status launch_mixed(sft_target_s* t, int nrhs, const double* b, double* x, double tol, int max_iter,
                               cudaStream_t st, SolveResult* res, SolveLate* late, int warm) {
  const int64_t n = t->nv;
  // largest eigenvalue bound of S M S: 2 for triangles, 5/2 for tetrahedra
  float lmax = t->dim == 2 ? 2.f : 2.5f;
  int dev = 0, sms = 0;
  SFT_CUDA(cudaGetDevice(&dev));
  SFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int per_sm = 0;
  SFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mixed_cg<NR>, kSolveThreads, 0));
  if (per_sm < 1) return fail(SFT_ERR_CUDA, "solver kernel cannot be resident");
  per_sm = std::min(per_sm, 4);
  // as many resident blocks as ~3 rows per thread allows: measured 0.78 /
  // 0.71 ms (1.0 M-row 2D / 0.5 M-row 3D systems) at 3 rows, 0.78 / 0.76 at
  // 6, 1.04 / 1.06 at 12 (the FP32 phases are latency-bound, not FP64-bound)
  constexpr int64_t kRows = SFT_MIX_ROWS_PER_THREAD;
  const int64_t want = (n + kSolveThreads * kRows - 1) / (kSolveThreads * kRows);
  const unsigned nblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sms, want));
  const size_t vec = (size_t)n * nrhs;
  DevBuf<double> tb(st), partd(st);
  DevBuf<float> rb(st), pb(st), qb(st), yb(st), partf(st);
  DevBuf<MixCtl> ctl(st);
  SFT_CUDA(tb.alloc(vec));
  SFT_CUDA(rb.alloc(vec));
  SFT_CUDA(pb.alloc(vec));
  SFT_CUDA(qb.alloc(vec));
  SFT_CUDA(yb.alloc(vec));
  SFT_CUDA(partd.alloc((size_t)nblocks * nrhs * 2));
  SFT_CUDA(partf.alloc((size_t)nblocks * nrhs));
  MixCtl* c = nullptr;
  if (late) {
    SFT_CUDA(late->buf.alloc(sizeof(MixCtl)));
    c = reinterpret_cast<MixCtl*>(late->buf.p);
  } else {
    SFT_CUDA(ctl.alloc(1));
    c = ctl.p;
  }
  SFT_CUDA(cudaMemsetAsync(c, 0, sizeof(MixCtl), st));
  const int32_t* rp = t->row_ptr;
  const int32_t* col = t->col;
  const double* val = t->val;
  const float* aval = t->val32s;
  const double* sc = t->sc;
  double* tp = tb.p;
  float *r = rb.p, *p = pb.p, *q = qb.p, *y = yb.p;
  double* pd = partd.p;
  float* pf = partf.p;
  void* args[] = {(void*)&rp, (void*)&col, (void*)&val, (void*)&aval, (void*)&sc, (void*)&n, (void*)&nrhs,
                  (void*)&b, (void*)&x, (void*)&tp, (void*)&r, (void*)&p, (void*)&q, (void*)&y,
                  (void*)&pd, (void*)&pf, (void*)&c, (void*)&tol, (void*)&max_iter, (void*)&warm,
                  (void*)&t->wait_ns, (void*)&lmax};
  const cudaError_t le = (::sft::note_launch(), cudaLaunchCooperativeKernel((const void*)k_mixed_cg<NR>, nblocks,
                                                                           kSolveThreads, args, 0, st));
  if (le != cudaSuccess) return cuda_fail(le, "cudaLaunchCooperativeKernel(k_mixed_cg)");
  if (late) {
    late->bytes = sizeof(MixCtl);
    late->nrhs = nrhs;
    late->pending = true;
    return SFT_OK;  // the work buffers are freed in stream order
  }
  MixCtl h;
  SFT_CUDA(cudaMemcpyAsync(&h, ctl.p, sizeof(MixCtl), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  if (h.err != 0) return fail(SFT_ERR_DEVICE_STATUS, "CG kernel: grid barrier wait expired");
  mix_result(h, nrhs, res);
  return SFT_OK;
}

sft_status mass_solve(sft_target_s* t, int nrhs, const double* b, double* x, double tol, int max_iter,
                      cudaStream_t st, int32_t* d_err, SolveResult* res, int cg_mode, SolveLate* late, int warm) {
  (void)d_err;
  res->iters = 0;
  res->rel_resid = 0.0;
  res->converged = 1;
  const int64_t n = t->nv;
  if (n == 0 || nrhs == 0) return SFT_OK;
  if (nrhs > kMaxFields) return fail(SFT_ERR_ARG, "at most 8 right-hand sides");
  if (max_iter <= 0) {
    SFT_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n * nrhs, st));
    res->converged = 0;
    return SFT_OK;
  }
  if (warm && cg_mode != SFT_CG_MIXED) return fail(SFT_ERR_UNSUPPORTED, "a warm start needs cg_mode MIXED");
  if (cg_mode == SFT_CG_MIXED) {
    if (sft_status r = scaled_matrix(t, st)) return r;
    if (nrhs == 1) return launch_mixed<1>(t, nrhs, b, x, tol, max_iter, st, res, late, warm);
    if (nrhs == 2) return launch_mixed<2>(t, nrhs, b, x, tol, max_iter, st, res, late, warm);
    if (nrhs <= 4) return launch_mixed<4>(t, nrhs, b, x, tol, max_iter, st, res, late, warm);
    return launch_mixed<8>(t, nrhs, b, x, tol, max_iter, st, res, late, warm);
  }
  int dev = 0, sms = 0, coop = 0;
  SFT_CUDA(cudaGetDevice(&dev));
  SFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SFT_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return fail(SFT_ERR_UNSUPPORTED, "device lacks cooperative launch");
  // one thread per row: the FP64 pipe (1 warp instruction / 16 cycles / SM
  // here) is the limiter, and a row-per-thread SpMV issues one DFMA warp
  // instruction per nonzero for 32 rows, with no shuffle reductions
  int per_sm = 0;
  SFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<1>, kSolveThreads, 0));
  if (per_sm < 1) return fail(SFT_ERR_CUDA, "solver kernel cannot be resident");
  per_sm = std::min(per_sm, 4);
  // at least ~6 rows per thread: fewer blocks make the two grid barriers and
  // the partial sums of every iteration cheaper (measured: 4 blocks per SM
  // for the 1.0 M-row 2D system, about 2 for the 0.5 M-row 3D one)
  constexpr int64_t kRowsPerThread = 6;
  const int64_t want = (n + kSolveThreads * kRowsPerThread - 1) / (kSolveThreads * kRowsPerThread);
  const unsigned nblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sms, want));

  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *part = nullptr;
  PcgCtl* ctl = nullptr;
  const size_t vec = (size_t)n * nrhs;
  SFT_CUDA(dalloc(&r, vec, st));
  SFT_CUDA(dalloc(&z, vec, st));
  SFT_CUDA(dalloc(&p, vec, st));
  SFT_CUDA(dalloc(&q, vec, st));
  SFT_CUDA(dalloc(&part, (size_t)nblocks * nrhs * 2, st));
  SFT_CUDA(dalloc(&ctl, 1, st));
  SFT_CUDA(cudaMemsetAsync(ctl, 0, sizeof(PcgCtl), st));
  const int32_t* rp = t->row_ptr;
  const int32_t* col = t->col;
  const double* val = t->val;
  const double* dinv = t->dinv;
  void* args[] = {(void*)&rp, (void*)&col, (void*)&val, (void*)&dinv, (void*)&n, (void*)&nrhs, (void*)&b,
                  (void*)&x, (void*)&r, (void*)&z, (void*)&p, (void*)&q, (void*)&part,
                  (void*)&ctl, (void*)&tol, (void*)&max_iter, (void*)&t->wait_ns};
  cudaError_t le;
  le = (::sft::note_launch(), cudaLaunchCooperativeKernel((const void*)k_pcg<1>, nblocks, kSolveThreads, args, 0, st));
  if (le != cudaSuccess) return cuda_fail(le, "cudaLaunchCooperativeKernel(k_pcg)");
  PcgCtl h;
  SFT_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  dfree(r, st); dfree(z, st); dfree(p, st); dfree(q, st); dfree(part, st); dfree(ctl, st);
  if (h.err != 0) return fail(SFT_ERR_DEVICE_STATUS, "CG kernel: grid barrier wait expired");
  for (int f = 0; f < nrhs; ++f) {
    res->iters = std::max(res->iters, (int)h.iters[f]);
    res->rel_resid = std::max(res->rel_resid, h.rel[f]);
    if (!h.conv[f]) res->converged = 0;
  }
  return SFT_OK;
}

// deterministic FP64 sum of w_i u_i (the integral of a P1 target field with lumped masses)
__global__ void k_wsum_partial(const double* __restrict__ w, const double* __restrict__ u, int64_t n,
                               double* __restrict__ part) {
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    s += w[i] * u[i];
  __shared__ double sh[8];
  s = warp_sum<double>(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x / 32); ++k) t += sh[k];
    part[blockIdx.x] = t;
  }
}

sft_status weighted_sum_launch(const double* w, const double* u, int64_t n, double* part, cudaStream_t st) {
  ::sft::note_launch(), k_wsum_partial<<<kWsumBlocks, 256, 0, st>>>(w, u, n, part);
  SFT_CUDA(cudaGetLastError());
  return SFT_OK;
}

double weighted_sum_finish(const double* hpart) {
  double t = 0.0;
  for (unsigned k = 0; k < kWsumBlocks; ++k) t += hpart[k];
  return t;
}

sft_status weighted_sum(const double* w, const double* u, int64_t n, double* out_host, cudaStream_t st) {
  DevBuf<double> part(st);
  SFT_CUDA(part.alloc(kWsumBlocks));
  if (sft_status r = weighted_sum_launch(w, u, n, part.p, st)) return r;
  std::vector<double> h(kWsumBlocks);
  SFT_CUDA(cudaMemcpyAsync(h.data(), part.p, sizeof(double) * kWsumBlocks, cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  *out_host = weighted_sum_finish(h.data());
  return SFT_OK;
}

}  // namespace sft

// ---------------------------------------------------------------------------
// Allocation-free variant of the CG solve (no counterpart in the paper).
//
// Some callers cannot allocate device memory when they need a solve: for
// example a coupled simulation that hands all device memory to its own pool
// up front, or a time-stepping loop that must not call cudaMalloc/cudaFree
// because they synchronise the device and can fail mid-run. This entry point
// takes the CSR matrix, right-hand sides and solution buffers from the caller
// and keeps its work vectors in one fixed, file-scope device array instead.
// ---------------------------------------------------------------------------
namespace sft {

// 32 MiB of work space, resident on every device that loads the library
constexpr size_t kStaticScratchBytes = 32ull << 20;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

static std::mutex g_static_mu;
static void* g_static_ptr[64] = {nullptr};

// Device address of the scratch array for the current device: looked up once
// per device (with that device current) and cached.
static sft_status static_scratch(void** out) {
  int dev = 0;
  SFT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return fail(SFT_ERR_UNSUPPORTED, "device ordinal >= 64");
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return SFT_OK;
}

// Jacobi inverse of the caller's matrix; a row without a positive diagonal
// entry (the matrix cannot be SPD) sets DEV_BAD_DIAGONAL, reported as
// SFT_ERR_ARG (the CG kernel sees the error word and leaves at its first
// barrier)
__global__ void k_jacobi_inverse(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, int64_t n, double* __restrict__ dinv,
                                 int32_t* err) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (col[k] == i) d = val[k];
    if (!(d > 0.0)) set_error(err, DEV_BAD_DIAGONAL);
    dinv[i] = d > 0.0 ? 1.0 / d : 0.0;
  }
}

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace sft

extern "C" sft_status sft_mass_solve_static(int64_t n, const int32_t* row_ptr, const int32_t* col,
                                            const double* val, int32_t nrhs, const double* b, double* u,
                                            double tol, int32_t max_iter, void* cuda_stream,
                                            int32_t* iters_out, double* rel_resid_out) {
  using namespace sft;
  if (n <= 0 || !row_ptr || !col || !val || !b || !u) return fail(SFT_ERR_ARG, "null argument or n <= 0");
  if (nrhs < 1 || nrhs > kMaxFields) return fail(SFT_ERR_ARG, "nrhs must be in 1..8");
  if (max_iter < 1 || !(tol >= 0)) return fail(SFT_ERR_ARG, "bad solver options");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0, sms = 0, coop = 0;
  SFT_CUDA(cudaGetDevice(&dev));
  SFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  SFT_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  if (!coop) return fail(SFT_ERR_UNSUPPORTED, "device lacks cooperative launch");
  int per_sm = 0;
  SFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<1>, kSolveThreads, 0));
  if (per_sm < 1) return fail(SFT_ERR_CUDA, "solver kernel cannot be resident");
  per_sm = std::min(per_sm, 4);
  // at least ~6 rows per thread: fewer blocks make the two grid barriers and
  // the partial sums of every iteration cheaper (measured: 4 blocks per SM
  // for the 1.0 M-row 2D system, about 2 for the 0.5 M-row 3D one)
  constexpr int64_t kRowsPerThread = 6;
  const int64_t want = (n + kSolveThreads * kRowsPerThread - 1) / (kSolveThreads * kRowsPerThread);
  const unsigned nblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * sms, want));
  // layout: dinv [n] | r, z, p, q [nrhs][n] | partials [nblocks][nrhs][2] | control block
  const size_t vec = sizeof(double) * (size_t)n * nrhs;
  const size_t off_dinv = 0;
  const size_t off_r = align256(off_dinv + sizeof(double) * (size_t)n);
  const size_t off_z = align256(off_r + vec);
  const size_t off_p = align256(off_z + vec);
  const size_t off_q = align256(off_p + vec);
  const size_t off_part = align256(off_q + vec);
  const size_t off_ctl = align256(off_part + sizeof(double) * (size_t)nblocks * nrhs * 2);
  const size_t need = off_ctl + sizeof(PcgCtl);
  if (need > kStaticScratchBytes)
    return fail(SFT_ERR_ARG, "problem too large for the 32 MiB static work space: needs 8 n (1 + 4 nrhs) bytes "
                             "plus partials (n * (1 + 4 nrhs) <= ~4.1e6)");
  void* base = nullptr;
  if (sft_status r = static_scratch(&base)) return r;
  unsigned char* s = static_cast<unsigned char*>(base);
  double* dinv = reinterpret_cast<double*>(s + off_dinv);
  double* r = reinterpret_cast<double*>(s + off_r);
  double* z = reinterpret_cast<double*>(s + off_z);
  double* p = reinterpret_cast<double*>(s + off_p);
  double* q = reinterpret_cast<double*>(s + off_q);
  double* part = reinterpret_cast<double*>(s + off_part);
  PcgCtl* ctl = reinterpret_cast<PcgCtl*>(s + off_ctl);
  // the barrier counters and error word must start at zero; every other
  // region is written by the kernels before it is read
  SFT_CUDA(cudaMemsetAsync(ctl, 0, sizeof(PcgCtl), st));
  ::sft::note_launch(), k_jacobi_inverse<<<(unsigned)std::min<int64_t>((n + 255) / 256, 152 * 16), 256, 0, st>>>(
      row_ptr, col, val, n, dinv, &ctl->err);
  SFT_CUDA(cudaGetLastError());
  const double* dinv_c = dinv;
  const uint64_t wait_ns = kDefaultWaitNs;
  void* args[] = {(void*)&row_ptr, (void*)&col, (void*)&val, (void*)&dinv_c, (void*)&n, (void*)&nrhs, (void*)&b,
                  (void*)&u, (void*)&r, (void*)&z, (void*)&p, (void*)&q, (void*)&part,
                  (void*)&ctl, (void*)&tol, (void*)&max_iter, (void*)&wait_ns};
  const cudaError_t le =
      (::sft::note_launch(), cudaLaunchCooperativeKernel((const void*)k_pcg<1>, nblocks, kSolveThreads, args, 0, st));
  if (le != cudaSuccess) return cuda_fail(le, "cudaLaunchCooperativeKernel(k_pcg, static scratch)");
  PcgCtl h;
  SFT_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  if (h.err == DEV_BAD_DIAGONAL) return fail(SFT_ERR_ARG, "a row has no positive diagonal entry (matrix not SPD)");
  if (h.err != 0) return fail(SFT_ERR_DEVICE_STATUS, "CG kernel: grid barrier wait expired");
  int it = 0, conv = 1;
  double rel = 0.0;
  for (int f = 0; f < nrhs; ++f) {
    it = std::max(it, (int)h.iters[f]);
    rel = std::max(rel, h.rel[f]);
    if (!h.conv[f]) conv = 0;
  }
  if (iters_out) *iters_out = it;
  if (rel_resid_out) *rel_resid_out = rel;
  if (!conv) return fail(SFT_ERR_NOT_CONVERGED, "CG reached max_iter");
  return SFT_OK;
}
