// Step 7 of Sec. 4: solve the target Galerkin system M u = b (Eq.
// cv_galerkin_system) in FP64 with Jacobi-preconditioned CG from u = 0,
// stopping at ||b - M u||_2 <= tol ||b||_2 (the paper does not name its
// solver; see the design notes).
//
// One cooperative (co-resident) kernel runs the whole iteration: no host round
// trip per step. Each iteration has two grid barriers:
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
                                                       int max_iter) {
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
  if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
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
    if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
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
    if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
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

sft_status mass_solve(sft_target_s* t, int nrhs, const double* b, double* x, double tol, int max_iter,
                      cudaStream_t st, int32_t* d_err, SolveResult* res) {
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
                  (void*)&ctl, (void*)&tol, (void*)&max_iter};
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

sft_status weighted_sum(const double* w, const double* u, int64_t n, double* out_host, cudaStream_t st) {
  const unsigned nb = 304;
  double* part = nullptr;
  SFT_CUDA(dalloc(&part, nb, st));
  ::sft::note_launch(), k_wsum_partial<<<nb, 256, 0, st>>>(w, u, n, part);
  SFT_CUDA(cudaGetLastError());
  std::vector<double> h(nb);
  SFT_CUDA(cudaMemcpyAsync(h.data(), part, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  dfree(part, st);
  double t = 0.0;
  for (unsigned k = 0; k < nb; ++k) t += h[k];
  *out_host = t;
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

__global__ void k_jacobi_inverse(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                                 const double* __restrict__ val, int64_t n, double* __restrict__ dinv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double d = 0.0;
    for (int32_t k = rp[i]; k < rp[i + 1]; ++k)
      if (col[k] == i) d = val[k];
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
      row_ptr, col, val, n, dinv);
  SFT_CUDA(cudaGetLastError());
  const double* dinv_c = dinv;
  void* args[] = {(void*)&row_ptr, (void*)&col, (void*)&val, (void*)&dinv_c, (void*)&n, (void*)&nrhs, (void*)&b,
                  (void*)&u, (void*)&r, (void*)&z, (void*)&p, (void*)&q, (void*)&part,
                  (void*)&ctl, (void*)&tol, (void*)&max_iter};
  const cudaError_t le =
      (::sft::note_launch(), cudaLaunchCooperativeKernel((const void*)k_pcg<1>, nblocks, kSolveThreads, args, 0, st));
  if (le != cudaSuccess) return cuda_fail(le, "cudaLaunchCooperativeKernel(k_pcg, static scratch)");
  PcgCtl h;
  SFT_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(PcgCtl), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
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
