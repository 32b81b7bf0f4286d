// Batched transfers: many (source, target, options) requests of uneven size
// run together (Sec. 4 steps 1-7 per request; batching itself has no
// counterpart in the paper). A plan groups the requests by dimension and
// field-count class and records one CUDA graph:
//   1. control values of every request      (k_batch_control, one per dim)
//   2. fused assembly of every request      (k_batch_assemble, persistent, one per group:
//      warps pull (request, element-task) tiles from an atomic work counter)
//   3. one cooperative solve of the block-diagonal system of every
//      (request, field) right-hand side     (k_batch_mixed: mixed-precision
//      refinement, the default; k_batch_pcg: FP64 CG when a request asks)
// The tile size of each group is chosen by a small autotuner (timed trial
// launches, cached per process and optionally in a file).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>
#include "internal.hpp"
#include "util.cuh"

namespace sft {

constexpr int kMaxBatch = 4096;
constexpr int kBatchThreads = 256;

// one request, FP32 path (device copy)
struct BReq {
  const float* tx;
  const int32_t* tconn;
  const float* vol32;
  int64_t nv, ne;
  const GridP<float>* grid;
  const int32_t* cell_start;
  const int32_t* cell_items;
  const int32_t* cell_first;
  const float* recs;
  const int32_t* adj;
  const float* vals;
  int32_t snf;  // the source's field count (stride of its value copies)
  int32_t nf, N, U, G, LPE;
  int64_t ntasks;
  PhiloxKey key;
  uint32_t stream_id;
  float alpha, c_det, inv_n;
  Strat st;   // sampling scheme
  float* g;   // [nf][nv]
  double* b;  // [nf][nv]
};

// one (request, field) linear system of the batched CG
struct BSys {
  const int32_t* rp;
  const int32_t* col;
  const double* val;
  const double* dinv;
  const float* aval;  // FP32 values of S M S (mixed mode)
  const double* sc;   // S = diag(M)^-1/2 (mixed mode)
  const double* b;
  double* x;
  int64_t off;  // first global row
  int64_t n;
  double tol;
  int32_t max_iter;
  int32_t blo, bhi;  // blocks owning its rows
  float lmax;        // spectrum bound of the scaled matrix: 2 (triangles), 5/2 (tetrahedra)
};

// a block's share of the mixed-precision batched solve: matrix rows [i0, i1)
// of one request with all its nf field systems s0 .. s0 + nf - 1 (the
// fields of a matrix row are visited back to back, so the row's matrix
// entries are read once from memory and again from cache for the others)
struct BPiece {
  int32_t s0, nf;
  int64_t i0, i1;
};

struct BSysOut {
  int32_t iters;
  int32_t conv;
  double rel;
};

// index of the last entry of off[0..n] that is <= key (off ascending, off[0] = 0)
__device__ __forceinline__ int find_seg(const int64_t* off, int n, int64_t key) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= key) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// step 1: control values of every request of one dimension
// ---------------------------------------------------------------------------
template <int D>
__global__ void __launch_bounds__(kBatchThreads) k_batch_control(const BReq* __restrict__ reqs,
                                                                 const int32_t* __restrict__ greq,
                                                                 const int64_t* __restrict__ goff, int ng,
                                                                 int64_t total, int64_t* __restrict__ counters) {
  extern __shared__ int64_t s_off[];  // [ng + 1]
  for (int i = threadIdx.x; i <= ng; i += blockDim.x) s_off[i] = goff[i];
  __syncthreads();
  int n_fb = 0, n_em = 0;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int gi = find_seg(s_off, ng, k);
    const BReq& R = reqs[greq[gi]];
    const int64_t i = k - s_off[gi];
    const GridP<float> gr = *R.grid;
    float X[D];
#pragma unroll
    for (int a = 0; a < D; ++a) X[a] = R.tx[i * D + a];
    float mu[D + 1];
    int status;
    const int32_t e = locate_point<D, float>(gr, R.cell_start, R.cell_items, R.cell_first, R.recs, R.adj, X, mu, status);
    n_fb += status == 1;
    n_em += status == 2;
    for (int f = 0; f < R.nf; ++f) R.g[(int64_t)f * R.nv + i] = e >= 0 ? eval_p1<D, float>(R.vals, R.snf, f, e, mu) : 0.f;
  }
  const int fb = warp_sum<int>(n_fb), em = warp_sum<int>(n_em);
  if ((threadIdx.x & 31) == 0) {
    if (fb) atomicAdd(reinterpret_cast<unsigned long long*>(counters), (unsigned long long)fb);
    if (em) atomicAdd(reinterpret_cast<unsigned long long*>(counters + 1), (unsigned long long)em);
  }
}

// ---------------------------------------------------------------------------
// steps 2-6: persistent fused assembly over the tasks of a request group.
// A task is one warp's share of one request: 32/LPE elements, LPE lanes per
// element (1, 2, 4 or 8, chosen per group by the autotuner; default min(U, 4))
// striding over its Philox units. Per-lane partials are plain FP32 sums of a
// lane's few samples; the warp combine is compensated.
// ---------------------------------------------------------------------------
template <int D, int NF>
__global__ void __launch_bounds__(kBatchThreads, NF <= 2 ? 4 : (NF <= 4 ? 3 : 2)) k_batch_assemble(const BReq* __restrict__ reqs,
                                                                  const int32_t* __restrict__ greq,
                                                                  const int64_t* __restrict__ goff, int ng,
                                                                  int64_t total, int tile,
                                                                  unsigned long long* __restrict__ work,
                                                                  int64_t* __restrict__ counters) {
  constexpr int K = D + 1;
  constexpr int SPU = D == 2 ? 2 : 1;
  using A = Ar<float>;
  extern __shared__ int64_t s_off[];  // [ng + 1]
  // each slot's control values at its element's vertices, one float4 per
  // field (w = 0 in 2D), staged once per task: the sample loop reads them
  // with one shared load per field instead of K global loads (slot stride
  // NF + 1 float4 keeps the slots of a load phase on different banks)
  __shared__ float4 s_g[kBatchThreads / 32][32 * (NF + 1)];
  for (int i = threadIdx.x; i <= ng; i += blockDim.x) s_off[i] = goff[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  int n_fb = 0, n_em = 0;
  for (;;) {
    unsigned long long start = 0;
    if (lane == 0) start = atomicAdd(work, (unsigned long long)tile);
    start = __shfl_sync(0xffffffffu, start, 0);
    if (start >= (unsigned long long)total) break;
    for (int kk = 0; kk < tile; ++kk) {
      const int64_t task_g = (int64_t)start + kk;
      if (task_g >= total) break;
      const int gi = find_seg(s_off, ng, task_g);
      const BReq& R = reqs[greq[gi]];
      const int64_t task = task_g - s_off[gi];
      const int U = R.U, G = R.G, N = R.N, nf = R.nf, LPE = R.LPE;
      int64_t t;
      int u0, ustep, seg_lo, seg_hi;
      bool active;
      {
        const int slot = lane / LPE;
        t = task * G + slot; u0 = lane - slot * LPE; ustep = LPE; seg_lo = slot * LPE; seg_hi = seg_lo + LPE;
        active = slot < G;
      }
      active = active && t < R.ne;
      int32_t v[K];
      float xv[K][D];
      float acc[NF][K];
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int i = 0; i < K; ++i) acc[f][i] = 0.f;
      if (active) {
#pragma unroll
        for (int m = 0; m < K; ++m) {
          v[m] = __ldg(R.tconn + t * K + m);
#pragma unroll
          for (int a = 0; a < D; ++a) xv[m][a] = __ldg(R.tx + (int64_t)v[m] * D + a);
        }
      }
      float4* sg = s_g[threadIdx.x >> 5] + (lane / LPE) * (NF + 1);
      __syncwarp();  // the previous task's reads of the slots are done
      if (active) {
        for (int f = lane - seg_lo; f < nf && f < NF; f += seg_hi - seg_lo) {
          const float* gf = R.g + (int64_t)f * R.nv;
          float4 q;
          q.x = __ldg(gf + v[0]);
          q.y = __ldg(gf + v[1]);
          q.z = __ldg(gf + v[2]);
          if constexpr (K == 4) q.w = __ldg(gf + v[3]);
          else q.w = 0.f;
          sg[f] = q;
        }
      }
      __syncwarp();
      const GridP<float> gr = *R.grid;
      for (int u = u0; active && u < U; u += ustep) {
        const uint4 w = philox4x32_10(make_uint4((uint32_t)u, (uint32_t)t, R.stream_id, 0u), R.key);
#pragma unroll
        for (int s = 0; s < SPU; ++s) {
          const int j = SPU * u + s;
          if (j >= N) break;
          float lam[K];
          sample_lambda<D, float>(w, j, R.st, lam);
          float X[D];
          map_point<D, float>(lam, xv, X);
          float mu[K];
          int status;
          const int32_t e = locate_point<D, float>(gr, R.cell_start, R.cell_items, R.cell_first, R.recs, R.adj, X, mu, status);
          n_fb += status == 1;
          n_em += status == 2;
#pragma unroll
          for (int f = 0; f < NF; ++f) {
            if (f >= nf) break;
            const float fs = e >= 0 ? eval_p1<D, float>(R.vals, R.snf, f, e, mu) : 0.f;
            const float4 gq = sg[f];
            float gX = A::mul(gq.x, lam[0]);
            gX = A::fma(gq.y, lam[1], gX);
            gX = A::fma(gq.z, lam[2], gX);
            if constexpr (K == 4) gX = A::fma(gq.w, lam[3], gX);
            const float r = A::sub(fs, A::mul(R.alpha, gX));
#pragma unroll
            for (int i = 0; i < K; ++i) acc[f][i] = A::fma(r, lam[i], acc[f][i]);
          }
        }
      }
      // compensated segmented suffix combine of every field's partials
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if (f >= nf) break;  // nf is warp-uniform
#pragma unroll
        for (int i = 0; i < K; ++i) {
          float s = acc[f][i], e = 0.f;
          for (int o = 1; o < LPE; o <<= 1) {  // log2 LPE rounds: a segment spans LPE lanes
            const float s2 = __shfl_down_sync(0xffffffffu, s, o);
            const float e2 = __shfl_down_sync(0xffffffffu, e, o);
            if (lane + o < seg_hi) {
              float tt, err;
              two_sum(s, s2, tt, err);
              s = tt;
              e = __fadd_rn(__fadd_rn(e, e2), err);
            }
          }
          acc[f][i] = __fadd_rn(s, e);
        }
      }
      if (active && lane == seg_lo) {
        const float wv = __ldg(R.vol32 + t);
        const float cd = __fmul_rn(wv, R.c_det), cm = __fmul_rn(wv, R.inv_n);
        for (int f = 0; f < nf && f < NF; ++f) {
          const float4 gq = sg[f];
          const float gl[4] = {gq.x, gq.y, gq.z, gq.w};
          float gsum = 0.f;
#pragma unroll
          for (int m = 0; m < K; ++m) gsum = __fadd_rn(gsum, gl[m]);
#pragma unroll
          for (int i = 0; i < K; ++i) {
            const float c = __fmaf_rn(cd, __fadd_rn(gsum, gl[i]), __fmul_rn(cm, acc[f][i]));
            atomicAdd(R.b + (int64_t)f * R.nv + v[i], (double)c);
          }
        }
      }
    }
  }
  const int fb = warp_sum<int>(n_fb), em = warp_sum<int>(n_em);
  if (lane == 0) {
    if (fb) atomicAdd(reinterpret_cast<unsigned long long*>(counters), (unsigned long long)fb);
    if (em) atomicAdd(reinterpret_cast<unsigned long long*>(counters + 1), (unsigned long long)em);
  }
}

// ---------------------------------------------------------------------------
// step 7: one cooperative Jacobi-PCG over all systems (block-diagonal).
// Block b owns global rows [b R, (b+1) R); its systems are s_lo(b)..s_hi(b).
// Rows are swept warp by warp (32 consecutive rows per step, steps 256 rows
// apart, so every lane's system index only moves forward). A warp reduces
// its step's per-row values by system with a segmented shuffle scan; the
// head lane of each segment adds the sum to the warp's slot of that system
// (fixed order: no atomics). One block barrier per phase combines the eight
// warp slots in order into the block's partial of each local system. After
// the grid barrier a warp per local system sums that system's partials over
// the blocks that own its rows, lanes in block order, then a fixed shuffle
// tree (deterministic and identical in every block). A system stops when it
// converges or reaches its own iteration cap; the kernel stops when a round
// finds every system stopped (a flag summed over blocks).
// ---------------------------------------------------------------------------
constexpr int kMaxLocalSys = 64;
constexpr int kBatchWarps = kBatchThreads / 32;

struct BCgCtl {
  GridBarrier bar;
  int32_t err;
  int32_t pad;
  unsigned int flag[3];
};

// segmented (by system index j, contiguous in lane order) warp sums of two
// values; the first lane of each segment adds them to slot[j] of this warp
// (T = float: the shuffle tree runs on the FP32 pipe; the slot stays FP64)
template <typename T>
__device__ __forceinline__ void warp_seg_add(int j, T a, T b, double (*slot)[2]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int j2 = __shfl_down_sync(0xffffffffu, j, o);
    const T a2 = __shfl_down_sync(0xffffffffu, a, o);
    const T b2 = __shfl_down_sync(0xffffffffu, b, o);
    if (lane + o < 32 && j2 == j) {
      a += a2;
      b += b2;
    }
  }
  const int jp = __shfl_up_sync(0xffffffffu, j, 1);
  if (j >= 0 && (lane == 0 || jp != j)) {
    slot[j][0] += (double)a;
    slot[j][1] += (double)b;
  }
}

__global__ void __launch_bounds__(kBatchThreads) k_batch_pcg(const BSys* __restrict__ sys, int nsys, int64_t ntot,
                                                             int64_t rows_per_block,
                                                             const int32_t* __restrict__ blk_slo,
                                                             const int32_t* __restrict__ blk_shi, int maxs,
                                                             double* r, double* z, double* p, double* q, double* part,
                                                             BSysOut* __restrict__ out, BCgCtl* ctl) {
  __shared__ double s_rz[kMaxLocalSys], s_bn[kMaxLocalSys], s_beta[kMaxLocalSys], s_alpha[kMaxLocalSys],
      s_rel[kMaxLocalSys];
  __shared__ int s_done[kMaxLocalSys], s_it[kMaxLocalSys], s_conv[kMaxLocalSys];
  __shared__ int64_t s_off[kMaxLocalSys + 1];
  __shared__ double s_w[kBatchWarps][kMaxLocalSys][2];
  __shared__ double s_g[kMaxLocalSys][2];
  __shared__ int s_any;
  const unsigned nb = gridDim.x;
  const int b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row0 = (int64_t)b * rows_per_block;
  const int64_t row1 = min(ntot, row0 + rows_per_block);
  const int slo = blk_slo[b], shi = blk_shi[b];
  const int nloc = row0 < row1 ? shi - slo + 1 : 0;
  for (int j = threadIdx.x; j <= nloc; j += blockDim.x)
    s_off[j] = j < nloc ? max(row0, sys[slo + j].off) : row1;

  // clear the warp slots (each warp its own)
  auto clear_slots = [&]() {
    for (int j = lane; j < nloc; j += 32) s_w[warp][j][0] = s_w[warp][j][1] = 0.0;
    __syncwarp();
  };
  // combine the warp slots in order into this block's partials
  auto publish = [&]() {
    __syncthreads();
    for (int k = threadIdx.x; k < nloc * 2; k += blockDim.x) {
      const int j = k >> 1, c = k & 1;
      double t = 0.0;
      for (int w = 0; w < kBatchWarps; ++w) t += s_w[w][j][c];
      part[((int64_t)b * maxs + j) * 2 + c] = t;
    }
  };
  // totals of every local system over its blocks -> s_g (warp per system)
  auto gather_all = [&]() {
    for (int j = warp; j < nloc; j += kBatchWarps) {
      const int s = slo + j;
      const BSys& S = sys[s];
      double a0 = 0.0, a1 = 0.0;
      for (int bb = S.blo + lane; bb <= S.bhi; bb += 32) {
        const double* pp = part + ((int64_t)bb * maxs + (s - blk_slo[bb])) * 2;
        a0 += __ldcg(pp);
        a1 += __ldcg(pp + 1);
      }
      a0 = warp_sum<double>(a0);
      a1 = warp_sum<double>(a1);
      if (lane == 0) {
        s_g[j][0] = a0;
        s_g[j][1] = a1;
      }
    }
    __syncthreads();
  };

  // init: x = 0, r = b, z = D^-1 r, p = q = 0; partials b.b and r.z
  clear_slots();
  __syncthreads();
  {
    int j = 0;
    for (int64_t base = row0 + warp * 32; base < row1; base += kBatchThreads) {
      const int64_t gr = base + lane;
      double bb = 0.0, rzv = 0.0;
      int jj = -1;
      if (gr < row1) {
        while (j + 1 < nloc && gr >= s_off[j + 1]) ++j;
        const BSys& S = sys[slo + j];
        const int64_t i = gr - S.off;
        const double bi = S.b[i], di = S.dinv[i];
        S.x[i] = 0.0;
        r[gr] = bi;
        z[gr] = di * bi;
        p[gr] = 0.0;
        q[gr] = 0.0;
        bb = bi * bi;
        rzv = bi * di * bi;
        jj = j;
      }
      warp_seg_add<double>(jj, bb, rzv, s_w[warp]);
    }
  }
  publish();
  if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
  gather_all();
  if (threadIdx.x < nloc) {
    const int j = threadIdx.x;
    s_bn[j] = sqrt(s_g[j][0]);
    s_rz[j] = s_g[j][1];
    s_beta[j] = 0.0;
    s_it[j] = 0;
    s_conv[j] = s_bn[j] == 0.0;
    s_done[j] = s_conv[j];
    s_rel[j] = 0.0;
  }
  __syncthreads();

  for (int it = 0;; ++it) {
    // phase A: w = M z, p = z + beta p, q = w + beta q, partial p.q
    clear_slots();
    {
      int j = 0;
      for (int64_t base = row0 + warp * 32; base < row1; base += kBatchThreads) {
        const int64_t gr = base + lane;
        double pq = 0.0;
        int jj = -1;
        if (gr < row1) {
          while (j + 1 < nloc && gr >= s_off[j + 1]) ++j;
          if (!s_done[j]) {
            const BSys& S = sys[slo + j];
            const int64_t i = gr - S.off;
            const double* zs = z + S.off;
            const int32_t k0 = __ldg(S.rp + i), k1 = __ldg(S.rp + i + 1);
            double w = 0.0;
            // z of other blocks is visible to ordinary loads after the grid barrier
            for (int32_t k = k0; k < k1; ++k) w += __ldg(S.val + k) * zs[__ldg(S.col + k)];
            const double bt = s_beta[j];
            const double pn = __ldcg(z + gr) + bt * __ldcg(p + gr);
            const double qn = w + bt * __ldcg(q + gr);
            p[gr] = pn;
            q[gr] = qn;
            pq = pn * qn;
            jj = j;
          }
        }
        warp_seg_add<double>(jj, pq, 0.0, s_w[warp]);
      }
    }
    publish();
    if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
    if (it > 0) {
      const unsigned int any = *reinterpret_cast<volatile unsigned int*>(&ctl->flag[(it - 1) % 3]);
      if (any == 0) break;
    }
    gather_all();
    if (threadIdx.x < nloc) {
      const int j = threadIdx.x;
      s_alpha[j] = s_done[j] ? 0.0 : s_rz[j] / s_g[j][0];
    }
    __syncthreads();
    // phase B: x += a p, r -= a q, z = D^-1 r, partials r.r and r.z
    clear_slots();
    {
      int j = 0;
      for (int64_t base = row0 + warp * 32; base < row1; base += kBatchThreads) {
        const int64_t gr = base + lane;
        double rr = 0.0, rzv = 0.0;
        int jj = -1;
        if (gr < row1) {
          while (j + 1 < nloc && gr >= s_off[j + 1]) ++j;
          if (!s_done[j]) {
            const BSys& S = sys[slo + j];
            const int64_t i = gr - S.off;
            const double al = s_alpha[j];
            S.x[i] = __ldcg(S.x + i) + al * __ldcg(p + gr);
            const double ri = __ldcg(r + gr) - al * __ldcg(q + gr);
            r[gr] = ri;
            const double zi = S.dinv[i] * ri;
            z[gr] = zi;
            rr = ri * ri;
            rzv = ri * zi;
            jj = j;
          }
        }
        warp_seg_add<double>(jj, rr, rzv, s_w[warp]);
      }
    }
    publish();
    if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
    gather_all();
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    if (threadIdx.x < nloc) {
      const int j = threadIdx.x;
      if (!s_done[j]) {
        const BSys& S = sys[slo + j];
        const double rn = sqrt(s_g[j][0]);
        const double rz_new = s_g[j][1];
        s_it[j] += 1;
        s_rel[j] = rn / s_bn[j];
        if (rn <= S.tol * s_bn[j]) s_conv[j] = 1;
        s_beta[j] = rz_new / s_rz[j];
        s_rz[j] = rz_new;
        s_done[j] = s_conv[j] || s_it[j] >= S.max_iter;
        if (!s_done[j]) atomicOr(&s_any, 1);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      if (b == 0) atomicExch(&ctl->flag[(it + 1) % 3], 0u);
      if (s_any) atomicAdd(&ctl->flag[it % 3], 1u);
    }
  }
  // results: written by the first block of each system
  if (threadIdx.x < nloc) {
    const int j = threadIdx.x;
    const int s = slo + j;
    if (sys[s].blo == b) {
      out[s].iters = s_it[j];
      out[s].conv = s_conv[j];
      out[s].rel = s_rel[j];
    }
  }
}


// ---------------------------------------------------------------------------
// Row phases of one piece of the batched mixed-precision solve. The piece's
// field f is system P.s0 + f; the fields of one request share the matrix and
// lie at stride S.n (S = the first field's system) in b, x and the work
// vectors, so a row's matrix entries are loaded once for all fields. NFC
// (1, 2, 4, 8) bounds the piece's field count; bit f of m marks the fields
// that work in the phase. A thread sums its rows' dot-product terms per
// field, and the warp adds them to its shared slots once per piece.
// ---------------------------------------------------------------------------
template <int NFC>
__device__ __forceinline__ void piece_flush(const double (&a)[NFC], const double (&c)[NFC], unsigned m,
                                            double (*slot)[2], int j0) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int f = 0; f < NFC; ++f) {
    if (!((m >> f) & 1u)) continue;
    const double u = warp_sum<double>(a[f]), v = warp_sum<double>(c[f]);
    if (lane == 0) {
      slot[j0 + f][0] += u;
      slot[j0 + f][1] += v;
    }
  }
}

template <int NFC>
__device__ __forceinline__ void piece_flush_f(const float (&a)[NFC], unsigned m, double (*slot)[2], int j0) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int f = 0; f < NFC; ++f) {
    if (!((m >> f) & 1u)) continue;
    const float u = warp_sum<float>(a[f]);
    if (lane == 0) slot[j0 + f][0] += (double)u;
  }
}

// R: r = b - M x in FP64 (x = 0 in cycle 0), t = S r; terms r.r, t.t
template <int NFC>
__device__ __forceinline__ void piece_R(const BPiece P, const BSys& S, unsigned m, int cyc, double* t,
                                        double (*slot)[2], int j0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = S.n;
  double a0[NFC], a1[NFC];
#pragma unroll
  for (int f = 0; f < NFC; ++f) a0[f] = a1[f] = 0.0;
  for (int64_t base = P.i0 + warp * 32; base < P.i1; base += kBatchThreads) {
    const int64_t i = base + lane;
    if (i >= P.i1) continue;
    double w[NFC];
#pragma unroll
    for (int f = 0; f < NFC; ++f) w[f] = 0.0;
    if (cyc > 0) {
      const int32_t k0 = __ldg(S.rp + i), k1 = __ldg(S.rp + i + 1);
      // x of other blocks is visible to ordinary loads after the grid barrier
      for (int32_t k = k0; k < k1; ++k) {
        const double v = __ldg(S.val + k);
        const int64_t c = __ldg(S.col + k);
#pragma unroll
        for (int f = 0; f < NFC; ++f)
          if ((m >> f) & 1u) w[f] += v * S.x[f * n + c];
      }
    }
    const double si = S.sc[i];
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      if (!((m >> f) & 1u)) continue;
      const int64_t o = f * n + i;
      if (cyc == 0) S.x[o] = 0.0;
      const double ri = S.b[o] - w[f];
      const double ti = si * ri;
      t[S.off + o] = ti;
      a0[f] += ri * ri;
      a1[f] += ti * ti;
    }
  }
  piece_flush<NFC>(a0, a1, m, slot, j0);
}

// I: c = t / ||t|| in FP32, y = p = q = 0; term c.c
template <int NFC>
__device__ __forceinline__ void piece_I(const BPiece P, const BSys& S, unsigned m, const double* t, float* r,
                                        float* p, float* q, float* y, const double* isig, double (*slot)[2],
                                        int j0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = S.n;
  float a[NFC];
  double is[NFC];
#pragma unroll
  for (int f = 0; f < NFC; ++f) {
    a[f] = 0.f;
    is[f] = (m >> f) & 1u ? isig[j0 + f] : 0.0;
  }
  for (int64_t base = P.i0 + warp * 32; base < P.i1; base += kBatchThreads) {
    const int64_t i = base + lane;
    if (i >= P.i1) continue;
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      if (!((m >> f) & 1u)) continue;
      const int64_t gr = S.off + f * n + i;
      const float ci = (float)(t[gr] * is[f]);
      r[gr] = ci;
      y[gr] = 0.f;
      p[gr] = 0.f;
      q[gr] = 0.f;
      a[f] += ci * ci;
    }
  }
  piece_flush_f<NFC>(a, m, slot, j0);
}

// A: w = A r, p = r + beta p, q = w + beta q (= A p); term p.q
template <int NFC>
__device__ __forceinline__ void piece_A(const BPiece P, const BSys& S, unsigned m, float* r, float* p, float* q,
                                        const float* beta, double (*slot)[2], int j0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = S.n;
  const float* rs = r + S.off;
  float a[NFC], bt[NFC];
#pragma unroll
  for (int f = 0; f < NFC; ++f) {
    a[f] = 0.f;
    bt[f] = (m >> f) & 1u ? beta[j0 + f] : 0.f;
  }
  for (int64_t base = P.i0 + warp * 32; base < P.i1; base += kBatchThreads) {
    const int64_t i = base + lane;
    if (i >= P.i1) continue;
    const int32_t k0 = __ldg(S.rp + i), k1 = __ldg(S.rp + i + 1);
    float w[NFC];
#pragma unroll
    for (int f = 0; f < NFC; ++f) w[f] = 0.f;
    // r was written by other blocks before the grid barrier (plain loads)
    for (int32_t k = k0; k < k1; ++k) {
      const float v = __ldg(S.aval + k);
      const int64_t c = __ldg(S.col + k);
#pragma unroll
      for (int f = 0; f < NFC; ++f)
        if ((m >> f) & 1u) w[f] += v * rs[f * n + c];
    }
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      if (!((m >> f) & 1u)) continue;
      const int64_t gr = S.off + f * n + i;
      const float pn = r[gr] + bt[f] * p[gr];
      const float qn = w[f] + bt[f] * q[gr];
      p[gr] = pn;
      q[gr] = qn;
      a[f] += pn * qn;
    }
  }
  piece_flush_f<NFC>(a, m, slot, j0);
}

// B: y += alpha p, r -= alpha q; term r.r
template <int NFC>
__device__ __forceinline__ void piece_B(const BPiece P, const BSys& S, unsigned m, float* r, const float* p,
                                        const float* q, float* y, const float* alpha, double (*slot)[2], int j0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = S.n;
  float a[NFC], al[NFC];
#pragma unroll
  for (int f = 0; f < NFC; ++f) {
    a[f] = 0.f;
    al[f] = (m >> f) & 1u ? alpha[j0 + f] : 0.f;
  }
  for (int64_t base = P.i0 + warp * 32; base < P.i1; base += kBatchThreads) {
    const int64_t i = base + lane;
    if (i >= P.i1) continue;
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      if (!((m >> f) & 1u)) continue;
      const int64_t gr = S.off + f * n + i;
      y[gr] += al[f] * p[gr];
      const float ri = r[gr] - al[f] * q[gr];
      r[gr] = ri;
      a[f] += ri * ri;
    }
  }
  piece_flush_f<NFC>(a, m, slot, j0);
}

// Chebyshev I: c = t / ||t|| in FP32, r = c, y = 0, d = c / theta (in p)
template <int NFC>
__device__ __forceinline__ void piece_Ic(const BPiece P, const BSys& S, unsigned m, const double* t, float* r,
                                         float* p, float* y, const double* isig, float ith, int j0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = S.n;
  double is[NFC];
#pragma unroll
  for (int f = 0; f < NFC; ++f) is[f] = (m >> f) & 1u ? isig[j0 + f] : 0.0;
  for (int64_t base = P.i0 + warp * 32; base < P.i1; base += kBatchThreads) {
    const int64_t i = base + lane;
    if (i >= P.i1) continue;
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      if (!((m >> f) & 1u)) continue;
      const int64_t gr = S.off + f * n + i;
      const float ci = (float)(t[gr] * is[f]);
      r[gr] = ci;
      y[gr] = 0.f;
      p[gr] = ci * ith;
    }
  }
}

// Chebyshev step: w = A d, y += d, r -= w, d' = c1 d + c2 r (d' in the
// other buffer: the SpMV reads the d every block wrote in the step before)
template <int NFC>
__device__ __forceinline__ void piece_C(const BPiece P, const BSys& S, unsigned m, const float* dc, float* dn,
                                        float* r, float* y, float c1, float c2, int j0) {
  (void)j0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = S.n;
  const float* ds = dc + S.off;
  for (int64_t base = P.i0 + warp * 32; base < P.i1; base += kBatchThreads) {
    const int64_t i = base + lane;
    if (i >= P.i1) continue;
    const int32_t k0 = __ldg(S.rp + i), k1 = __ldg(S.rp + i + 1);
    float w[NFC];
#pragma unroll
    for (int f = 0; f < NFC; ++f) w[f] = 0.f;
    // d was written by other blocks before the grid barrier (plain loads)
    for (int32_t k = k0; k < k1; ++k) {
      const float v = __ldg(S.aval + k);
      const int64_t c = __ldg(S.col + k);
#pragma unroll
      for (int f = 0; f < NFC; ++f)
        if ((m >> f) & 1u) w[f] += v * ds[f * n + c];
    }
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      if (!((m >> f) & 1u)) continue;
      const int64_t gr = S.off + f * n + i;
      const float di = dc[gr];
      y[gr] += di;
      const float ri = r[gr] - w[f];
      r[gr] = ri;
      dn[gr] = c1 * di + c2 * ri;
    }
  }
}

// U: x += ||t|| S y
template <int NFC>
__device__ __forceinline__ void piece_U(const BPiece P, const BSys& S, unsigned m, const float* y,
                                        const double* sig, int j0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t n = S.n;
  double sg[NFC];
#pragma unroll
  for (int f = 0; f < NFC; ++f) sg[f] = (m >> f) & 1u ? sig[j0 + f] : 0.0;
  for (int64_t base = P.i0 + warp * 32; base < P.i1; base += kBatchThreads) {
    const int64_t i = base + lane;
    if (i >= P.i1) continue;
    const double si = S.sc[i];
#pragma unroll
    for (int f = 0; f < NFC; ++f) {
      if (!((m >> f) & 1u)) continue;
      const int64_t o = f * n + i;
      S.x[o] += (sg[f] * si) * (double)y[S.off + o];
    }
  }
}

// the piece's field class and its mask of working fields (flags[j0 + f])
__device__ __forceinline__ unsigned piece_mask(const BPiece& P, const int* flags, int j0) {
  unsigned m = 0u;
  for (int f = 0; f < P.nf; ++f) m |= flags[j0 + f] ? 1u << f : 0u;
  return m;
}

// run phase PH on piece P (locals P, m, j0, sys) by its field class; with
// MAXF = 4 a piece of more fields runs as two halves (field 4's system
// starts the second), which bounds the registers the unrolled fields take
#define SFT_PIECE_RUN(PH, MAXF, ...)                                             \
  do {                                                                           \
    if (P.nf <= 1) PH<1>(P, sys[P.s0], m, __VA_ARGS__, j0);                      \
    else if (P.nf <= 2) PH<2>(P, sys[P.s0], m, __VA_ARGS__, j0);                 \
    else if (P.nf <= 4) PH<4>(P, sys[P.s0], m, __VA_ARGS__, j0);                 \
    else if ((MAXF) == 8) PH<8>(P, sys[P.s0], m, __VA_ARGS__, j0);               \
    else {                                                                       \
      const BPiece H{P.s0 + 4, P.nf - 4, P.i0, P.i1};                            \
      if (m & 0xfu) PH<4>(P, sys[P.s0], m & 0xfu, __VA_ARGS__, j0);              \
      if (m >> 4) PH<4>(H, sys[H.s0], m >> 4, __VA_ARGS__, j0 + 4);              \
    }                                                                            \
  } while (0)
// field bound of the FP64 phase R and of the FP32 phases
constexpr int kPieceFieldsR = 4, kPieceFields = 8;

// ---------------------------------------------------------------------------
// Batched mixed-precision iterative refinement (the cg_mode MIXED solve of
// every (request, field) system at once; see the single-system k_mixed_cg):
// per refinement cycle an FP64 residual pass R, the FP32 right-hand side
// pass I, the FP32 inner solve on S M S and the FP64 update U. The inner
// solve is the Chebyshev iteration (one step phase per step; each system
// takes the step count its spectrum interval fixes for its target), or CG
// (phases A and B) when built with the CG alternative. All systems step
// through the same phases; a system whose inner solve reached its target
// (or that converged) skips the row work of the phase. Whether
// any system still works is a flag summed over blocks, read after the next
// grid barrier (three rotating flags: the one of decision d is cleared at
// decision d + 2, when every block has read it).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kBatchThreads, 4) k_batch_mixed(const BSys* __restrict__ sys,
                                                               const BPiece* __restrict__ pcs,
                                                               const int32_t* __restrict__ blk_pc,
                                                               const int32_t* __restrict__ blk_slo,
                                                               const int32_t* __restrict__ blk_shi, int maxs,
                                                               double* t, float* r, float* p, float* q, float* y,
                                                               double* part, BSysOut* __restrict__ out, BCgCtl* ctl) {
  __shared__ double s_bn[kMaxLocalSys], s_prev[kMaxLocalSys], s_sig[kMaxLocalSys], s_isig[kMaxLocalSys],
      s_rel[kMaxLocalSys];
  __shared__ float s_eta2[kMaxLocalSys], s_rr[kMaxLocalSys], s_alpha[kMaxLocalSys], s_beta[kMaxLocalSys];
  __shared__ int s_live[kMaxLocalSys], s_act[kMaxLocalSys], s_conv[kMaxLocalSys], s_it[kMaxLocalSys];
  __shared__ int s_ks[kMaxLocalSys];  // Chebyshev steps of the cycle
  __shared__ double s_w[kBatchWarps][kMaxLocalSys][2];
  __shared__ double s_g[kMaxLocalSys][2];
  __shared__ int s_any;
  const unsigned nb = gridDim.x;
  const int b = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pc0 = blk_pc[b], pc1 = blk_pc[b + 1];
  const int slo = blk_slo[b], shi = blk_shi[b];
  const int nloc = pc0 < pc1 ? shi - slo + 1 : 0;
  for (int j = threadIdx.x; j < nloc; j += blockDim.x) {
    s_live[j] = sys[slo + j].n > 0;
    s_act[j] = 0;
    s_conv[j] = sys[slo + j].n == 0;
    s_it[j] = 0;
    s_rel[j] = 0.0;
  }

  auto clear_slots = [&]() {
    for (int j = lane; j < nloc; j += 32) s_w[warp][j][0] = s_w[warp][j][1] = 0.0;
    __syncwarp();
  };
  auto publish = [&]() {
    __syncthreads();
    for (int k = threadIdx.x; k < nloc * 2; k += blockDim.x) {
      const int j = k >> 1, c = k & 1;
      double v = 0.0;
      for (int w = 0; w < kBatchWarps; ++w) v += s_w[w][j][c];
      part[((int64_t)b * maxs + j) * 2 + c] = v;
    }
  };
  auto gather_all = [&]() {
    for (int j = warp; j < nloc; j += kBatchWarps) {
      const int s = slo + j;
      const BSys& S = sys[s];
      double a0 = 0.0, a1 = 0.0;
      for (int bb = S.blo + lane; bb <= S.bhi; bb += 32) {
        const double* pp = part + ((int64_t)bb * maxs + (s - blk_slo[bb])) * 2;
        a0 += __ldcg(pp);
        a1 += __ldcg(pp + 1);
      }
      a0 = warp_sum<double>(a0);
      a1 = warp_sum<double>(a1);
      if (lane == 0) {
        s_g[j][0] = a0;
        s_g[j][1] = a1;
      }
    }
    __syncthreads();
  };
  int dcount = 0;
  // block's vote for decision dcount (s_any set by the per-system threads)
  auto post = [&]() {
    __syncthreads();
    if (threadIdx.x == 0) {
      if (b == 0) atomicExch(&ctl->flag[(dcount + 1) % 3], 0u);
      if (s_any) atomicAdd(&ctl->flag[dcount % 3], 1u);
    }
    ++dcount;
  };
  auto voted = [&]() -> bool {
    return *reinterpret_cast<volatile unsigned int*>(&ctl->flag[(dcount - 1) % 3]) != 0u;
  };
  __syncthreads();

  for (int cyc = 0;; ++cyc) {
    // R: r = b - M x in FP64 (x = 0 in the first cycle), t = S r; partials r.r, t.t
    clear_slots();
    for (int pc = pc0; pc < pc1; ++pc) {
      const BPiece P = pcs[pc];
      const int j0 = P.s0 - slo;
      const unsigned m = piece_mask(P, s_live, j0);
      if (!m) continue;
      SFT_PIECE_RUN(piece_R, kPieceFieldsR, cyc, t, s_w[warp]);
    }
    publish();
    if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
    gather_all();
    if (threadIdx.x == 0) s_any = 0;
    __syncthreads();
    if (threadIdx.x < nloc) {
      const int j = threadIdx.x;
      if (s_live[j]) {
        const BSys& S = sys[slo + j];
        const double rn = sqrt(s_g[j][0]), tn = sqrt(s_g[j][1]);
        if (cyc == 0) s_bn[j] = rn;
        s_rel[j] = s_bn[j] > 0.0 ? rn / s_bn[j] : 0.0;
        if (rn <= S.tol * s_bn[j]) {
          s_live[j] = 0;
          s_conv[j] = 1;
        } else if ((cyc > 0 && rn > 0.5 * s_prev[j]) || !(tn > 0.0) || s_it[j] >= S.max_iter) {
          s_live[j] = 0;  // stagnated, no scaled residual, or out of iterations: unconverged
        } else {
          s_prev[j] = rn;
          s_sig[j] = tn;
          s_isig[j] = 1.0 / tn;
          const double e = fmin(0.25, fmax(1e-5, 0.1 * S.tol * s_bn[j] / rn));
          s_eta2[j] = (float)(e * e);
          s_ks[j] = cheb_steps(e, cheb_coef(S.lmax).s1);
          s_act[j] = 1;
          atomicOr(&s_any, 1);
        }
      }
    }
    post();
    if (kMixCheb) {
      // I: r = c, y = 0, d = c / theta; the barrier makes d whole for the first step
      for (int pc = pc0; pc < pc1; ++pc) {
        const BPiece P = pcs[pc];
        const int j0 = P.s0 - slo;
        const unsigned m = piece_mask(P, s_act, j0);
        if (!m) continue;
        const float ith = 1.f / cheb_coef(sys[P.s0].lmax).theta;
        SFT_PIECE_RUN(piece_Ic, kPieceFields, t, r, p, y, s_isig, ith);
      }
      if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
      if (!voted()) break;  // no system left to refine
      const ChebCoef c2d = cheb_coef(2.f), c3d = cheb_coef(2.5f);
      float rho2 = 1.f / c2d.s1, rho3 = 1.f / c3d.s1;
      for (int s = 0;; ++s) {
        const float n2 = 1.f / (2.f * c2d.s1 - rho2), n3 = 1.f / (2.f * c3d.s1 - rho3);
        const float a2 = n2 * rho2, b2 = n2 * (2.f / c2d.delta), a3 = n3 * rho3, b3 = n3 * (2.f / c3d.delta);
        const float* dc = (s & 1) ? q : p;
        float* dn = (s & 1) ? p : q;
        for (int pc = pc0; pc < pc1; ++pc) {
          const BPiece P = pcs[pc];
          const int j0 = P.s0 - slo;
          unsigned m = 0u;
          for (int f = 0; f < P.nf; ++f) m |= s_act[j0 + f] && s < s_ks[j0 + f] ? 1u << f : 0u;
          if (!m) continue;
          const bool d3 = sys[P.s0].lmax > 2.25f;
          SFT_PIECE_RUN(piece_C, kPieceFields, dc, dn, r, y, d3 ? a3 : a2, d3 ? b3 : b2);
        }
        rho2 = n2;
        rho3 = n3;
        if (threadIdx.x == 0) s_any = 0;
        __syncthreads();
        if (threadIdx.x < nloc) {
          const int j = threadIdx.x;
          if (s_act[j] && s < s_ks[j]) {
            s_it[j] += 1;
            if (s + 1 < s_ks[j] && s_it[j] < sys[slo + j].max_iter) atomicOr(&s_any, 1);
            else s_act[j] = 0;
          }
        }
        post();
        if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
        if (!voted()) break;  // every system took its steps
      }
    } else {
    // I: c = t / ||t|| in FP32, y = p = q = 0; partial c.c
    clear_slots();
    __syncthreads();
    for (int pc = pc0; pc < pc1; ++pc) {
      const BPiece P = pcs[pc];
      const int j0 = P.s0 - slo;
      const unsigned m = piece_mask(P, s_act, j0);
      if (!m) continue;
      SFT_PIECE_RUN(piece_I, kPieceFields, t, r, p, q, y, s_isig, s_w[warp]);
    }
    publish();
    if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
    if (!voted()) break;  // no system left to refine
    gather_all();
    if (threadIdx.x < nloc) {
      const int j = threadIdx.x;
      s_rr[j] = (float)s_g[j][0];
      s_beta[j] = 0.f;
    }
    __syncthreads();

    // FP32 CG on S M S y = c
    for (int inner = 0;; ++inner) {
      // A: w = A r, p = r + beta p, q = w + beta q; partial p.q
      clear_slots();
      for (int pc = pc0; pc < pc1; ++pc) {
        const BPiece P = pcs[pc];
        const int j0 = P.s0 - slo;
        const unsigned m = piece_mask(P, s_act, j0);
        if (!m) continue;
        SFT_PIECE_RUN(piece_A, kPieceFields, r, p, q, s_beta, s_w[warp]);
      }
      publish();
      if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
      if (inner > 0 && !voted()) break;  // every inner solve reached its target
      gather_all();
      if (threadIdx.x < nloc) {
        const int j = threadIdx.x;
        s_alpha[j] = s_act[j] ? s_rr[j] / (float)s_g[j][0] : 0.f;
      }
      __syncthreads();
      // B: y += alpha p, r -= alpha q; partial r.r
      clear_slots();
      for (int pc = pc0; pc < pc1; ++pc) {
        const BPiece P = pcs[pc];
        const int j0 = P.s0 - slo;
        const unsigned m = piece_mask(P, s_act, j0);
        if (!m) continue;
        SFT_PIECE_RUN(piece_B, kPieceFields, r, p, q, y, s_alpha, s_w[warp]);
      }
      publish();
      if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
      gather_all();
      if (threadIdx.x == 0) s_any = 0;
      __syncthreads();
      if (threadIdx.x < nloc) {
        const int j = threadIdx.x;
        if (s_act[j]) {
          const float rn = (float)s_g[j][0];
          s_it[j] += 1;
          s_beta[j] = rn / s_rr[j];
          s_rr[j] = rn;
          if (rn <= s_eta2[j] || s_it[j] >= sys[slo + j].max_iter) s_act[j] = 0;
          else atomicOr(&s_any, 1);
        }
      }
      post();
    }
    }
    // U: x += ||t|| S y for every system that refined in this cycle
    for (int pc = pc0; pc < pc1; ++pc) {
      const BPiece P = pcs[pc];
      const int j0 = P.s0 - slo;
      const unsigned m = piece_mask(P, s_live, j0);
      if (!m) continue;
      SFT_PIECE_RUN(piece_U, kPieceFields, y, s_sig);
    }
    if (!grid_sync(&ctl->bar, nb, &ctl->err)) return;
  }
  if (threadIdx.x < nloc) {
    const int j = threadIdx.x;
    const int s = slo + j;
    if (sys[s].blo == b) {
      out[s].iters = s_it[j];
      out[s].conv = s_conv[j];
      out[s].rel = s_rel[j];
    }
  }
}

// ---------------------------------------------------------------------------
// autotune cache: (dim, field class, log2 mean N, log2 tasks) -> tile
// ---------------------------------------------------------------------------
using TuneKey = std::tuple<int, int, int, int>;
using TuneVal = std::pair<int, int>;  // (tile, lanes per element; 0 = the default min(U, 4))
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune;
static bool g_tune_loaded = false;

static const char* tune_file() { return std::getenv("SFT_AUTOTUNE_CACHE"); }

static void tune_load_locked() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = tune_file();
  if (!path) return;
  FILE* fh = std::fopen(path, "r");
  if (!fh) return;
  int d, c, n, t, tile, lpe;
  while (std::fscanf(fh, "%d %d %d %d %d %d", &d, &c, &n, &t, &tile, &lpe) == 6)
    g_tune[TuneKey(d, c, n, t)] = TuneVal(tile, lpe);
  std::fclose(fh);
}

static void tune_store_locked(const TuneKey& k, TuneVal v) {
  g_tune[k] = v;
  const char* path = tune_file();
  if (!path) return;
  FILE* fh = std::fopen(path, "a");
  if (!fh) return;
  std::fprintf(fh, "%d %d %d %d %d %d\n", std::get<0>(k), std::get<1>(k), std::get<2>(k), std::get<3>(k), v.first,
               v.second);
  std::fclose(fh);
}

static int ilog2(double x) { return x < 1.0 ? 0 : (int)std::floor(std::log2(x)); }

}  // namespace sft

// ---------------------------------------------------------------------------
// the plan
// ---------------------------------------------------------------------------
struct sft_batch_s {
  int nreq = 0;
  cudaStream_t stream = nullptr;
  std::vector<sft_source> srcs;
  std::vector<sft_target> tgts;
  std::vector<sft::BReq> hreq;
  sft::BReq* dreq = nullptr;
  // groups: index = (dim - 2) * 3 + field class (0: nf <= 2, 1: <= 4, 2: <= 8)
  struct Group {
    std::vector<int32_t> req;
    std::vector<int64_t> off;  // task offsets
    int32_t* dreq = nullptr;
    int64_t* doff = nullptr;
    int64_t total = 0;
    int tile = 4;
    int lpe = 0;  // lanes per element of every request in the group (0: min(U, 4) per request)
    unsigned long long* work = nullptr;
  } grp[6];
  struct CtlGroup {
    std::vector<int32_t> req;
    std::vector<int64_t> off;  // node offsets
    int32_t* dreq = nullptr;
    int64_t* doff = nullptr;
    int64_t total = 0;
  } ctl[2];
  // buffers
  float* g = nullptr;
  double* b = nullptr;
  double* u = nullptr;
  std::vector<int64_t> vec_off;  // per request offset into g/b/u (elements)
  int64_t vec_total = 0;
  int64_t* counters = nullptr;
  // CG
  std::vector<sft::BSys> hsys;
  sft::BSys* dsys = nullptr;
  int nsys = 0;
  int64_t ntot = 0, rows_per_block = 0;
  int nblocks = 0, maxs = 1;
  int32_t *blk_slo = nullptr, *blk_shi = nullptr;
  sft::BPiece* pcs = nullptr;     // mixed mode: the blocks' pieces
  int32_t* blk_pc = nullptr;      // [nblocks + 1]: block b owns pcs[blk_pc[b] .. blk_pc[b + 1])
  double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *part = nullptr;
  bool mixed = true;  // every request asked for cg_mode MIXED (else the FP64 CG for all)
  sft::BSysOut* sysout = nullptr;
  sft::BCgCtl* cgctl = nullptr;
  std::vector<int> sys_first;  // first system of each request
  // graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_ok = false;
  int64_t graph_kernels = 0;  // kernels recorded in the graph (counted per replay)
  cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t queries = 0;
};

namespace sft {

static sft_status enqueue_batch(sft_batch_s* B, cudaStream_t st) {
  SFT_CUDA(cudaEventRecordWithFlags(B->ev[0], st, cudaEventRecordExternal));
  SFT_CUDA(cudaMemsetAsync(B->b, 0, sizeof(double) * B->vec_total, st));
  SFT_CUDA(cudaMemsetAsync(B->counters, 0, sizeof(int64_t) * 2, st));
  SFT_CUDA(cudaMemsetAsync(B->cgctl, 0, sizeof(BCgCtl), st));
  for (auto& G : B->grp)
    if (G.total) SFT_CUDA(cudaMemsetAsync(G.work, 0, sizeof(unsigned long long), st));
  for (int d = 0; d < 2; ++d) {
    auto& C = B->ctl[d];
    if (!C.total) continue;
    const unsigned blocks = (unsigned)std::min<int64_t>((C.total + kBatchThreads - 1) / kBatchThreads, 152 * 16);
    if (d == 0)
      ::sft::note_launch(), k_batch_control<2><<<blocks, kBatchThreads, sizeof(int64_t) * (C.req.size() + 1), st>>>(B->dreq, C.dreq, C.doff,
                                                                                  (int)C.req.size(), C.total, B->counters);
    else
      ::sft::note_launch(), k_batch_control<3><<<blocks, kBatchThreads, sizeof(int64_t) * (C.req.size() + 1), st>>>(B->dreq, C.dreq, C.doff,
                                                                                  (int)C.req.size(), C.total, B->counters);
    SFT_CUDA(cudaGetLastError());
  }
  SFT_CUDA(cudaEventRecordWithFlags(B->ev[1], st, cudaEventRecordExternal));
  int sms = 152;
  {
    int dev = 0;
    SFT_CUDA(cudaGetDevice(&dev));
    SFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  for (int gi = 0; gi < 6; ++gi) {
    auto& G = B->grp[gi];
    if (!G.total) continue;
    const unsigned blocks = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)sms * 4, (G.total + (kBatchThreads / 32) - 1) / (kBatchThreads / 32)));
    const int ng = (int)G.req.size();
#define SFT_BA(DD, NN)                                                                                          \
  ::sft::note_launch(), k_batch_assemble<DD, NN><<<blocks, kBatchThreads, sizeof(int64_t) * (ng + 1), st>>>(B->dreq, G.dreq, G.doff, ng, \
                                                                                   G.total, G.tile, G.work,   \
                                                                                   B->counters)
    switch (gi) {
      case 0: SFT_BA(2, 2); break;
      case 1: SFT_BA(2, 4); break;
      case 2: SFT_BA(2, 8); break;
      case 3: SFT_BA(3, 2); break;
      case 4: SFT_BA(3, 4); break;
      default: SFT_BA(3, 8); break;
    }
#undef SFT_BA
    SFT_CUDA(cudaGetLastError());
  }
  SFT_CUDA(cudaEventRecordWithFlags(B->ev[2], st, cudaEventRecordExternal));
  if (B->nsys > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)B->nblocks);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ::sft::note_launch();
    if (B->mixed) {
      // FP32 work vectors packed into the FP64 ones: r | y in r, p | q in p; t in z
      float* r32 = reinterpret_cast<float*>(B->r);
      float* p32 = reinterpret_cast<float*>(B->p);
      SFT_CUDA(cudaLaunchKernelEx(&cfg, k_batch_mixed, (const BSys*)B->dsys, (const BPiece*)B->pcs,
                                  (const int32_t*)B->blk_pc, (const int32_t*)B->blk_slo, (const int32_t*)B->blk_shi,
                                  B->maxs, B->z, r32, p32, p32 + B->ntot, r32 + B->ntot, B->part, B->sysout,
                                  B->cgctl));
    } else {
      SFT_CUDA(cudaLaunchKernelEx(&cfg, k_batch_pcg, (const BSys*)B->dsys, B->nsys, B->ntot, B->rows_per_block,
                                  (const int32_t*)B->blk_slo, (const int32_t*)B->blk_shi, B->maxs, B->r, B->z, B->p,
                                  B->q, B->part, B->sysout, B->cgctl));
    }
  }
  SFT_CUDA(cudaEventRecordWithFlags(B->ev[3], st, cudaEventRecordExternal));
  return SFT_OK;
}

// lanes per element of a request: the group's choice, or min(U, 4)
static int request_lpe(const BReq& R, int lpe) { return lpe > 0 ? lpe : (R.U >= 4 ? 4 : R.U); }

// apply lanes per element `lpe` to every request of group gi: elements per
// task, task counts, the group's task offsets (host and device copies)
static sft_status set_group_lpe(sft_batch_s* B, int gi, int lpe, cudaStream_t st) {
  auto& G = B->grp[gi];
  G.lpe = lpe;
  G.off.assign(1, 0);
  for (int32_t r : G.req) {
    BReq& R = B->hreq[r];
    R.LPE = request_lpe(R, lpe);
    R.G = 32 / R.LPE;
    R.ntasks = (R.ne + R.G - 1) / R.G;
    G.off.push_back(G.off.back() + R.ntasks);
  }
  G.total = G.off.back();
  if (G.doff) SFT_CUDA(cudaMemcpyAsync(G.doff, G.off.data(), sizeof(int64_t) * G.off.size(), cudaMemcpyHostToDevice, st));
  if (B->dreq)
    SFT_CUDA(cudaMemcpyAsync(B->dreq, B->hreq.data(), sizeof(BReq) * B->hreq.size(), cudaMemcpyHostToDevice, st));
  return SFT_OK;
}

// Timed trials of the group's assembly over lanes per element {1, 2, 4, 8}
// x tiles {1, 2, 4, 8, 16} (tasks a warp takes per atomic); the fastest pair
// is kept and cached per (dimension, field class, log2 mean N, log2 tasks).
static sft_status autotune_group(sft_batch_s* B, int gi, cudaStream_t st) {
  auto& G = B->grp[gi];
  const int dim = gi < 3 ? 2 : 3;
  double mean_n = 0.0;
  for (int32_t r : G.req) mean_n += B->hreq[r].N;
  mean_n /= (double)G.req.size();
  const TuneKey key(dim, gi % 3, ilog2(mean_n), ilog2((double)G.total));
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_load_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      G.tile = it->second.first;
      return set_group_lpe(B, gi, it->second.second, st);
    }
  }
  // control values must exist before trial assemblies
  int sms = 152, dev = 0;
  SFT_CUDA(cudaGetDevice(&dev));
  SFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  cudaEvent_t e0, e1;
  SFT_CUDA(cudaEventCreate(&e0));
  SFT_CUDA(cudaEventCreate(&e1));
  const int tiles[] = {1, 2, 4, 8, 16};
  const int lpes[] = {1, 2, 4, 8};
  float best = 1e30f;
  TuneVal best_v(4, 0);
  const int ng = (int)G.req.size();
  for (int lpe : lpes) {
    if (sft_status e = set_group_lpe(B, gi, lpe, st)) return e;
    const unsigned blocks = (unsigned)std::max<int64_t>(
        1, std::min<int64_t>((int64_t)sms * 4, (G.total + (kBatchThreads / 32) - 1) / (kBatchThreads / 32)));
    for (int tile : tiles) {
      float tsum = 0.f;
      for (int rep = 0; rep < 2; ++rep) {
        SFT_CUDA(cudaMemsetAsync(G.work, 0, sizeof(unsigned long long), st));
        SFT_CUDA(cudaEventRecord(e0, st));
#define SFT_BA(DD, NN)                                                                                          \
  ::sft::note_launch(), k_batch_assemble<DD, NN><<<blocks, kBatchThreads, sizeof(int64_t) * (ng + 1), st>>>(B->dreq, G.dreq, G.doff, ng, \
                                                                                   G.total, tile, G.work,     \
                                                                                   B->counters)
        switch (gi) {
          case 0: SFT_BA(2, 2); break;
          case 1: SFT_BA(2, 4); break;
          case 2: SFT_BA(2, 8); break;
          case 3: SFT_BA(3, 2); break;
          case 4: SFT_BA(3, 4); break;
          default: SFT_BA(3, 8); break;
        }
#undef SFT_BA
        SFT_CUDA(cudaGetLastError());
        SFT_CUDA(cudaEventRecord(e1, st));
        SFT_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        SFT_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) tsum += ms;
      }
      if (tsum < best) {
        best = tsum;
        best_v = TuneVal(tile, lpe);
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  G.tile = best_v.first;
  if (sft_status e = set_group_lpe(B, gi, best_v.second, st)) return e;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  tune_store_locked(key, best_v);
  return SFT_OK;
}

static void free_batch(sft_batch_s* B) {
  cudaStream_t st = B->stream;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (auto& e : B->ev)
    if (e) cudaEventDestroy(e);
  for (auto& G : B->grp) {
    dfree(G.dreq, st);
    dfree(G.doff, st);
    dfree(G.work, st);
  }
  for (auto& C : B->ctl) {
    dfree(C.dreq, st);
    dfree(C.doff, st);
  }
  dfree(B->dreq, st);
  dfree(B->g, st);
  dfree(B->b, st);
  dfree(B->u, st);
  dfree(B->counters, st);
  dfree(B->dsys, st);
  dfree(B->blk_slo, st);
  dfree(B->blk_shi, st);
  dfree(B->pcs, st);
  dfree(B->blk_pc, st);
  dfree(B->r, st);
  dfree(B->z, st);
  dfree(B->p, st);
  dfree(B->q, st);
  dfree(B->part, st);
  dfree(B->sysout, st);
  dfree(B->cgctl, st);
  delete B;
}

template <typename T>
static sft_status upload(T** dst, const std::vector<T>& v, cudaStream_t st) {
  SFT_CUDA(dalloc(dst, v.size(), st));
  if (!v.empty()) SFT_CUDA(cudaMemcpyAsync(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return SFT_OK;
}

static sft_status build_batch(sft_batch_s* B, const sft_options* opts, int autotune) {
  cudaStream_t st = B->stream;
  const int nreq = B->nreq;
  int32_t* d_err = nullptr;
  SFT_CUDA(dalloc(&d_err, 1, st));
  SFT_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int32_t), st));
  // buffers per request
  B->vec_off.resize(nreq + 1);
  B->vec_off[0] = 0;
  for (int r = 0; r < nreq; ++r) {
    const int nf = opts[r].field_count > 0 ? opts[r].field_count : B->srcs[r]->nf;
    B->vec_off[r + 1] = B->vec_off[r] + (int64_t)nf * B->tgts[r]->nv;
  }
  B->vec_total = B->vec_off[nreq];
  SFT_CUDA(dalloc(&B->g, (size_t)B->vec_total, st));
  SFT_CUDA(dalloc(&B->b, (size_t)B->vec_total, st));
  SFT_CUDA(dalloc(&B->u, (size_t)B->vec_total, st));
  SFT_CUDA(dalloc(&B->counters, 2, st));
  B->hreq.resize(nreq);
  B->queries = 0;
  for (int r = 0; r < nreq; ++r) {
    sft_source s = B->srcs[r];
    sft_target t = B->tgts[r];
    if (sft_status e = build_locator(s, SFT_PREC_FP32, st, d_err)) return e;
    if (sft_status e = target_coordsP(t, SFT_PREC_FP32, st)) return e;
    const Locator& L = s->loc[SFT_PREC_FP32];
    BReq& R = B->hreq[r];
    const sft_options& o = opts[r];
    R.tx = (const float*)t->coordsP[SFT_PREC_FP32];
    R.tconn = t->conn;
    R.vol32 = t->vol32;
    R.nv = t->nv;
    R.ne = t->ne;
    R.grid = (const GridP<float>*)L.grid;
    R.cell_start = L.cell_start;
    R.cell_items = L.cell_items;
    R.cell_first = L.cell_first;
    R.recs = (const float*)L.recs;
    R.adj = L.adj;
    R.vals = (const float*)L.vals;
    R.snf = s->nf;
    R.nf = o.field_count > 0 ? o.field_count : s->nf;
    R.N = o.samples_per_elem;
    const int spu = t->dim == 2 ? 2 : 1;
    R.U = (R.N + spu - 1) / spu;
    R.LPE = request_lpe(R, 0);  // lanes per element, as in the single-transfer kernel (until tuned)
    R.G = 32 / R.LPE;
    R.ntasks = (t->ne + R.G - 1) / R.G;
    R.key.k0 = (uint32_t)o.seed;
    R.key.k1 = (uint32_t)(o.seed >> 32);
    R.stream_id = o.stream_id;
    R.alpha = (float)o.alpha;
    R.c_det = (float)(o.alpha / (double)((t->dim + 1) * (t->dim + 2)));
    R.inv_n = (float)(1.0 / (double)R.N);
    R.st = strat_for(t->dim, R.N, opts[r].sampling);
    R.g = B->g + B->vec_off[r];
    R.b = B->b + B->vec_off[r];
    B->queries += t->nv + t->ne * (int64_t)R.N;
    const int cls = R.nf <= 2 ? 0 : (R.nf <= 4 ? 1 : 2);
    auto& G = B->grp[(t->dim - 2) * 3 + cls];
    G.req.push_back(r);
    auto& C = B->ctl[t->dim - 2];
    C.req.push_back(r);
  }
  for (auto& G : B->grp) {
    if (G.req.empty()) continue;
    G.off.assign(1, 0);
    for (int32_t r : G.req) G.off.push_back(G.off.back() + B->hreq[r].ntasks);
    G.total = G.off.back();
    if (sft_status e = upload(&G.dreq, G.req, st)) return e;
    if (sft_status e = upload(&G.doff, G.off, st)) return e;
    SFT_CUDA(dalloc(&G.work, 1, st));
  }
  for (int d = 0; d < 2; ++d) {
    auto& C = B->ctl[d];
    if (C.req.empty()) continue;
    C.off.assign(1, 0);
    for (int32_t r : C.req) C.off.push_back(C.off.back() + B->hreq[r].nv);
    C.total = C.off.back();
    if (sft_status e = upload(&C.dreq, C.req, st)) return e;
    if (sft_status e = upload(&C.doff, C.off, st)) return e;
  }
  if (sft_status e = upload(&B->dreq, B->hreq, st)) return e;
  // systems of the batched CG
  B->sys_first.resize(nreq + 1);
  for (int r = 0; r < nreq; ++r) B->mixed = B->mixed && opts[r].cg_mode == SFT_CG_MIXED;
  int64_t off = 0;
  for (int r = 0; r < nreq; ++r) {
    B->sys_first[r] = (int)B->hsys.size();
    sft_target t = B->tgts[r];
    if (B->mixed)
      if (sft_status e = scaled_matrix(t, st)) return e;
    for (int f = 0; f < B->hreq[r].nf; ++f) {
      BSys S;
      S.rp = t->row_ptr;
      S.col = t->col;
      S.val = t->val;
      S.dinv = t->dinv;
      S.aval = t->val32s;
      S.sc = t->sc;
      S.b = B->b + B->vec_off[r] + (int64_t)f * t->nv;
      S.x = B->u + B->vec_off[r] + (int64_t)f * t->nv;
      S.off = off;
      S.n = t->nv;
      S.tol = opts[r].cg_tol;
      S.max_iter = std::max(1, opts[r].cg_max_iter);
      S.lmax = t->dim == 2 ? 2.f : 2.5f;
      off += t->nv;
      B->hsys.push_back(S);
    }
  }
  B->sys_first[nreq] = (int)B->hsys.size();
  B->nsys = (int)B->hsys.size();
  B->ntot = off;
  int dev = 0, sms = 0, per_sm = 0;
  SFT_CUDA(cudaGetDevice(&dev));
  SFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (B->mixed)
    SFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_mixed, kBatchThreads, 0));
  else
    SFT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batch_pcg, kBatchThreads, 0));
  if (per_sm < 1) return fail(SFT_ERR_CUDA, "batched CG kernel cannot be resident");
  B->nblocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)std::min(per_sm, 4) * sms,
                                                           (B->ntot + kBatchThreads - 1) / kBatchThreads));
  B->rows_per_block = (B->ntot + B->nblocks - 1) / B->nblocks;
  std::vector<int32_t> slo(B->nblocks), shi(B->nblocks);
  if (B->mixed) {
    // pieces: whole matrix rows of one request with all its fields, in
    // request order (so a request's systems are owned by consecutive
    // blocks), an equal share of the estimated row cost per block. A row of
    // a request with z matrix entries per row and nf fields costs about
    // 8 z (its FP32 entries and columns, loaded once for all fields) +
    // nf (44 + 4 z) (per field the CG vectors of the two FP32 phases and
    // the z gathered entries of r): 3D rows (z ~ 15) cost about twice 2D
    // rows (z ~ 7), and a field of an 8-field row 0.6 of a lone field.
    std::vector<BPiece> hp;
    std::vector<int32_t> hbpc(B->nblocks + 1);
    std::vector<double> rcost(nreq, 0.0);
    double total = 0.0;
    for (int q = 0; q < nreq; ++q) {
      const sft_target tq = B->tgts[q];
      const int nf = B->hreq[q].nf;
      if (tq->nv <= 0 || nf < 1) continue;
      const double z = (double)tq->nnz / (double)tq->nv;
      rcost[q] = 8.0 * z + nf * (44.0 + 4.0 * z);
      total += rcost[q] * (double)tq->nv;
    }
    const double share = total / B->nblocks;
    int r = 0;
    int64_t i = 0;
    for (int b = 0; b < B->nblocks; ++b) {
      hbpc[b] = (int32_t)hp.size();
      const bool last = b == B->nblocks - 1;
      double budget = share;
      while ((last || budget > 0.0) && r < nreq) {
        const int64_t nv = B->tgts[r]->nv;
        const int nf = B->hreq[r].nf;
        if (i >= nv || nf < 1) {
          ++r;
          i = 0;
          continue;
        }
        int64_t take = nv - i;
        if (!last) take = std::min<int64_t>(take, std::max<int64_t>(1, (int64_t)std::ceil(budget / rcost[r])));
        hp.push_back(BPiece{B->sys_first[r], nf, i, i + take});
        i += take;
        budget -= (double)take * rcost[r];
      }
    }
    hbpc[B->nblocks] = (int32_t)hp.size();
    for (int s = 0; s < B->nsys; ++s) {
      B->hsys[s].blo = INT32_MAX;
      B->hsys[s].bhi = -1;
    }
    for (int b = 0; b < B->nblocks; ++b) {
      if (hbpc[b] == hbpc[b + 1]) {
        slo[b] = shi[b] = B->nsys - 1;
        continue;
      }
      const BPiece& first = hp[hbpc[b]];
      const BPiece& last = hp[hbpc[b + 1] - 1];
      slo[b] = first.s0;
      shi[b] = last.s0 + last.nf - 1;
      B->maxs = std::max(B->maxs, shi[b] - slo[b] + 1);
      for (int q = hbpc[b]; q < hbpc[b + 1]; ++q)
        for (int f = 0; f < hp[q].nf; ++f) {
          BSys& S = B->hsys[hp[q].s0 + f];
          S.blo = std::min(S.blo, (int32_t)b);
          S.bhi = std::max(S.bhi, (int32_t)b);
        }
    }
    for (int s = 0; s < B->nsys; ++s)
      if (B->hsys[s].bhi < 0) B->hsys[s].blo = B->hsys[s].bhi = 0;  // no rows
    if (sft_status e = upload(&B->pcs, hp, st)) return e;
    if (sft_status e = upload(&B->blk_pc, hbpc, st)) return e;
  } else {
    int s = 0;
    for (int b = 0; b < B->nblocks; ++b) {
      const int64_t r0 = (int64_t)b * B->rows_per_block;
      const int64_t r1 = std::min(B->ntot, r0 + B->rows_per_block) - 1;
      if (r0 > r1) {
        slo[b] = shi[b] = B->nsys - 1;
        continue;
      }
      while (s + 1 < B->nsys && B->hsys[s + 1].off <= r0) ++s;
      slo[b] = s;
      int e = s;
      while (e + 1 < B->nsys && B->hsys[e + 1].off <= r1) ++e;
      shi[b] = e;
      B->maxs = std::max(B->maxs, e - s + 1);
    }
    for (int s2 = 0; s2 < B->nsys; ++s2) {
      BSys& S = B->hsys[s2];
      if (S.n == 0) { S.blo = S.bhi = 0; continue; }
      S.blo = (int32_t)(S.off / B->rows_per_block);
      S.bhi = (int32_t)((S.off + S.n - 1) / B->rows_per_block);
    }
  }
  if (B->maxs > kMaxLocalSys) return fail(SFT_ERR_UNSUPPORTED, "too many small systems per CG block");
  if (sft_status e = upload(&B->dsys, B->hsys, st)) return e;
  if (sft_status e = upload(&B->blk_slo, slo, st)) return e;
  if (sft_status e = upload(&B->blk_shi, shi, st)) return e;
  SFT_CUDA(dalloc(&B->r, (size_t)B->ntot, st));
  SFT_CUDA(dalloc(&B->z, (size_t)B->ntot, st));
  SFT_CUDA(dalloc(&B->p, (size_t)B->ntot, st));
  SFT_CUDA(dalloc(&B->q, (size_t)B->ntot, st));
  SFT_CUDA(dalloc(&B->part, (size_t)B->nblocks * B->maxs * 2, st));
  SFT_CUDA(dalloc(&B->sysout, (size_t)std::max(1, B->nsys), st));
  SFT_CUDA(dalloc(&B->cgctl, 1, st));
  for (auto& e : B->ev) SFT_CUDA(cudaEventCreate(&e));
  int32_t herr = 0;
  SFT_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  dfree(d_err, st);
  if (herr) return fail(SFT_ERR_MESH, "a batch source mesh failed to build");
  // autotune the tile of every group (control values first)
  if (autotune) {
    SFT_CUDA(cudaMemsetAsync(B->counters, 0, sizeof(int64_t) * 2, st));
    for (int d = 0; d < 2; ++d) {
      auto& C = B->ctl[d];
      if (!C.total) continue;
      const unsigned blocks = (unsigned)std::min<int64_t>((C.total + kBatchThreads - 1) / kBatchThreads, 152 * 16);
      if (d == 0)
        ::sft::note_launch(), k_batch_control<2><<<blocks, kBatchThreads, sizeof(int64_t) * (C.req.size() + 1), st>>>(B->dreq, C.dreq, C.doff,
                                                                                    (int)C.req.size(), C.total, B->counters);
      else
        ::sft::note_launch(), k_batch_control<3><<<blocks, kBatchThreads, sizeof(int64_t) * (C.req.size() + 1), st>>>(B->dreq, C.dreq, C.doff,
                                                                                    (int)C.req.size(), C.total, B->counters);
      SFT_CUDA(cudaGetLastError());
    }
    for (int gi = 0; gi < 6; ++gi)
      if (B->grp[gi].total)
        if (sft_status e = autotune_group(B, gi, st)) return e;
  }
  // record the graph (fallback: direct launches)
  cudaStream_t cap = nullptr;
  SFT_CUDA(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (ok) {
    const int64_t l0 = launch_count();
    const sft_status e = enqueue_batch(B, cap);
    B->graph_kernels = launch_count() - l0;  // recorded, not run
    note_launches(-B->graph_kernels);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cap, &g);
    ok = e == SFT_OK && ce == cudaSuccess && g;
    if (ok) {
      B->graph = g;
      ok = cudaGraphInstantiate(&B->exec, g, 0) == cudaSuccess;
    } else if (g) {
      cudaGraphDestroy(g);
    }
  }
  cudaGetLastError();  // clear a failed capture
  cudaStreamDestroy(cap);
  B->graph_ok = ok;
  return SFT_OK;
}

}  // namespace sft

using namespace sft;

extern "C" {

sft_status sft_batch_create(int32_t nreq, const sft_source* srcs, const sft_target* tgts, const sft_options* opts,
                            int32_t autotune, void* cuda_stream, sft_batch* out) {
  if (!out) return fail(SFT_ERR_ARG, "null output handle");
  *out = nullptr;
  if (nreq < 1 || nreq > kMaxBatch) return fail(SFT_ERR_ARG, "nreq must be in 1..4096");
  if (!srcs || !tgts || !opts) return fail(SFT_ERR_ARG, "null request arrays");
  for (int r = 0; r < nreq; ++r) {
    if (!srcs[r] || !tgts[r]) return fail(SFT_ERR_ARG, "null source or target in the batch");
    if (srcs[r]->dim != tgts[r]->dim) return fail(SFT_ERR_ARG, "source and target dimensions differ");
    const sft_options& o = opts[r];
    if (o.precision != SFT_PREC_FP32) return fail(SFT_ERR_UNSUPPORTED, "batched transfers use the FP32 path");
    if (o.samples_per_elem < 1 || o.cg_max_iter < 0 || !(o.cg_tol >= 0) || !std::isfinite(o.alpha))
      return fail(SFT_ERR_ARG, "bad request options");
    if (o.cg_mode != SFT_CG_MIXED && o.cg_mode != SFT_CG_FP64) return fail(SFT_ERR_ARG, "unknown cg_mode");
    if (o.sampling == SFT_SAMPLING_IMPORTANCE || o.adapt_ref_measure != 0.0)
      return fail(SFT_ERR_UNSUPPORTED, "importance sampling and adaptive sample counts: sft_transfer only");
    if (o.sampling != SFT_SAMPLING_UNIFORM && o.sampling != SFT_SAMPLING_STRATIFIED)
      return fail(SFT_ERR_ARG, "unknown sampling scheme");
    if (o.cg_warm_start) return fail(SFT_ERR_UNSUPPORTED, "batched transfers start every solve from 0");
    if (o.sampling == SFT_SAMPLING_STRATIFIED && o.samples_per_elem > kMaxStratifiedN)
      return fail(SFT_ERR_UNSUPPORTED, "stratified sampling supports at most 2^20 samples per element");
    if (o.field_count < 0 || o.field_count > srcs[r]->nf) return fail(SFT_ERR_ARG, "field_count out of range");
  }
  auto* B = new sft_batch_s();
  B->nreq = nreq;
  B->stream = (cudaStream_t)cuda_stream;
  B->srcs.assign(srcs, srcs + nreq);
  B->tgts.assign(tgts, tgts + nreq);
  const sft_status r = build_batch(B, opts, autotune);
  if (r != SFT_OK) {
    free_batch(B);
    return r;
  }
  *out = B;
  return SFT_OK;
}

sft_status sft_batch_run(sft_batch B, void* cuda_stream, sft_batch_stats* stats) {
  if (!B) return fail(SFT_ERR_ARG, "null batch");
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : B->stream;
  if (B->graph_ok) {
    SFT_CUDA(cudaGraphLaunch(B->exec, st));
    note_launches(B->graph_kernels);
  } else {
    if (sft_status e = enqueue_batch(B, st)) return e;
  }
  std::vector<BSysOut> so((size_t)std::max(1, B->nsys));
  int64_t hc[2] = {0, 0};
  BCgCtl hctl;
  if (B->nsys) SFT_CUDA(cudaMemcpyAsync(so.data(), B->sysout, sizeof(BSysOut) * B->nsys, cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaMemcpyAsync(hc, B->counters, sizeof(hc), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaMemcpyAsync(&hctl, B->cgctl, sizeof(BCgCtl), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  if (hctl.err) return fail(SFT_ERR_DEVICE_STATUS, "batched CG: grid barrier wait expired");
  int maxit = 0, nonconv = 0;
  double maxrel = 0.0;
  for (int s = 0; s < B->nsys; ++s) {
    maxit = std::max(maxit, (int)so[s].iters);
    maxrel = std::max(maxrel, so[s].rel);
    nonconv += !so[s].conv;
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->nreq = B->nreq;
    stats->graph = B->graph_ok ? 1 : 0;
    stats->max_cg_iters = maxit;
    stats->nonconverged = nonconv;
    stats->max_rel_resid = maxrel;
    stats->queries = B->queries;
    stats->fallback_queries = hc[0];
    stats->empty_queries = hc[1];
    auto ms = [&](int a, int b) {
      float t = -1.f;
      if (cudaEventElapsedTime(&t, B->ev[a], B->ev[b]) != cudaSuccess) {
        t = -1.f;
        cudaGetLastError();  // timing unavailable: do not leave a sticky error behind
      }
      return t;
    };
    stats->ms_control = ms(0, 1);
    stats->ms_assembly = ms(1, 2);
    stats->ms_solve = ms(2, 3);
    stats->ms_total = ms(0, 3);
    for (int gi = 0; gi < 6; ++gi) stats->tile[gi] = B->grp[gi].total ? B->grp[gi].tile : 0;
  }
  if (nonconv) return fail(SFT_ERR_NOT_CONVERGED, "a batched system reached its iteration cap");
  return SFT_OK;
}

sft_status sft_batch_result(sft_batch B, int32_t req, double* u_out, double* b_out, int32_t out_device,
                            void* cuda_stream) {
  if (!B || req < 0 || req >= B->nreq || !u_out) return fail(SFT_ERR_ARG, "bad batch result request");
  cudaStream_t st = cuda_stream ? (cudaStream_t)cuda_stream : B->stream;
  const size_t bytes = sizeof(double) * (size_t)(B->vec_off[req + 1] - B->vec_off[req]);
  const cudaMemcpyKind k = out_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  SFT_CUDA(cudaMemcpyAsync(u_out, B->u + B->vec_off[req], bytes, k, st));
  if (b_out) SFT_CUDA(cudaMemcpyAsync(b_out, B->b + B->vec_off[req], bytes, k, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  return SFT_OK;
}

sft_status sft_batch_groups(sft_batch B, int32_t* out) {
  if (!B || !out) return fail(SFT_ERR_ARG, "null argument");
  for (int gi = 0; gi < 6; ++gi) {
    const auto& G = B->grp[gi];
    int32_t* o = out + gi * 5;
    o[0] = (int32_t)G.req.size();
    o[1] = gi < 3 ? 2 : 3;
    o[2] = gi % 3 == 0 ? 2 : (gi % 3 == 1 ? 4 : 8);
    o[3] = G.tile;
    int lpe = 0;
    for (int32_t r : G.req) lpe = std::max(lpe, B->hreq[r].LPE);
    o[4] = G.req.empty() ? 0 : (G.lpe > 0 ? G.lpe : lpe);
  }
  return SFT_OK;
}

void sft_batch_destroy(sft_batch B) {
  if (B) free_batch(B);
}

}  // extern "C"
