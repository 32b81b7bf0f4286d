// The fused control-variate Monte Carlo assembly (Sec. 4, steps 2-6;
// Eq. cv_element_load_residual_operator summed as in Eq. cv_load_expanded):
//
//   b_i += alpha int_t g psi_i                       (exact P1 mass, FP64)
//        + |T|/N sum_j (f^s - alpha g)(X_tj) psi_i(X_tj)
//
// Work mapping: a warp owns whole target elements. The unit of work is one
// Philox call: two samples in 2D, one in 3D. With U units per element, LPE =
// min(U, 4) lanes share an element (lanes stride over its units) and a warp
// holds floor(32/LPE) elements (lane -> element lane/LPE). Per sample a lane
// maps the draw into the element (psi_i(X) are the barycentric weights used
// to build X), locates X in the source grid, evaluates every field, forms the
// residual against the P1 control and accumulates r psi_i. FP32 partials are
// compensated (TwoSum). A segmented suffix scan over lanes combines the
// partials of each element; the segment head adds the deterministic control
// term and scatters k*nf FP64 atomics into b.
#include "accum.cuh"
#include "internal.hpp"
#include "util.cuh"

namespace sft {

struct AsmParams {
  int64_t nv, ne, snf;  // snf: the source's field count (stride of its value copies)
  int nf, N, U, G, LPE;
  int64_t ntasks;
  PhiloxRoundKeys rk;
  uint32_t stream_id;
  double alpha;
  double c_det;   // alpha / ((d+1)(d+2)): exact P1 mass factor of the control term
  double inv_n;   // 1 / N
  Strat st;       // sampling scheme (st.n = 0: uniform)
  int imp;        // importance sampling (the EXT kernel)
  int adapt;      // per-element sample counts (the EXT kernel)
  double dref;    // d! x the reference measure of the adaptive count
  int nmax;       // samples per element at most (row length of sample_elem)
  const int32_t* nt;  // per-element sample counts (p.adapt; k_adaptive_counts)
};

// Adaptive sample count of an element (the EXT kernel): N_t = min(8 N,
// max(1, ceil(N D / dref))) with D = d! |T| the edge determinant of its
// vertices in P, evaluated in FP64 left to right (the oracle's order).
template <int D, typename P>
__device__ __forceinline__ int adaptive_count(const P xv[D + 1][D], int N, double dref) {
  double x[D + 1][D];
#pragma unroll
  for (int m = 0; m <= D; ++m)
#pragma unroll
    for (int a = 0; a < D; ++a) x[m][a] = f2d(xv[m][a]);
  double det;
  if constexpr (D == 2) {
    det = __dsub_rn(__dmul_rn(__dsub_rn(x[1][0], x[0][0]), __dsub_rn(x[2][1], x[0][1])),
                    __dmul_rn(__dsub_rn(x[2][0], x[0][0]), __dsub_rn(x[1][1], x[0][1])));
  } else {
    double e1[3], e2[3], e3[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      e1[a] = __dsub_rn(x[1][a], x[0][a]);
      e2[a] = __dsub_rn(x[2][a], x[0][a]);
      e3[a] = __dsub_rn(x[3][a], x[0][a]);
    }
    const double t0 = __dmul_rn(e1[0], __dsub_rn(__dmul_rn(e2[1], e3[2]), __dmul_rn(e2[2], e3[1])));
    const double t1 = __dmul_rn(e1[1], __dsub_rn(__dmul_rn(e2[0], e3[2]), __dmul_rn(e2[2], e3[0])));
    const double t2 = __dmul_rn(e1[2], __dsub_rn(__dmul_rn(e2[0], e3[1]), __dmul_rn(e2[1], e3[0])));
    det = __dadd_rn(__dsub_rn(t0, t1), t2);
  }
  const double q = ceil(__ddiv_rn(__dmul_rn((double)N, det), dref));
  const double cap = 8.0 * (double)N;
  return (int)(q < 1.0 ? 1.0 : (q > cap ? cap : q));
}

// The adaptive count of every target element, once per assembly: the FP64
// determinant runs with every lane of a warp busy (inside the assembly only
// the 8 lanes that count the warp's 8 elements would be: tet5m assembly
// 2.67 ms with the counts inline).
template <int D, typename P>
__global__ void k_adaptive_counts(const P* __restrict__ tx, const int32_t* __restrict__ tconn, int64_t ne, int N,
                                  double dref, int32_t* __restrict__ nt) {
  constexpr int K = D + 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    P xv[K][D];
#pragma unroll
    for (int m = 0; m < K; ++m) {
      const int32_t vm = __ldg(tconn + e * K + m);
#pragma unroll
      for (int a = 0; a < D; ++a) xv[m][a] = __ldg(tx + (int64_t)vm * D + a);
    }
    nt[e] = adaptive_count<D, P>(xv, N, dref);
  }
}

// MODE: kAsmPlain; kAsmDebug also writes the source element of every sample
// (sample_elem); kAsmRecord also writes its barycentric coordinates mu_1..d
// (pmu, [d][N ne]) for later online transfers; kAsmCached takes element and
// mu from those arrays instead of locating the sample (the samples' target
// weights are regenerated from the same Philox counters).
// Four resident blocks per SM (64 registers a thread) in both dimensions:
// the kernel is bound by the latency of its dependent cache loads (cell ->
// start element -> record -> neighbour -> record), and more resident warps
// would hide more of it, but at five or six blocks the register cap spills
// inside the walk. Measured on tri4m: 1.265 ms at four blocks, 1.406 at five;
// tet5m 2.110 at four, 2.219 at five, 2.132 at six.
// EXT: the kernel with importance sampling (p.imp) and per-element sample
// counts (p.adapt); without it the kernel is the uniform / stratified one.
template <int D, typename P, int NF, int MODE, bool EXT>
__global__ void __launch_bounds__(256, 4) k_assemble(const P* __restrict__ tx, const int32_t* __restrict__ tconn,
                                                  const double* __restrict__ vol, const float* __restrict__ vol32,
                                                  const P* __restrict__ g,
                                                  const GridP<P>* __restrict__ gp,
                                                  const int32_t* __restrict__ cell_start,
                                                  const int32_t* __restrict__ cell_items,
                                                  const int32_t* __restrict__ cell_first,
                                                  const P* __restrict__ recs, const int32_t* __restrict__ adj,
                                                  const P* __restrict__ vals,
                                                  AsmParams p, double* __restrict__ b,
                                                  int32_t* __restrict__ sample_elem, P* __restrict__ pmu,
                                                  int64_t* __restrict__ counters) {
  using A = Ar<P>;
  constexpr int K = D + 1;
  constexpr int SPU = D == 2 ? 2 : 1;  // samples per Philox call
  GridP<P> gr;
  if (MODE != kAsmCached) gr = *gp;
  const int lane = threadIdx.x & 31;
  const int64_t ns = p.ne * (int64_t)p.N;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const P alphaP = (P)p.alpha;
  const int snf = NF == 1 ? 1 : (int)p.snf;  // value-copy stride (NF = 1: one-field sources only)
  int n_fallback = 0, n_empty = 0;

  // importance sampling draws one sample per unit (two Philox blocks)
  const int spu = EXT && p.imp ? 1 : SPU;
  for (int64_t task = warp0; task < p.ntasks; task += nwarps) {
    int64_t t;
    int u0, ustep, seg_lo, seg_hi;
    bool active;
    int Nt = p.N;   // this element's samples
    int span = p.LPE;
    if (EXT && p.adapt) {
      // per-element counts: the G elements of the task share the 32 lanes in
      // proportion to their units (each at least one lane), so a warp runs
      // as long as its mean element, not its largest. Lane s < G reads the
      // count of element s; slot s starts at lane s + floor((32 - G) C_s / C),
      // C_s the units of the slots before it and C the task's total.
      const int64_t ts = task * p.G + lane;
      const int Ns = lane < p.G && ts < p.ne ? __ldg(p.nt + ts) : 0;
      const int Us = (Ns + spu - 1) / spu;
      int cum = Us;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, cum, o);
        if (lane >= o) cum += y;
      }
      const int tot = __shfl_sync(0xffffffffu, cum, 31);
      const int start = lane + (tot > 0 ? (int)((int64_t)(32 - p.G) * (cum - Us) / tot) : lane * (32 / p.G - 1));
      int slot = 0;
      for (int q = 1; q < p.G; ++q) slot += __shfl_sync(0xffffffffu, start, q) <= lane;
      seg_lo = __shfl_sync(0xffffffffu, start, slot);
      const int nxt = __shfl_sync(0xffffffffu, start, slot + 1 < p.G ? slot + 1 : slot);
      seg_hi = slot + 1 < p.G ? nxt : 32;
      Nt = __shfl_sync(0xffffffffu, Ns, slot);
      span = (int)__reduce_max_sync(0xffffffffu, (unsigned)(seg_hi - seg_lo));
      t = task * p.G + slot;
      u0 = lane - seg_lo;
      ustep = seg_hi - seg_lo;
      active = true;
    } else {
      // G elements per warp, LPE = lanes per element; lanes stride over the
      // element's units
      const int slot = lane / p.LPE;
      t = task * p.G + slot;
      u0 = lane - slot * p.LPE;
      ustep = p.LPE;
      seg_lo = slot * p.LPE;
      seg_hi = seg_lo + p.LPE;
      active = slot < p.G;
    }
    active = active && t < p.ne;

    int32_t v[K];
    P xv[K][D];
    P gl[NF][K];
    Acc<P> acc[NF][K];
    if (active) {
#pragma unroll
      for (int m = 0; m < K; ++m) {
        v[m] = __ldg(tconn + t * K + m);
#pragma unroll
        for (int a = 0; a < D; ++a) xv[m][a] = MODE == kAsmCached ? P(0) : __ldg(tx + (int64_t)v[m] * D + a);
#pragma unroll
        for (int f = 0; f < NF; ++f) gl[f][m] = f < p.nf ? __ldg(g + (int64_t)f * p.nv + v[m]) : P(0);
      }
    }
    const int Ut = EXT ? (Nt + spu - 1) / spu : p.U;
    if (EXT && MODE == kAsmDebug && active && lane == seg_lo)
      for (int j = Nt; j < p.nmax; ++j) sample_elem[t * p.nmax + j] = -1;

    for (int u = u0; active && u < Ut; u += ustep) {
      uint4 w, wb;
      if (EXT && p.imp) {
        w = philox4x32_10(make_uint4((uint32_t)u, (uint32_t)t, p.stream_id, 6u), p.rk);
        wb = philox4x32_10(make_uint4((uint32_t)u, (uint32_t)t, p.stream_id, 7u), p.rk);
      } else {
        w = philox4x32_10(make_uint4((uint32_t)u, (uint32_t)t, p.stream_id, 0u), p.rk);
      }
#pragma unroll
      for (int s = 0; s < SPU; ++s) {
        const int j = EXT && p.imp ? u : SPU * u + s;
        if ((EXT && p.imp && s > 0) || j >= Nt) break;
        P lam[K];
        P wgt = P(1);
        if (EXT && p.imp) wgt = importance_lambda<D, P>(w, wb, lam);
        else sample_lambda<D, P>(w, j, p.st, lam);
        P mu[K];
        int status = 0;
        int32_t e;
        const int64_t idx = t * (EXT ? p.nmax : p.N) + j;
        if constexpr (MODE == kAsmCached) {
          e = __ldg(sample_elem + idx);
          P m0 = P(1);
#pragma unroll
          for (int a = 0; a < D; ++a) {
            mu[a + 1] = __ldg(pmu + a * ns + idx);
            m0 = A::sub(m0, mu[a + 1]);  // the predicate's mu_0, bit for bit
          }
          mu[0] = m0;
        } else {
          P X[D];
          map_point<D, P>(lam, xv, X);
          e = locate_point<D, P>(gr, cell_start, cell_items, cell_first, recs, adj, X, mu, status);
          if (MODE != kAsmPlain) sample_elem[idx] = e;
          if (MODE == kAsmRecord) {
#pragma unroll
            for (int a = 0; a < D; ++a) pmu[a * ns + idx] = mu[a + 1];
          }
        }
        n_fallback += status == 1;
        n_empty += status == 2;
#pragma unroll
        for (int f = 0; f < NF; ++f) {
          if (f >= p.nf) break;
          const P fs = e >= 0 ? eval_p1<D, P>(vals, snf, f, e, mu) : P(0);
          P gX = A::mul(gl[f][0], lam[0]);
#pragma unroll
          for (int m = 1; m < K; ++m) gX = A::fma(gl[f][m], lam[m], gX);
          P r = A::sub(fs, A::mul(alphaP, gX));
          if (EXT && p.imp) r = A::mul(wgt, r);   // w_j (f^s - alpha g): the density's weight
          acc_add_sample<K>(acc[f], r, lam);
        }
      }
    }

    // segmented suffix combine: lane seg_lo ends with its element's totals
    // (log2 of the longest segment rounds: LPE lanes, or with per-element
    // counts the task's widest lane range)
    for (int o = 1; o < span; o <<= 1) {
      const bool take = lane + o < seg_hi;
#pragma unroll
      for (int f = 0; f < NF; ++f)
#pragma unroll
        for (int i = 0; i < K; ++i) {
          const P s2 = __shfl_down_sync(0xffffffffu, acc[f][i].s, o);
          const P e2 = __shfl_down_sync(0xffffffffu, acc[f][i].e, o);
          if (take) acc[f][i].combine(s2, e2);
        }
    }

    if (active && lane == seg_lo) {
      const double w = sizeof(P) == 8 ? __ldg(vol + t) : 0.0;
      const float wf = sizeof(P) == 4 ? __ldg(vol32 + t) : 0.f;
      const P cdet = (P)p.c_det;
      const P cmc = EXT && p.adapt ? (P)__drcp_rn((double)Nt) : (P)p.inv_n;   // 1 / N_t
      if (EXT && counters) atomicAdd(reinterpret_cast<unsigned long long*>(counters + 2), (unsigned long long)Nt);
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        if (f >= p.nf) break;
        P gsum = gl[f][0];
#pragma unroll
        for (int m = 1; m < K; ++m) gsum = A::add(gsum, gl[f][m]);
#pragma unroll
        for (int i = 0; i < K; ++i)
          atomicAdd(b + (int64_t)f * p.nv + v[i], Epi<P>::contrib(wf, w, cdet, cmc, gsum, gl[f][i], acc[f][i]));
      }
    }
  }
  const int fb = warp_sum<int>(n_fallback), em = warp_sum<int>(n_empty);
  if (lane == 0 && counters) {
    if (fb) atomicAdd(reinterpret_cast<unsigned long long*>(counters), (unsigned long long)fb);
    if (em) atomicAdd(reinterpret_cast<unsigned long long*>(counters + 1), (unsigned long long)em);
  }
}

template <int D, typename P, int NF>
static void launch_t(sft_source_s* s, sft_target_s* t, const AssembleArgs& a, const AsmParams& p, cudaStream_t st) {
  const Locator& L = s->loc[a.prec];
  const int threads = 256;
  const int64_t warps_needed = p.ntasks;
  int64_t blocks = (warps_needed + (threads / 32) - 1) / (threads / 32);
  if (blocks > (1 << 20)) blocks = 1 << 20;
  if (blocks < 1) blocks = 1;
  auto args = [&](auto kern) {
    ::sft::note_launch(), kern<<<(unsigned)blocks, threads, 0, st>>>((const P*)t->coordsP[a.prec], t->conn, t->vol, t->vol32, (const P*)a.g,
                                               (const GridP<P>*)L.grid, L.cell_start, L.cell_items, L.cell_first,
                                               (const P*)L.recs, L.adj, (const P*)L.vals, p, a.b, a.sample_elem,
                                               (P*)a.pmu, a.counters);
  };
  const bool ext = p.imp || p.adapt;  // only with the plain and debug modes (checked by the callers)
  if (a.mode == kAsmCached) args(k_assemble<D, P, NF, kAsmCached, false>);
  else if (a.mode == kAsmRecord) args(k_assemble<D, P, NF, kAsmRecord, false>);
  else if (a.sample_elem) {
    if (ext) args(k_assemble<D, P, NF, kAsmDebug, true>);
    else args(k_assemble<D, P, NF, kAsmDebug, false>);
  } else {
    if (ext) args(k_assemble<D, P, NF, kAsmPlain, true>);
    else args(k_assemble<D, P, NF, kAsmPlain, false>);
  }
}

// NF = 1 only for a one-field source (the kernel then takes the value-copy
// stride as the constant 1); one field of a multi-field source goes to NF = 2
template <int D, typename P>
static void launch_nf(sft_source_s* s, sft_target_s* t, const AssembleArgs& a, const AsmParams& p, cudaStream_t st) {
  if (a.nf <= 1 && s->nf == 1) launch_t<D, P, 1>(s, t, a, p, st);
  else if (a.nf <= 2) launch_t<D, P, 2>(s, t, a, p, st);
  else if (a.nf <= 4) launch_t<D, P, 4>(s, t, a, p, st);
  else launch_t<D, P, 8>(s, t, a, p, st);
}

sft_status launch_assembly(sft_source_s* s, sft_target_s* t, const AssembleArgs& a, cudaStream_t st) {
  if (t->ne == 0) return SFT_OK;
  AsmParams p;
  p.nv = t->nv;
  p.ne = t->ne;
  p.snf = s->nf;
  p.nf = a.nf;
  p.N = a.N;
  const int spu = t->dim == 2 ? 2 : 1;
  p.U = (a.N + spu - 1) / spu;
  // 4 lanes per element (8 elements per warp): every lane runs a loop over
  // several units, and the per-element reduction is 2 shuffle rounds shared
  // by 8 elements (measured on GB300: 1.68x over one element per warp on the
  // 2D benchmark, 1.6x in 3D; 8 and 2 lanes per element are slower)
  p.LPE = p.U >= 4 ? 4 : p.U;
  p.G = 32 / p.LPE;
  p.ntasks = (t->ne + p.G - 1) / p.G;
  p.rk = philox_round_keys(a.seed);
  p.stream_id = a.stream_id;
  p.alpha = a.alpha;
  p.c_det = a.alpha / (double)((t->dim + 1) * (t->dim + 2));
  p.inv_n = 1.0 / (double)a.N;
  p.st = strat_for(t->dim, a.N, a.sampling);
  p.imp = a.sampling == SFT_SAMPLING_IMPORTANCE ? 1 : 0;
  p.adapt = a.adapt_ref > 0.0 ? 1 : 0;
  p.dref = a.adapt_ref * (t->dim == 2 ? 2.0 : 6.0);
  p.nmax = p.adapt ? 8 * a.N : a.N;
  p.nt = nullptr;
  DevBuf<int32_t> nt(st);  // freed in stream order after the launches
  if (p.adapt) {
    SFT_CUDA(nt.alloc((size_t)t->ne));
    int dev = 0, sms = 1;
    SFT_CUDA(cudaGetDevice(&dev));
    SFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t want = (t->ne + 255) / 256;
    const unsigned nb = (unsigned)(want < 16LL * sms ? want : 16LL * sms);
    const void* tx = t->coordsP[a.prec];
    if (t->dim == 2 && a.prec == SFT_PREC_FP32)
      ::sft::note_launch(), k_adaptive_counts<2, float><<<nb, 256, 0, st>>>((const float*)tx, t->conn, t->ne, a.N, p.dref, nt.p);
    else if (t->dim == 2)
      ::sft::note_launch(), k_adaptive_counts<2, double><<<nb, 256, 0, st>>>((const double*)tx, t->conn, t->ne, a.N, p.dref, nt.p);
    else if (a.prec == SFT_PREC_FP32)
      ::sft::note_launch(), k_adaptive_counts<3, float><<<nb, 256, 0, st>>>((const float*)tx, t->conn, t->ne, a.N, p.dref, nt.p);
    else
      ::sft::note_launch(), k_adaptive_counts<3, double><<<nb, 256, 0, st>>>((const double*)tx, t->conn, t->ne, a.N, p.dref, nt.p);
    SFT_CUDA(cudaGetLastError());
    p.nt = nt.p;
  }
  if (t->dim == 2) {
    if (a.prec == SFT_PREC_FP32) launch_nf<2, float>(s, t, a, p, st);
    else launch_nf<2, double>(s, t, a, p, st);
  } else {
    if (a.prec == SFT_PREC_FP32) launch_nf<3, float>(s, t, a, p, st);
    else launch_nf<3, double>(s, t, a, p, st);
  }
  SFT_CUDA(cudaGetLastError());
  return SFT_OK;
}

}  // namespace sft
