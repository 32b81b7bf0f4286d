// Transfer plans: the paper's split of the transfer into an initialization,
// paid once per pair of fixed meshes (localization of the target nodes and of
// every sample point, Sec. 5.3), and an online part paid per coupling
// iteration (evaluation of the integrals with the source's current values and
// the global solve).
//
// sft_plan_create runs steps 1-6 once in record mode: for every target node
// and every sample it keeps the located source element and the barycentric
// coordinates mu_1..d (mu_0 is recomputed from them exactly as the predicate
// forms it). sft_plan_transfer then evaluates the control values and the
// load vector from those records and the source's current nodal values (set
// with sft_source_set_values), regenerating each sample's target weights from
// its Philox counter, and solves M u = b. The result equals sft_transfer with
// the same options and values up to the order of the floating-point sums.
#include <algorithm>
#include <cmath>
#include <cstring>
#include "internal.hpp"
#include "util.cuh"

struct sft_plan_s {
  sft_source_s* src = nullptr;
  sft_target_s* tgt = nullptr;
  sft_options opt{};
  int prec = SFT_PREC_FP32;
  int nf = 1;
  cudaStream_t stream = nullptr;
  int32_t* node_elem = nullptr;  // [nv_t]
  void* node_mu = nullptr;       // [d][nv_t] P
  int32_t* samp_elem = nullptr;  // [ne_t N]
  void* samp_mu = nullptr;       // [d][ne_t N] P
  int64_t fallback = 0, empty = 0;
  size_t bytes = 0;
};

namespace sft {

// control values g[f][i] = f^s at target node i from its recorded location
template <int D, typename P>
__global__ void k_plan_control(const int32_t* __restrict__ node_elem, const P* __restrict__ node_mu, int64_t nv,
                               const P* __restrict__ vals, int snf, int nf, P* __restrict__ g) {
  using A = Ar<P>;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t e = __ldg(node_elem + i);
    P mu[D + 1];
    P m0 = P(1);
#pragma unroll
    for (int a = 0; a < D; ++a) {
      mu[a + 1] = __ldg(node_mu + a * nv + i);
      m0 = A::sub(m0, mu[a + 1]);
    }
    mu[0] = m0;
    for (int f = 0; f < nf; ++f) g[(int64_t)f * nv + i] = e >= 0 ? eval_p1<D, P>(vals, snf, f, e, mu) : P(0);
  }
}

}  // namespace sft

using namespace sft;

extern "C" {

sft_status sft_plan_create(sft_source s, sft_target t, const sft_options* o, sft_plan* out) {
  if (!out) return fail(SFT_ERR_ARG, "null output handle");
  *out = nullptr;
  if (!s || !t || !o) return fail(SFT_ERR_ARG, "null argument");
  if (s->dim != t->dim) return fail(SFT_ERR_ARG, "source and target dimensions differ");
  if (o->samples_per_elem < 1) return fail(SFT_ERR_ARG, "samples_per_elem must be >= 1");
  if ((int64_t)o->samples_per_elem * t->ne >= ((int64_t)1 << 40)) return fail(SFT_ERR_UNSUPPORTED, "too many samples");
  if (o->precision != SFT_PREC_FP32 && o->precision != SFT_PREC_FP64) return fail(SFT_ERR_ARG, "bad precision");
  if (o->cg_max_iter < 0 || !(o->cg_tol >= 0) || !std::isfinite(o->alpha)) return fail(SFT_ERR_ARG, "bad solver options");
  if (o->cg_mode != SFT_CG_MIXED && o->cg_mode != SFT_CG_FP64) return fail(SFT_ERR_ARG, "unknown cg_mode");
  if (o->sampling == SFT_SAMPLING_IMPORTANCE || o->adapt_ref_measure != 0.0)
    return fail(SFT_ERR_UNSUPPORTED, "importance sampling and adaptive sample counts: sft_transfer only");
  if (o->sampling != SFT_SAMPLING_UNIFORM && o->sampling != SFT_SAMPLING_STRATIFIED)
    return fail(SFT_ERR_ARG, "unknown sampling scheme");
  if (o->cg_warm_start != 0 && o->cg_warm_start != 1) return fail(SFT_ERR_ARG, "cg_warm_start must be 0 or 1");
  if (o->cg_warm_start && o->cg_mode != SFT_CG_MIXED) return fail(SFT_ERR_UNSUPPORTED, "a warm start needs cg_mode MIXED");
  if (o->sampling == SFT_SAMPLING_STRATIFIED && o->samples_per_elem > kMaxStratifiedN)
    return fail(SFT_ERR_UNSUPPORTED, "stratified sampling supports at most 2^20 samples per element");
  if (o->field_count < 0 || o->field_count > s->nf) return fail(SFT_ERR_ARG, "field_count out of range");
  cudaStream_t st = (cudaStream_t)o->cuda_stream;
  const int prec = o->precision;
  const int d = t->dim;
  const size_t psz = prec == SFT_PREC_FP32 ? 4 : 8;
  const int64_t nv = t->nv, ne = t->ne, ns = ne * (int64_t)o->samples_per_elem;
  DevBuf<int32_t> d_err(st);
  SFT_CUDA(d_err.alloc(1));
  SFT_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int32_t), st));
  if (sft_status r = build_locator(s, prec, st, d_err.p)) return r;
  if (sft_status r = target_coordsP(t, prec, st)) return r;
  auto* pl = new sft_plan_s();
  pl->src = s;
  pl->tgt = t;
  pl->opt = *o;
  pl->prec = prec;
  pl->nf = o->field_count > 0 ? o->field_count : s->nf;
  pl->stream = st;
  sft_status r = SFT_OK;
  do {
    cudaError_t e = dalloc(&pl->node_elem, (size_t)nv, st);
    if (e == cudaSuccess) e = pool_alloc(&pl->node_mu, psz * d * (size_t)nv, st);
    if (e == cudaSuccess) e = dalloc(&pl->samp_elem, (size_t)ns, st);
    if (e == cudaSuccess) e = pool_alloc(&pl->samp_mu, psz * d * (size_t)ns, st);
    if (e != cudaSuccess) { r = cuda_fail(e, "plan arrays"); break; }
    pl->bytes = sizeof(int32_t) * (size_t)(nv + ns) + psz * d * (size_t)(nv + ns);
    DevBuf<char> g(st);
    DevBuf<double> b(st);
    DevBuf<int64_t> counters(st);
    e = g.alloc(psz * nv * pl->nf);
    if (e == cudaSuccess) e = b.alloc((size_t)nv * pl->nf);
    if (e == cudaSuccess) e = counters.alloc(2);
    if (e == cudaSuccess) e = cudaMemsetAsync(b.p, 0, sizeof(double) * nv * pl->nf, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(counters.p, 0, sizeof(int64_t) * 2, st);
    if (e != cudaSuccess) { r = cuda_fail(e, "plan scratch"); break; }
    // step 1 recorded: node locations (and this round's control values)
    if ((r = locate_points(s, prec, nv, t->coordsP[prec], prec == SFT_PREC_FP64, pl->node_elem, g.p,
                           prec == SFT_PREC_FP64, nv, counters.p, st, pl->nf, pl->node_mu)))
      break;
    // steps 2-6 recorded: every sample's element and mu
    AssembleArgs a;
    a.prec = prec;
    a.nf = pl->nf;
    a.N = o->samples_per_elem;
    a.seed = o->seed;
    a.stream_id = o->stream_id;
    a.alpha = o->alpha;
    a.g = g.p;
    a.b = b.p;
    a.sample_elem = pl->samp_elem;
    a.counters = counters.p;
    a.mode = kAsmRecord;
    a.pmu = pl->samp_mu;
    a.sampling = o->sampling;
    if ((r = launch_assembly(s, t, a, st))) break;
    int64_t hc[2] = {0, 0};
    int32_t herr = 0;
    e = cudaMemcpyAsync(hc, counters.p, sizeof(hc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { r = cuda_fail(e, "plan record"); break; }
    if (herr) { r = fail(SFT_ERR_DEVICE_STATUS, "a plan kernel reported an error"); break; }
    pl->fallback = hc[0];
    pl->empty = hc[1];
    if (o->strict_inside && hc[1] > 0) { r = fail(SFT_ERR_OUTSIDE, "a query fell in an empty grid cell"); break; }
  } while (false);
  if (r != SFT_OK) {
    sft_plan_destroy(pl);
    return r;
  }
  *out = pl;
  return SFT_OK;
}

sft_status sft_plan_transfer(sft_plan pl, double* u_out, double* b_out, double* g_out, sft_stats* stats) {
  if (!pl || !u_out) return fail(SFT_ERR_ARG, "null argument");
  const sft_options& o = pl->opt;
  sft_source_s* s = pl->src;
  sft_target_s* t = pl->tgt;
  cudaStream_t st = pl->stream;
  const int prec = pl->prec, nf = pl->nf;
  const int64_t nv = t->nv, ne = t->ne;
  const size_t psz = prec == SFT_PREC_FP32 ? 4 : 8;
  const Locator& L = s->loc[prec];
  Events ev;
  if (ev.ok) cudaEventRecord(ev.e[0], st);
  DevBuf<int32_t> d_err(st);
  DevBuf<char> g(st);
  DevBuf<double> b(st), u_tmp(st);
  SFT_CUDA(d_err.alloc(1));
  SFT_CUDA(g.alloc(psz * nv * nf));
  SFT_CUDA(b.alloc((size_t)nv * nf));
  SFT_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int32_t), st));
  SFT_CUDA(cudaMemsetAsync(b.p, 0, sizeof(double) * nv * nf, st));
  if (ev.ok) cudaEventRecord(ev.e[1], st);
  // step 1 online: control values from the recorded node locations
  const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((nv + 255) / 256, 152 * 16));
  if (t->dim == 2) {
    if (prec == SFT_PREC_FP32)
      ::sft::note_launch(), k_plan_control<2, float><<<nb, 256, 0, st>>>(pl->node_elem, (const float*)pl->node_mu, nv,
                                                                        (const float*)L.vals, s->nf, nf, (float*)g.p);
    else
      ::sft::note_launch(), k_plan_control<2, double><<<nb, 256, 0, st>>>(pl->node_elem, (const double*)pl->node_mu, nv,
                                                                         (const double*)L.vals, s->nf, nf, (double*)g.p);
  } else {
    if (prec == SFT_PREC_FP32)
      ::sft::note_launch(), k_plan_control<3, float><<<nb, 256, 0, st>>>(pl->node_elem, (const float*)pl->node_mu, nv,
                                                                        (const float*)L.vals, s->nf, nf, (float*)g.p);
    else
      ::sft::note_launch(), k_plan_control<3, double><<<nb, 256, 0, st>>>(pl->node_elem, (const double*)pl->node_mu, nv,
                                                                         (const double*)L.vals, s->nf, nf, (double*)g.p);
  }
  SFT_CUDA(cudaGetLastError());
  if (ev.ok) cudaEventRecord(ev.e[2], st);
  // steps 2-6 online
  AssembleArgs a;
  a.prec = prec;
  a.nf = nf;
  a.N = o.samples_per_elem;
  a.seed = o.seed;
  a.stream_id = o.stream_id;
  a.alpha = o.alpha;
  a.g = g.p;
  a.b = b.p;
  a.sample_elem = pl->samp_elem;
  a.counters = nullptr;
  a.mode = kAsmCached;
  a.pmu = pl->samp_mu;
  a.sampling = o.sampling;
  if (sft_status r = launch_assembly(s, t, a, st)) return r;
  if (ev.ok) cudaEventRecord(ev.e[3], st);
  // step 7
  double* u_dev = u_out;
  if (!o.out_device) {
    SFT_CUDA(u_tmp.alloc((size_t)nv * nf));
    u_dev = u_tmp.p;
    if (o.cg_warm_start)
      SFT_CUDA(cudaMemcpyAsync(u_dev, u_out, sizeof(double) * nv * nf, cudaMemcpyHostToDevice, st));
  }
  SolveResult sr;
  SolveLate late(st);  // the solve's status is read with the final readback
  if (sft_status r = mass_solve(t, nf, b.p, u_dev, o.cg_tol, o.cg_max_iter, st, d_err.p, &sr, o.cg_mode, &late,
                                o.cg_warm_start))
    return r;
  if (ev.ok) cudaEventRecord(ev.e[4], st);
  const cudaMemcpyKind d2o = o.out_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (!o.out_device) SFT_CUDA(cudaMemcpyAsync(u_out, u_dev, sizeof(double) * nv * nf, d2o, st));
  if (b_out) SFT_CUDA(cudaMemcpyAsync(b_out, b.p, sizeof(double) * nv * nf, d2o, st));
  DevBuf<double> g64(st);
  if (g_out) {
    if (prec == SFT_PREC_FP64) {
      SFT_CUDA(cudaMemcpyAsync(g_out, g.p, sizeof(double) * nv * nf, d2o, st));
    } else {
      SFT_CUDA(g64.alloc((size_t)nv * nf));
      if (sft_status r = convert_coords(g.p, SFT_F32, g64.p, SFT_PREC_FP64, nv * nf, st)) return r;
      SFT_CUDA(cudaMemcpyAsync(g_out, g64.p, sizeof(double) * nv * nf, d2o, st));
    }
  }
  int32_t herr = 0;
  SFT_CUDA(cudaMemcpyAsync(&herr, d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (late.pending) SFT_CUDA(cudaMemcpyAsync(late.host, late.buf.p, late.bytes, cudaMemcpyDeviceToHost, st));
  if (ev.ok) cudaEventRecord(ev.e[5], st);
  SFT_CUDA(cudaStreamSynchronize(st));
  if (sft_status r = finish_solve(late, &sr)) return r;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->cg_iters = sr.iters;
    stats->cg_rel_resid = sr.rel_resid;
    stats->queries = nv + ne * (int64_t)o.samples_per_elem;
    stats->fallback_queries = pl->fallback;
    stats->empty_queries = pl->empty;
    stats->ms_setup = ev.ms(0, 1);
    stats->ms_control = ev.ms(1, 2);
    stats->ms_assembly = ev.ms(2, 3);
    stats->ms_solve = ev.ms(3, 4);
    stats->ms_total = ev.ms(0, 5);
  }
  if (herr) return fail(SFT_ERR_DEVICE_STATUS, "a transfer kernel reported an error");
  if (!sr.converged && o.cg_max_iter > 0) return fail(SFT_ERR_NOT_CONVERGED, "CG reached cg_max_iter");
  return SFT_OK;
}

int64_t sft_plan_bytes(sft_plan pl) { return pl ? (int64_t)pl->bytes : 0; }

void sft_plan_destroy(sft_plan pl) {
  if (!pl) return;
  dfree(pl->node_elem, pl->stream);
  if (pl->node_mu) cudaFreeAsync(pl->node_mu, pl->stream);
  dfree(pl->samp_elem, pl->stream);
  if (pl->samp_mu) cudaFreeAsync(pl->samp_mu, pl->stream);
  cudaStreamSynchronize(pl->stream);
  delete pl;
}

}  // extern "C"
