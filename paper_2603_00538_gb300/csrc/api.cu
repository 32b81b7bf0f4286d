// C ABI of libsft (declared in include/sft.h): argument validation, device
// copies of the meshes, the order of the transfer steps (Sec. 4, steps 1-7),
// host staging of host-memory outputs, timing events and status mapping.
#include <cmath>
#include <cstring>
#include <atomic>
#include <mutex>
#include <string>
#include <vector>
#include "internal.hpp"
#include "util.cuh"

namespace sft {

static thread_local std::string g_last_error;
static std::atomic<int64_t> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void note_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

void set_last_error(const std::string& msg) { g_last_error = msg; }

sft_status fail(sft_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

sft_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? SFT_ERR_OOM : SFT_ERR_CUDA;
}

// Keep freed stream-ordered allocations in the device's default pool (the
// create/transfer/destroy cycle then does not return memory to the driver).
static sft_status init_device_pool() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  SFT_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  if (dev >= 0 && dev < 64 && !done[dev]) {
    cudaMemPool_t pool;
    SFT_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
    uint64_t thr = UINT64_MAX;
    SFT_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
    done[dev] = true;
  }
  return SFT_OK;
}

static sft_status check_desc(const sft_mesh_desc* d, bool source) {
  if (!d) return fail(SFT_ERR_ARG, "null mesh descriptor");
  if (d->dim != 2 && d->dim != 3) return fail(SFT_ERR_ARG, "dim must be 2 or 3");
  if (d->dtype != SFT_F32 && d->dtype != SFT_F64) return fail(SFT_ERR_ARG, "dtype must be SFT_F32 or SFT_F64");
  if (d->nnodes < d->dim + 1 || d->nelems < 1) return fail(SFT_ERR_ARG, "mesh needs >= dim+1 nodes and >= 1 element");
  if (d->nnodes >= INT32_MAX || d->nelems >= INT32_MAX / 4) return fail(SFT_ERR_UNSUPPORTED, "mesh too large for int32 indices");
  if (!d->coords || !d->conn) return fail(SFT_ERR_ARG, "null coords or conn");
  if (source) {
    if (d->nfields < 1 || d->nfields > kMaxFields) return fail(SFT_ERR_ARG, "nfields must be in 1..8");
    if (!d->values) return fail(SFT_ERR_ARG, "null source values");
  }
  // non-finite coordinates (host or device inputs) are found on the device
  // after the copy (check_finite), before the first kernel that reads them
  return SFT_OK;
}

static sft_status copy_in(void** dst, const void* src, size_t bytes, cudaStream_t st) {
  SFT_CUDA(pool_alloc(dst, bytes ? bytes : 1, st));
  if (bytes) SFT_CUDA(cudaMemcpyAsync(*dst, src, bytes, cudaMemcpyDefault, st));
  return SFT_OK;
}

static void free_locator(Locator& L, cudaStream_t st) {
  if (L.grid) cudaFreeAsync(L.grid, st);
  if (L.cell_start) cudaFreeAsync(L.cell_start, st);
  if (L.cell_items) cudaFreeAsync(L.cell_items, st);
  if (L.cell_first) cudaFreeAsync(L.cell_first, st);
  if (L.recs) cudaFreeAsync(L.recs, st);
  if (L.vals) cudaFreeAsync(L.vals, st);
  if (L.coordsP) cudaFreeAsync(L.coordsP, st);
  L = Locator();
}

}  // namespace sft

using namespace sft;

extern "C" {

const char* sft_status_str(sft_status s) {
  switch (s) {
    case SFT_OK: return "SFT_OK";
    case SFT_ERR_ARG: return "SFT_ERR_ARG";
    case SFT_ERR_MESH: return "SFT_ERR_MESH";
    case SFT_ERR_CUDA: return "SFT_ERR_CUDA";
    case SFT_ERR_OOM: return "SFT_ERR_OOM";
    case SFT_ERR_NOT_CONVERGED: return "SFT_ERR_NOT_CONVERGED";
    case SFT_ERR_OUTSIDE: return "SFT_ERR_OUTSIDE";
    case SFT_ERR_DEVICE_STATUS: return "SFT_ERR_DEVICE_STATUS";
    case SFT_ERR_UNSUPPORTED: return "SFT_ERR_UNSUPPORTED";
  }
  return "SFT_ERR_UNKNOWN";
}

const char* sft_last_error(void) { return g_last_error.c_str(); }

int64_t sft_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

sft_status sft_trim_memory(void) {
  trim_pools();
  return SFT_OK;
}

void sft_source_destroy(sft_source s) {
  if (!s) return;
  cudaStream_t st = s->stream;
  for (auto& L : s->loc) free_locator(L, st);
  if (s->coords) cudaFreeAsync(s->coords, st);
  if (s->conn) cudaFreeAsync(s->conn, st);
  if (s->values) cudaFreeAsync(s->values, st);
  if (s->evol) cudaFreeAsync(s->evol, st);
  if (s->adj) cudaFreeAsync(s->adj, st);
  delete s;
}

void sft_target_destroy(sft_target t) {
  if (!t) return;
  cudaStream_t st = t->stream;
  void* bufs[] = {t->coords, t->conn, t->coordsP[0], t->coordsP[1], t->vol, t->vol32, t->row_ptr, t->col, t->val, t->dinv, t->lumped, t->sc, t->val32s};
  for (void* p : bufs)
    if (p) cudaFreeAsync(p, st);
  delete t;
}

sft_status sft_source_create(const sft_mesh_desc* d, sft_source* out) {
  if (!out) return fail(SFT_ERR_ARG, "null output handle");
  *out = nullptr;
  if (sft_status r = check_desc(d, true)) return r;
  if (sft_status r = init_device_pool()) return r;
  cudaStream_t st = (cudaStream_t)d->cuda_stream;
  auto* s = new sft_source_s();
  s->dim = d->dim;
  s->nf = d->nfields;
  s->nv = d->nnodes;
  s->ne = d->nelems;
  s->dtype = d->dtype;
  s->L = d->grid_scale_L > 0 ? d->grid_scale_L : 1.0;
  s->stream = st;
  const size_t esz = d->dtype == SFT_F64 ? 8 : 4;
  sft_status r = SFT_OK;
  int32_t* d_err = nullptr;
  do {
    if ((r = copy_in(&s->coords, d->coords, esz * s->nv * s->dim, st))) break;
    if ((r = copy_in((void**)&s->conn, d->conn, sizeof(int32_t) * s->ne * (s->dim + 1), st))) break;
    if ((r = copy_in(&s->values, d->values, esz * s->nv * s->nf, st))) break;
    cudaError_t e = dalloc(&d_err, 1, st);
    if (e != cudaSuccess) { r = cuda_fail(e, "alloc"); break; }
    e = cudaMemsetAsync(d_err, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) { r = cuda_fail(e, "memset"); break; }
    e = check_finite(s->coords, s->nv * s->dim, d->dtype == SFT_F64, d_err, DEV_NONFINITE, st);
    if (e != cudaSuccess) { r = cuda_fail(e, "check_finite"); break; }
    const int prec = d->dtype == SFT_F64 ? SFT_PREC_FP64 : SFT_PREC_FP32;
    if ((r = build_locator(s, prec, st, d_err))) break;
  } while (0);
  if (d_err) cudaFreeAsync(d_err, st);
  if (r != SFT_OK) {
    sft_source_destroy(s);
    return r;
  }
  *out = s;
  return SFT_OK;
}

sft_status sft_source_set_values(sft_source s, const void* values, int32_t device_ptrs, void* cuda_stream) {
  if (!s || !values) return fail(SFT_ERR_ARG, "null argument");
  (void)device_ptrs;  // cudaMemcpyDefault resolves host or device memory
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const size_t esz = s->dtype == SFT_F64 ? 8 : 4;
  SFT_CUDA(cudaMemcpyAsync(s->values, values, esz * s->nv * s->nf, cudaMemcpyDefault, st));
  s->integral_valid = false;
  return refresh_value_copies(s, st);
}

sft_status sft_target_create(const sft_mesh_desc* d, sft_target* out) {
  if (!out) return fail(SFT_ERR_ARG, "null output handle");
  *out = nullptr;
  if (sft_status r = check_desc(d, false)) return r;
  if (sft_status r = init_device_pool()) return r;
  cudaStream_t st = (cudaStream_t)d->cuda_stream;
  auto* t = new sft_target_s();
  t->dim = d->dim;
  t->nv = d->nnodes;
  t->ne = d->nelems;
  t->dtype = d->dtype;
  t->stream = st;
  const size_t esz = d->dtype == SFT_F64 ? 8 : 4;
  sft_status r = SFT_OK;
  int32_t* d_err = nullptr;
  do {
    if ((r = copy_in(&t->coords, d->coords, esz * t->nv * t->dim, st))) break;
    if ((r = copy_in((void**)&t->conn, d->conn, sizeof(int32_t) * t->ne * (t->dim + 1), st))) break;
    cudaError_t e = dalloc(&d_err, 1, st);
    if (e != cudaSuccess) { r = cuda_fail(e, "alloc"); break; }
    e = cudaMemsetAsync(d_err, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) { r = cuda_fail(e, "memset"); break; }
    e = check_finite(t->coords, t->nv * t->dim, d->dtype == SFT_F64, d_err, DEV_NONFINITE, st);
    if (e != cudaSuccess) { r = cuda_fail(e, "check_finite"); break; }
    if ((r = build_target(t, st, d_err))) break;
    const int prec = d->dtype == SFT_F64 ? SFT_PREC_FP64 : SFT_PREC_FP32;
    if ((r = target_coordsP(t, prec, st))) break;
  } while (0);
  if (d_err) cudaFreeAsync(d_err, st);
  if (r != SFT_OK) {
    sft_target_destroy(t);
    return r;
  }
  *out = t;
  return SFT_OK;
}

sft_status sft_transfer(sft_source s, sft_target t, const sft_options* o, double* u_out, double* b_out,
                        double* g_out, sft_stats* stats) {
  if (!s || !t || !o || !u_out) return fail(SFT_ERR_ARG, "null argument");
  if (s->dim != t->dim) return fail(SFT_ERR_ARG, "source and target dimensions differ");
  if (o->samples_per_elem < 1) return fail(SFT_ERR_ARG, "samples_per_elem must be >= 1");
  if ((int64_t)o->samples_per_elem * t->ne >= ((int64_t)1 << 40)) return fail(SFT_ERR_UNSUPPORTED, "too many samples");
  if (o->precision != SFT_PREC_FP32 && o->precision != SFT_PREC_FP64) return fail(SFT_ERR_ARG, "bad precision");
  if (o->cg_max_iter < 0 || !(o->cg_tol >= 0) || !std::isfinite(o->alpha)) return fail(SFT_ERR_ARG, "bad solver options");
  if (o->cg_mode != SFT_CG_MIXED && o->cg_mode != SFT_CG_FP64) return fail(SFT_ERR_ARG, "unknown cg_mode");
  if (o->sampling != SFT_SAMPLING_UNIFORM && o->sampling != SFT_SAMPLING_STRATIFIED &&
      o->sampling != SFT_SAMPLING_IMPORTANCE)
    return fail(SFT_ERR_ARG, "unknown sampling scheme");
  if (o->cg_warm_start != 0 && o->cg_warm_start != 1) return fail(SFT_ERR_ARG, "cg_warm_start must be 0 or 1");
  if (o->cg_warm_start && o->cg_mode != SFT_CG_MIXED) return fail(SFT_ERR_UNSUPPORTED, "a warm start needs cg_mode MIXED");
  if (o->sampling == SFT_SAMPLING_STRATIFIED && o->samples_per_elem > kMaxStratifiedN)
    return fail(SFT_ERR_UNSUPPORTED, "stratified sampling supports at most 2^20 samples per element");
  if (!(o->adapt_ref_measure >= 0.0) || !std::isfinite(o->adapt_ref_measure))
    return fail(SFT_ERR_ARG, "adapt_ref_measure must be finite and >= 0");
  const bool adapt = o->adapt_ref_measure > 0.0;
  if (adapt && o->sampling == SFT_SAMPLING_STRATIFIED)
    return fail(SFT_ERR_UNSUPPORTED, "adaptive sample counts need uniform or importance sampling");
  if (adapt && (int64_t)o->samples_per_elem * 8 * t->ne >= ((int64_t)1 << 40))
    return fail(SFT_ERR_UNSUPPORTED, "too many samples");
  if (o->field_count < 0 || o->field_count > s->nf) return fail(SFT_ERR_ARG, "field_count out of range");
  const int64_t nmax = (int64_t)o->samples_per_elem * (adapt ? 8 : 1);   // sample_elem row length
  cudaStream_t st = (cudaStream_t)o->cuda_stream;
  const int prec = o->precision;
  const int nf = o->field_count > 0 ? o->field_count : s->nf;
  const int64_t nv = t->nv, ne = t->ne;
  const size_t psz = prec == SFT_PREC_FP32 ? 4 : 8;
  Events ev;
  if (ev.ok) cudaEventRecord(ev.e[0], st);
  DevBuf<int32_t> d_err(st);
  SFT_CUDA(d_err.alloc(1));
  SFT_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int32_t), st));
  if (sft_status r = build_locator(s, prec, st, d_err.p)) return r;
  if (sft_status r = target_coordsP(t, prec, st)) return r;
  if (ev.ok) cudaEventRecord(ev.e[1], st);

  DevBuf<char> g(st);
  DevBuf<double> b(st), u_tmp(st);
  DevBuf<int64_t> counters(st);
  DevBuf<int32_t> se_tmp(st);
  SFT_CUDA(g.alloc(psz * nv * nf));
  SFT_CUDA(b.alloc((size_t)nv * nf));
  SFT_CUDA(counters.alloc(3));
  SFT_CUDA(cudaMemsetAsync(b.p, 0, sizeof(double) * nv * nf, st));
  SFT_CUDA(cudaMemsetAsync(counters.p, 0, sizeof(int64_t) * 3, st));

  // step 1: control values g = f^s at the target nodes
  if (sft_status r = locate_points(s, prec, nv, t->coordsP[prec], prec == SFT_PREC_FP64, nullptr, g.p,
                                   prec == SFT_PREC_FP64, nv, counters.p, st, nf))
    return r;
  if (ev.ok) cudaEventRecord(ev.e[2], st);

  // steps 2-6: fused sampling / query / control / scatter
  int32_t* se = nullptr;
  if (o->sample_elem_out) {
    if (o->out_device) {
      se = o->sample_elem_out;
    } else {
      SFT_CUDA(se_tmp.alloc((size_t)(ne * nmax)));
      se = se_tmp.p;
    }
  }
  AssembleArgs a;
  a.prec = prec;
  a.nf = nf;
  a.N = o->samples_per_elem;
  a.seed = o->seed;
  a.stream_id = o->stream_id;
  a.alpha = o->alpha;
  a.g = g.p;
  a.b = b.p;
  a.sample_elem = se;
  a.counters = counters.p;
  a.sampling = o->sampling;
  a.adapt_ref = o->adapt_ref_measure;
  if (sft_status r = launch_assembly(s, t, a, st)) return r;
  if (ev.ok) cudaEventRecord(ev.e[3], st);

  // step 7: M u = b
  double* u_dev = u_out;
  if (!o->out_device) {
    SFT_CUDA(u_tmp.alloc((size_t)nv * nf));
    u_dev = u_tmp.p;
    if (o->cg_warm_start)
      SFT_CUDA(cudaMemcpyAsync(u_dev, u_out, sizeof(double) * nv * nf, cudaMemcpyHostToDevice, st));
  }
  SolveResult sr;
  SolveLate late(st);  // the solve's status is read with the final readback below
  if (sft_status r = mass_solve(t, nf, b.p, u_dev, o->cg_tol, o->cg_max_iter, st, d_err.p, &sr, o->cg_mode, &late,
                                o->cg_warm_start))
    return r;
  if (ev.ok) cudaEventRecord(ev.e[4], st);

  const cudaMemcpyKind d2o = o->out_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (!o->out_device) SFT_CUDA(cudaMemcpyAsync(u_out, u_dev, sizeof(double) * nv * nf, d2o, st));
  if (b_out) SFT_CUDA(cudaMemcpyAsync(b_out, b.p, sizeof(double) * nv * nf, d2o, st));
  if (g_out) {
    if (prec == SFT_PREC_FP64) {
      SFT_CUDA(cudaMemcpyAsync(g_out, g.p, sizeof(double) * nv * nf, d2o, st));
    } else {
      DevBuf<double> g64(st);
      SFT_CUDA(g64.alloc((size_t)nv * nf));
      if (sft_status r = convert_coords(g.p, SFT_F32, g64.p, SFT_PREC_FP64, nv * nf, st)) return r;
      SFT_CUDA(cudaMemcpyAsync(g_out, g64.p, sizeof(double) * nv * nf, d2o, st));
      SFT_CUDA(cudaStreamSynchronize(st));
    }
  }
  if (se && !o->out_device)
    SFT_CUDA(cudaMemcpyAsync(o->sample_elem_out, se, sizeof(int32_t) * ne * nmax, d2o, st));
  int64_t hc[3] = {0, 0, 0};
  int32_t herr = 0;
  SFT_CUDA(cudaMemcpyAsync(hc, counters.p, sizeof(hc), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaMemcpyAsync(&herr, d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (late.pending) SFT_CUDA(cudaMemcpyAsync(late.host, late.buf.p, late.bytes, cudaMemcpyDeviceToHost, st));
  if (ev.ok) cudaEventRecord(ev.e[5], st);
  SFT_CUDA(cudaStreamSynchronize(st));
  if (sft_status r = finish_solve(late, &sr)) return r;
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->cg_iters = sr.iters;
    stats->cg_rel_resid = sr.rel_resid;
    stats->queries = nv + (adapt || o->sampling == SFT_SAMPLING_IMPORTANCE ? hc[2]
                                                                            : ne * (int64_t)o->samples_per_elem);
    stats->fallback_queries = hc[0];
    stats->empty_queries = hc[1];
    stats->ms_setup = ev.ms(0, 1);
    stats->ms_control = ev.ms(1, 2);
    stats->ms_assembly = ev.ms(2, 3);
    stats->ms_solve = ev.ms(3, 4);
    stats->ms_total = ev.ms(0, 5);
  }
  if (herr) return fail(SFT_ERR_DEVICE_STATUS, "a transfer kernel reported an error");
  if (o->strict_inside && hc[1] > 0) return fail(SFT_ERR_OUTSIDE, "a query fell in an empty grid cell");
  if (!sr.converged && o->cg_max_iter > 0) return fail(SFT_ERR_NOT_CONVERGED, "CG reached cg_max_iter");
  return SFT_OK;
}

sft_status sft_conservation_error(sft_source s, sft_target t, const double* u, int32_t u_on_device, int32_t field,
                                  void* cuda_stream, double* out3) {
  if (!s || !t || !u || !out3) return fail(SFT_ERR_ARG, "null argument");
  if (field < 0 || field >= s->nf) return fail(SFT_ERR_ARG, "field out of range");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  const double* ud = u;
  DevBuf<double> tmp(st);
  if (!u_on_device) {
    SFT_CUDA(tmp.alloc((size_t)t->nv));
    SFT_CUDA(cudaMemcpyAsync(tmp.p, u, sizeof(double) * t->nv, cudaMemcpyHostToDevice, st));
    ud = tmp.p;
  }
  // both reductions read back together (one wait on the stream)
  const size_t ni = s->integral_valid ? 0 : (size_t)kIntegralBlocks * kMaxFields;
  DevBuf<double> part(st);
  SFT_CUDA(part.alloc(ni + kWsumBlocks));
  if (ni)
    if (sft_status r = source_integrals_launch(s, part.p, st)) return r;
  if (sft_status r = weighted_sum_launch(t->lumped, ud, t->nv, part.p + ni, st)) return r;
  std::vector<double> h(ni + kWsumBlocks);
  SFT_CUDA(cudaMemcpyAsync(h.data(), part.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  if (ni) source_integrals_finish(s, h.data());
  const double it = weighted_sum_finish(h.data() + ni);
  const double is = s->integral[field];
  out3[0] = std::fabs(is - it) / std::fabs(is);
  out3[1] = is;
  out3[2] = it;
  return SFT_OK;
}

sft_status sft_locate(sft_source s, int32_t precision, int64_t n, const double* pts, int32_t device_ptrs,
                      int32_t* elem_out, double* val_out, void* cuda_stream) {
  if (!s || (n > 0 && !pts)) return fail(SFT_ERR_ARG, "null argument");
  if (precision != SFT_PREC_FP32 && precision != SFT_PREC_FP64) return fail(SFT_ERR_ARG, "bad precision");
  if (n <= 0) return SFT_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf<int32_t> d_err(st);
  SFT_CUDA(d_err.alloc(1));
  SFT_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int32_t), st));
  if (sft_status r = build_locator(s, precision, st, d_err.p)) return r;
  DevBuf<double> p_tmp(st), v_tmp(st);
  DevBuf<int32_t> e_tmp(st);
  const double* pd = pts;
  int32_t* ed = elem_out;
  double* vd = val_out;
  if (!device_ptrs) {
    SFT_CUDA(p_tmp.alloc((size_t)n * s->dim));
    SFT_CUDA(cudaMemcpyAsync(p_tmp.p, pts, sizeof(double) * n * s->dim, cudaMemcpyHostToDevice, st));
    pd = p_tmp.p;
    if (elem_out) { SFT_CUDA(e_tmp.alloc((size_t)n)); ed = e_tmp.p; }
    if (val_out) { SFT_CUDA(v_tmp.alloc((size_t)n * s->nf)); vd = v_tmp.p; }
  }
  if (sft_status r = locate_points(s, precision, n, pd, 1, ed, vd, 1, n, nullptr, st)) return r;
  if (!device_ptrs) {
    if (elem_out) SFT_CUDA(cudaMemcpyAsync(elem_out, ed, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st));
    if (val_out) SFT_CUDA(cudaMemcpyAsync(val_out, vd, sizeof(double) * n * s->nf, cudaMemcpyDeviceToHost, st));
  }
  SFT_CUDA(cudaStreamSynchronize(st));
  return SFT_OK;
}

sft_status sft_mass_solve(sft_target t, int32_t nrhs, const double* b, double* u, int32_t device_ptrs, double tol,
                          int32_t max_iter, int32_t cg_mode, void* cuda_stream, int32_t* iters_out,
                          double* rel_resid_out) {
  if (!t || !b || !u) return fail(SFT_ERR_ARG, "null argument");
  if (cg_mode != SFT_CG_MIXED && cg_mode != SFT_CG_FP64) return fail(SFT_ERR_ARG, "unknown cg_mode");
  if (nrhs < 1 || nrhs > kMaxFields) return fail(SFT_ERR_ARG, "nrhs must be in 1..8");
  if (max_iter < 0 || !(tol >= 0)) return fail(SFT_ERR_ARG, "bad solver options");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf<double> bt(st), ut(st);
  const double* bd = b;
  double* ud = u;
  const size_t cnt = (size_t)t->nv * nrhs;
  if (!device_ptrs) {
    SFT_CUDA(bt.alloc(cnt));
    SFT_CUDA(ut.alloc(cnt));
    SFT_CUDA(cudaMemcpyAsync(bt.p, b, sizeof(double) * cnt, cudaMemcpyHostToDevice, st));
    bd = bt.p;
    ud = ut.p;
  }
  SolveResult sr;
  if (sft_status r = mass_solve(t, nrhs, bd, ud, tol, max_iter, st, nullptr, &sr, cg_mode)) return r;
  if (!device_ptrs) SFT_CUDA(cudaMemcpyAsync(u, ud, sizeof(double) * cnt, cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  if (iters_out) *iters_out = sr.iters;
  if (rel_resid_out) *rel_resid_out = sr.rel_resid;
  if (!sr.converged && max_iter > 0) return fail(SFT_ERR_NOT_CONVERGED, "CG reached max_iter");
  return SFT_OK;
}

sft_status sft_source_grid(sft_source s, int32_t precision, int32_t n_out[3], int64_t* ncells_out,
                           int64_t* nitems_out, int64_t* start_out, int32_t* items_out) {
  if (!s) return fail(SFT_ERR_ARG, "null source");
  if (precision != SFT_PREC_FP32 && precision != SFT_PREC_FP64) return fail(SFT_ERR_ARG, "bad precision");
  cudaStream_t st = s->stream;
  DevBuf<int32_t> d_err(st);
  SFT_CUDA(d_err.alloc(1));
  SFT_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int32_t), st));
  if (sft_status r = build_locator(s, precision, st, d_err.p)) return r;
  const Locator& L = s->loc[precision];
  if (n_out)
    for (int a = 0; a < 3; ++a) n_out[a] = L.n[a];
  if (ncells_out) *ncells_out = L.ncells;
  if (nitems_out) *nitems_out = L.nitems;
  if (start_out) {
    std::vector<int32_t> h((size_t)L.ncells + 1);
    SFT_CUDA(cudaMemcpyAsync(h.data(), L.cell_start, sizeof(int32_t) * h.size(), cudaMemcpyDeviceToHost, st));
    SFT_CUDA(cudaStreamSynchronize(st));
    for (size_t i = 0; i < h.size(); ++i) start_out[i] = h[i];
  }
  if (items_out) SFT_CUDA(cudaMemcpyAsync(items_out, L.cell_items, sizeof(int32_t) * L.nitems, cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  return SFT_OK;
}

sft_status sft_source_cell_first(sft_source s, int32_t precision, int32_t* first_out) {
  if (!s || !first_out) return fail(SFT_ERR_ARG, "null source or output");
  if (precision != SFT_PREC_FP32 && precision != SFT_PREC_FP64) return fail(SFT_ERR_ARG, "bad precision");
  cudaStream_t st = s->stream;
  DevBuf<int32_t> d_err(st);
  SFT_CUDA(d_err.alloc(1));
  SFT_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int32_t), st));
  if (sft_status r = build_locator(s, precision, st, d_err.p)) return r;
  const Locator& L = s->loc[precision];
  SFT_CUDA(cudaMemcpyAsync(first_out, L.cell_first, sizeof(int32_t) * (size_t)L.ncells, cudaMemcpyDefault, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  return SFT_OK;
}

sft_status sft_target_set_wait_limit(sft_target t, double seconds) {
  if (!t) return fail(SFT_ERR_ARG, "null target");
  if (!(seconds > 0.0) || !(seconds <= 3600.0)) return fail(SFT_ERR_ARG, "wait limit must be in (0, 3600] s");
  const double ns = seconds * 1e9;
  t->wait_ns = ns < 1.0 ? 1ull : (uint64_t)ns;
  return SFT_OK;
}

sft_status sft_source_adjacency(sft_source s, int32_t precision, int32_t* adj_out) {
  if (!s || !adj_out) return fail(SFT_ERR_ARG, "null source or output");
  if (precision != SFT_PREC_FP32 && precision != SFT_PREC_FP64) return fail(SFT_ERR_ARG, "bad precision");
  cudaStream_t st = s->stream;
  DevBuf<int32_t> d_err(st);
  SFT_CUDA(d_err.alloc(1));
  SFT_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int32_t), st));
  if (sft_status r = build_locator(s, precision, st, d_err.p)) return r;
  SFT_CUDA(cudaMemcpyAsync(adj_out, s->adj, sizeof(int32_t) * (size_t)s->ne * (s->dim + 1), cudaMemcpyDefault, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  return SFT_OK;
}

sft_status sft_target_mass(sft_target t, int64_t* nnz_out, int64_t* row_ptr_out, int32_t* col_out, double* val_out,
                           double* lumped_out) {
  if (!t) return fail(SFT_ERR_ARG, "null target");
  cudaStream_t st = t->stream;
  if (nnz_out) *nnz_out = t->nnz;
  if (row_ptr_out) {
    std::vector<int32_t> h((size_t)t->nv + 1);
    SFT_CUDA(cudaMemcpyAsync(h.data(), t->row_ptr, sizeof(int32_t) * h.size(), cudaMemcpyDeviceToHost, st));
    SFT_CUDA(cudaStreamSynchronize(st));
    for (size_t i = 0; i < h.size(); ++i) row_ptr_out[i] = h[i];
  }
  if (col_out) SFT_CUDA(cudaMemcpyAsync(col_out, t->col, sizeof(int32_t) * t->nnz, cudaMemcpyDeviceToHost, st));
  if (val_out) SFT_CUDA(cudaMemcpyAsync(val_out, t->val, sizeof(double) * t->nnz, cudaMemcpyDeviceToHost, st));
  if (lumped_out) SFT_CUDA(cudaMemcpyAsync(lumped_out, t->lumped, sizeof(double) * t->nv, cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  return SFT_OK;
}

}  // extern "C"
