// Internal declarations shared by the translation units of libsft.
#pragma once
#include <cstdint>
#include <string>
#include <cuda_runtime.h>
#include "sft.h"
#include "common.cuh"

namespace sft {

constexpr int kMaxFields = 8;

// thread-local error message + status helpers (api.cu)
void set_last_error(const std::string& msg);
sft_status fail(sft_status s, const std::string& msg);
sft_status cuda_fail(cudaError_t e, const char* what);

#define SFT_CUDA(call)                                                   \
  do {                                                                   \
    cudaError_t _e = (call);                                             \
    if (_e != cudaSuccess) return ::sft::cuda_fail(_e, #call);           \
  } while (0)

// Stream-ordered device allocation from the library's memory pool of the
// current device (util.cu). The pool keeps freed blocks for reuse instead of
// returning them to the driver at each synchronisation, so repeated creates,
// transfers and destroys do not map fresh memory every time;
// sft_trim_memory hands the unused part back.
cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s);
// *err <- code (first error wins) if any of the n values at x (device
// memory, FP64 or FP32) is not finite (util.cu)
cudaError_t check_finite(const void* x, int64_t n, bool is_double, int32_t* err, int32_t code, cudaStream_t s);
void trim_pools();
template <typename T>
cudaError_t dalloc(T** p, size_t count, cudaStream_t s) {
  *p = nullptr;
  if (count == 0) count = 1;
  return pool_alloc(reinterpret_cast<void**>(p), sizeof(T) * count, s);
}
template <typename T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

// RAII device scratch on a stream
template <typename T>
struct DevBuf {
  T* p = nullptr;
  cudaStream_t s = nullptr;
  explicit DevBuf(cudaStream_t st) : s(st) {}
  cudaError_t alloc(size_t n) { return dalloc(&p, n, s); }
  ~DevBuf() { dfree(p, s); }
};

struct Events {
  cudaEvent_t e[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  bool ok = false;
  Events() {
    ok = true;
    for (auto& x : e) ok = ok && cudaEventCreate(&x) == cudaSuccess;
  }
  ~Events() {
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
  float ms(int a, int b) const {
    float t = 0.f;
    if (ok && cudaEventElapsedTime(&t, e[a], e[b]) != cudaSuccess) {
      t = -1.f;
      cudaGetLastError();  // timing unavailable: do not leave a sticky error behind
    }
    return t;
  }
};

// location structure of a source mesh in one precision
struct Locator {
  bool built = false;
  int32_t n[3] = {1, 1, 1};
  int64_t ncells = 0, nitems = 0;
  void* grid = nullptr;          // device GridP<P>
  int32_t* cell_start = nullptr;  // [ncells + 1]
  int32_t* cell_items = nullptr;  // [nitems] (in no particular order within a cell)
  int32_t* cell_first = nullptr;  // [ncells] start element of the location walk, -1: empty cell
  void* recs = nullptr;           // [ne][RecLen] P
  void* vals = nullptr;           // [ne][nf][4] P
  void* coordsP = nullptr;        // [nv][dim] P
  const int32_t* adj = nullptr;   // the source's face neighbours (sft_source_s::adj)
};

}  // namespace sft

struct sft_source_s {
  int dim = 2, nf = 1;
  int64_t nv = 0, ne = 0;
  int dtype = SFT_F64;
  double L = 1.0;
  cudaStream_t stream = nullptr;
  void* coords = nullptr;       // [nv][dim] input dtype
  int32_t* conn = nullptr;      // [ne][dim+1]
  void* values = nullptr;       // [nf][nv] input dtype
  double* evol = nullptr;       // [ne] FP64 element measures (made with the first locator)
  int32_t* adj = nullptr;       // [ne][dim+1] neighbour across the face opposite vertex m, -1 on
                                // the boundary (made with the first locator)
  double integral[sft::kMaxFields] = {0};
  bool integral_valid = false;  // integral[] matches the current values (made on first use)
  sft::Locator loc[2];          // index = sft_precision (0 FP64, 1 FP32)
};

struct sft_target_s {
  int dim = 2;
  int64_t nv = 0, ne = 0;
  int dtype = SFT_F64;
  cudaStream_t stream = nullptr;
  void* coords = nullptr;       // [nv][dim] input dtype
  int32_t* conn = nullptr;      // [ne][dim+1]
  void* coordsP[2] = {nullptr, nullptr};  // per precision copy (lazy)
  double* vol = nullptr;        // [ne] FP64 measures
  float* vol32 = nullptr;       // [ne] FP32 copy (the FP32 assembly epilogue)
  // mass matrix, CSR FP64
  int64_t nnz = 0;
  int32_t* row_ptr = nullptr;   // [nv+1]
  int32_t* col = nullptr;       // [nnz]
  double* val = nullptr;        // [nnz]
  double* dinv = nullptr;       // [nv]
  double* lumped = nullptr;     // [nv]
  // symmetric Jacobi scaling for the mixed-precision solve (made on first use):
  // sc = diag(M)^-1/2 and the FP32 values of sc_i M_ij sc_j
  double* sc = nullptr;         // [nv]
  float* val32s = nullptr;      // [nnz]
  // limit of the solves' device waits (grid barriers), nanoseconds
  uint64_t wait_ns = 2000000000ull;
};

namespace sft {
// locate.cu
sft_status build_locator(sft_source_s* s, int prec, cudaStream_t st, int32_t* d_err);
sft_status locate_points(sft_source_s* s, int prec, int64_t n, const void* pts, int pts_are_double,
                         int32_t* elem_out, void* val_out, int val_is_double, int64_t val_stride,
                         int64_t* d_counters, cudaStream_t st, int nf_out = -1, void* mu_out = nullptr);
sft_status source_integrals(sft_source_s* s, cudaStream_t st);
// the same split in launch (partials [kIntegralBlocks][kMaxFields] on the
// device) and the host's fixed-order sum of the copied partials
constexpr unsigned kIntegralBlocks = 152 * 8;
sft_status source_integrals_launch(sft_source_s* s, double* part, cudaStream_t st);
void source_integrals_finish(sft_source_s* s, const double* hpart);
sft_status refresh_value_copies(sft_source_s* s, cudaStream_t st);
// target.cu
sft_status build_target(sft_target_s* t, cudaStream_t st, int32_t* d_err);
sft_status target_coordsP(sft_target_s* t, int prec, cudaStream_t st);
// intersect.cu: exact load vector (u == nullptr) or L2 error of u (2D)
sft_status mesh_intersection_2d(sft_source_s* s, sft_target_s* t, int field, const double* u, double* b,
                                double* err_out, double* norm_out, cudaStream_t st);
// assemble.cu
enum AsmMode : int { kAsmPlain = 0, kAsmDebug = 1, kAsmRecord = 2, kAsmCached = 3 };
struct AssembleArgs {
  int prec;
  int nf;
  int N;
  uint64_t seed;
  uint32_t stream_id;
  double alpha;
  const void* g;          // [nf][nv_t] P
  double* b;              // [nf][nv_t] FP64 (accumulated)
  int32_t* sample_elem;   // optional [ne_t][N] (debug, record: written; cached: read)
  int64_t* counters;      // [2]: fallback, empty
  int mode = kAsmPlain;
  void* pmu = nullptr;    // record / cached: [d][ne_t N] P, mu_1..d of every sample
  int sampling = SFT_SAMPLING_UNIFORM;  // sft_sampling
  double adapt_ref = 0.0;  // > 0: per-element sample counts against this reference measure
};
sft_status launch_assembly(sft_source_s* s, sft_target_s* t, const AssembleArgs& a, cudaStream_t st);
// solve.cu
struct SolveResult { int iters; double rel_resid; int converged; };
// Deferred solve status: with a SolveLate, mass_solve returns without waiting
// for the kernel (mixed mode); the caller copies `bytes` from buf to host in
// its own final readback and then calls finish_solve.
struct SolveLate {
  explicit SolveLate(cudaStream_t st) : buf(st) {}
  DevBuf<unsigned char> buf;
  alignas(16) unsigned char host[256];
  size_t bytes = 0;
  int nrhs = 0;
  bool pending = false;
};
sft_status finish_solve(const SolveLate& late, SolveResult* res);
// cg_mode: SFT_CG_MIXED (FP64 refinement around FP32 CG) or SFT_CG_FP64
sft_status mass_solve(sft_target_s* t, int nrhs, const double* b, double* x, double tol, int max_iter,
                      cudaStream_t st, int32_t* d_err, SolveResult* res, int cg_mode = SFT_CG_MIXED,
                      SolveLate* late = nullptr, int warm = 0);
// S = diag(M)^-1/2 and the FP32 values of S M S on the target (made once, cached)
sft_status scaled_matrix(sft_target_s* t, cudaStream_t st);
sft_status weighted_sum(const double* w, const double* u, int64_t n, double* out_host, cudaStream_t st);
constexpr unsigned kWsumBlocks = 304;
sft_status weighted_sum_launch(const double* w, const double* u, int64_t n, double* part, cudaStream_t st);
double weighted_sum_finish(const double* hpart);
// conversions
sft_status convert_coords(const void* in, int in_dtype, void* out, int out_prec, int64_t n, cudaStream_t st);
}  // namespace sft
