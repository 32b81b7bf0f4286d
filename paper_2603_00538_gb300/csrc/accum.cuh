// Per-element partial sums of the Monte Carlo assembly and the per-element
// epilogue b_i += alpha int_t g psi_i + |T|/N sum_j r_j psi_i(X_j), shared by
// the mesh-source and the surrogate-source assembly kernels.
#pragma once
#include "common.cuh"

namespace sft {

template <typename P> struct Acc;
template <> struct Acc<float> {
  float s = 0.f, e = 0.f;
  __device__ __forceinline__ void add(float x) {
    float t, err;
    two_sum(s, x, t, err);
    s = t;
    e = __fadd_rn(e, err);
  }
  __device__ __forceinline__ void combine(float s2, float e2) {
    float t, err;
    two_sum(s, s2, t, err);
    s = t;
    e = __fadd_rn(__fadd_rn(e, e2), err);
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)e; }
};
template <> struct Acc<double> {
  double s = 0.0, e = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ void combine(double s2, double) { s += s2; }
  __device__ __forceinline__ double value() const { return s; }
};

// Per-element epilogue: b_i += |T| c_det (sum_m g_m + g_i) + |T|/N P_i.
// On this GPU the FP64 pipe retires one warp instruction per 16 cycles, and
// the epilogue runs on one lane per element, so the FP32 path keeps it in
// FP32 (error ~1e-7 relative, below the FP32 evaluation error of g) and only
// converts the final value for the FP64 atomic.
template <typename P> struct Epi;
template <> struct Epi<float> {
  static __device__ __forceinline__ double contrib(float volf, double, float cdet, float cmc, float gsum,
                                                   float gi, const Acc<float>& a) {
    const float mc = __fadd_rn(a.s, a.e);
    return (double)__fmaf_rn(__fmul_rn(volf, cdet), __fadd_rn(gsum, gi), __fmul_rn(__fmul_rn(volf, cmc), mc));
  }
};
template <> struct Epi<double> {
  static __device__ __forceinline__ double contrib(float, double vol, double cdet, double cmc, double gsum,
                                                   double gi, const Acc<double>& a) {
    return vol * cdet * (gsum + gi) + vol * cmc * a.value();
  }
};

}  // namespace sft
