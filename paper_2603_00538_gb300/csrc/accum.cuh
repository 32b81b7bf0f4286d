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

// The K component adds of one sample, x_i = r lam_i. The TwoSum steps of FP32
// components go in pairs through the packed two-lane instructions, in the
// same order, so the sums agree with add() bit for bit. The products stay
// scalar: a packed product feeding a packed add was contracted into a fused
// multiply-add (measured: 2.6 % of 1 M random pairs differed from the
// separately rounded scalar forms), which would break TwoSum's exactness.
template <int K>
__device__ __forceinline__ void acc_add_sample(Acc<float> (&a)[K], float r, const float (&lam)[K]) {
#pragma unroll
  for (int i = 0; i + 1 < K; i += 2) {
    const uint64_t x = f2_pack(__fmul_rn(r, lam[i]), __fmul_rn(r, lam[i + 1]));
    uint64_t t, err;
    two_sum2(f2_pack(a[i].s, a[i + 1].s), x, t, err);
    f2_unpack(t, a[i].s, a[i + 1].s);
    f2_unpack(f2_add(f2_pack(a[i].e, a[i + 1].e), err), a[i].e, a[i + 1].e);
  }
  if constexpr ((K & 1) != 0) a[K - 1].add(__fmul_rn(r, lam[K - 1]));
}
template <int K>
__device__ __forceinline__ void acc_add_sample(Acc<double> (&a)[K], double r, const double (&lam)[K]) {
#pragma unroll
  for (int i = 0; i < K; ++i) a[i].add(__dmul_rn(r, lam[i]));
}

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
