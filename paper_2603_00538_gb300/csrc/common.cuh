// Device primitives of the transfer path: counter-based random numbers, the
// element sample map (Sec. 4, step 3), the uniform-grid cell index and the
// point-location predicate (Sec. 5.3 grid search), P1 evaluation.
//
// The arithmetic that decides an integer (a located element) is written with
// explicit round-to-nearest intrinsics (__fmul_rn, __fmaf_rn, ...) so no
// compiler contraction changes it: the same operation sequence evaluated in
// IEEE arithmetic gives the same element on any conforming implementation.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace sft {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy
// as 1, 2, 3", SC'11): 10 rounds of two 32x32->64 multiplies; the key advances
// by the Weyl constants between rounds.
// ---------------------------------------------------------------------------
struct PhiloxKey { uint32_t k0, k1; };

// One round: the two 32x32 -> 64-bit products (one wide multiply each gives
// both halves), their high halves mixed with the other two words and the
// round key.
__device__ __forceinline__ uint4 philox_round(uint4 c, uint32_t k0, uint32_t k1) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
  return make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, PhiloxKey k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    c = philox_round(c, k.k0, k.k1);
    k.k0 += 0x9E3779B9u;
    k.k1 += 0xBB67AE85u;
  }
  return c;
}

// The ten round keys of one key (key + r (0x9E3779B9, 0xBB67AE85) mod 2^32),
// formed once on the host: passed in a kernel's parameters they are operands
// of the round's XOR, so the hot loop spends no instruction on the schedule.
struct PhiloxRoundKeys { uint32_t k0[10], k1[10]; };

inline PhiloxRoundKeys philox_round_keys(uint64_t seed) {
  PhiloxRoundKeys rk;
  uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k0[r] = a;
    rk.k1[r] = b;
    a += 0x9E3779B9u;
    b += 0xBB67AE85u;
  }
  return rk;
}

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, const PhiloxRoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) c = philox_round(c, rk.k0[r], rk.k1[r]);
  return c;
}

// Uniform(0,1) from one 32-bit word, exact in the target precision:
// FP32 odd multiples of 2^-24, u = ((x >> 8) | 1) 2^-24; FP64 (x + 1/2) 2^-32.
// Formed from the bit pattern (1 + m 2^-23 has mantissa m) and one exact
// addition, so no int->float conversion instruction is issued: on this GPU
// conversions share the narrow FP64 pipe. Value-identical to the definition
// above: (1 + k 2^-23) + (2^-24 - 1) = (2k + 1) 2^-24 has 24 significant bits,
// so the sum is exact, and (x >> 8) | 1 = 2 (x >> 9) + 1.
__device__ __forceinline__ float u01f(uint32_t x) {
  const float one_m = __uint_as_float(0x3F800000u | (x >> 9));  // 1 + (x>>9) 2^-23
  return __fadd_rn(one_m, -0x1.fffffep-1f);                      // (2 (x>>9) + 1) 2^-24
}
// float -> double without a conversion instruction (exact): a normal float's
// sign, rebiased exponent and mantissa placed in the double's fields; zero,
// subnormal, infinite and NaN inputs take the conversion instruction
__device__ __forceinline__ double f2d(float x) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t e = (b >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) return (double)x;
  const uint64_t bits = ((uint64_t)(b >> 31) << 63) | ((uint64_t)(e + 896u) << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)bits);
}
__device__ __forceinline__ double f2d(double x) { return x; }

__device__ __forceinline__ double u01d(uint32_t x) {
  const double one_m = __longlong_as_double((long long)(0x3FF0000000000000ull | ((uint64_t)x << 20)));
  return __dadd_rn(one_m, -0x1.ffffffffp-1);                     // (2x + 1) 2^-33, exact
}

// ---------------------------------------------------------------------------
// rounding-explicit arithmetic in precision P
// ---------------------------------------------------------------------------
template <typename P> struct Ar;
template <> struct Ar<float> {
  static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
  static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
  static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
  static __device__ __forceinline__ float fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
  static __device__ __forceinline__ float sqrt(float a) { return __fsqrt_rn(a); }
  static __device__ __forceinline__ float u01(uint32_t x) { return u01f(x); }
  static __device__ __forceinline__ float from_d(double x) { return __double2float_rn(x); }
  static __device__ __forceinline__ float floor(float x) { return floorf(x); }
  static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
};
template <> struct Ar<double> {
  static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
  static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
  static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
  static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
  static __device__ __forceinline__ double sqrt(double a) { return __dsqrt_rn(a); }
  static __device__ __forceinline__ double u01(uint32_t x) { return u01d(x); }
  static __device__ __forceinline__ double from_d(double x) { return x; }
  static __device__ __forceinline__ double floor(double x) { return ::floor(x); }
  static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
};

// ---------------------------------------------------------------------------
// Sample map (Sec. 4 step 3). 2D: Osada et al. (2002),
// (xi, eta) -> (1 - sqrt(xi), sqrt(xi)(1 - eta), sqrt(xi) eta).
// 3D: spacings of three sorted uniforms (uniform on the simplex).
// Counter layout: 2D one Philox call per sample pair q = j/2, counter
// (q, t, stream, 0), sample j uses words 2(j%2), 2(j%2)+1; 3D one call per
// sample, counter (j, t, stream, 0), words 0..2.
// ---------------------------------------------------------------------------
// Sampling scheme. Uniform: the maps above. Stratified (the general density
// p_t of Eq. mc_element_integral_operator_general with equal-measure strata):
// with m the largest integer such that m^D <= N, sample j < m^D replaces
// each uniform U_a by (c_a + U_a) / m, c_a the base-m digit a of j (least
// significant first), one rounding per operation; both maps carry the
// uniform measure of the unit square / cube to that of the simplex, so the
// m^D cells become equal-measure strata and the weights |T| / N stay
// unbiased. Samples j >= m^D keep their uniforms. n = 0 selects uniform.
struct Strat {
  int m;           // strata per axis
  int n;           // m^D (0: uniform sampling)
  uint32_t magic;  // ceil(2^32 / m): j / m = umulhi(j, magic) exactly while j m < 2^32
  float mf;        // m in FP32 and FP64
  double md;
};

// largest N for which the stratified digits are exact (j m <= N^(1+1/d) < 2^32)
constexpr int kMaxStratifiedN = 1 << 20;

// strata for N samples per element in dimension d (sampling 1 = stratified)
inline Strat strat_for(int d, int N, int sampling) {
  Strat st{0, 0, 0u, 1.f, 1.0};
  if (sampling != 1) return st;
  int m = 1;
  for (;;) {
    int64_t q = 1;
    for (int a = 0; a < d; ++a) q *= (int64_t)(m + 1);
    if (q > N) break;
    ++m;
  }
  st.m = m;
  st.n = m > 1 ? (d == 2 ? m * m : m * m * m) : 0;
  st.magic = m > 1 ? (uint32_t)((((uint64_t)1 << 32) + (uint64_t)m - 1) / (uint64_t)m) : 0u;
  st.mf = (float)m;
  st.md = (double)m;
  return st;
}

// small non-negative integer c (< 2^23) as P, from its bit pattern (no
// conversion instruction: conversions use the narrow FP64 pipe here)
__device__ __forceinline__ float small_int_f(uint32_t c) {
  return __fsub_rn(__uint_as_float(0x4B000000u | c), 8388608.0f);
}
__device__ __forceinline__ double small_int_d(uint32_t c) {
  return __dsub_rn(__longlong_as_double((long long)(0x4330000000000000ull | c)), 4503599627370496.0);
}

template <typename P>
__device__ __forceinline__ P strat_u(P u, uint32_t c, const Strat& st) {
  using A = Ar<P>;
  if constexpr (sizeof(P) == 4) return A::div(A::add(small_int_f(c), u), st.mf);
  else return A::div(A::add(small_int_d(c), u), st.md);
}

// barycentric weights of sample j from its Philox block w (2D: words
// 2(j%2), 2(j%2)+1; 3D: words 0..2)
template <int D, typename P>
__device__ __forceinline__ void sample_lambda(const uint4& w, int j, const Strat& st, P lam[D + 1]) {
  using A = Ar<P>;
  if constexpr (D == 2) {
    P xi = A::u01((j & 1) ? w.z : w.x), eta = A::u01((j & 1) ? w.w : w.y);
    if (j < st.n) {
      const uint32_t c1 = __umulhi((uint32_t)j, st.magic), c0 = (uint32_t)j - c1 * (uint32_t)st.m;
      xi = strat_u<P>(xi, c0, st);
      eta = strat_u<P>(eta, c1, st);
    }
    const P s = A::sqrt(xi);
    lam[0] = A::sub(P(1), s);
    lam[1] = A::mul(s, A::sub(P(1), eta));
    lam[2] = A::mul(s, eta);
  } else {
    P v0 = A::u01(w.x), v1 = A::u01(w.y), v2 = A::u01(w.z), s;
    if (j < st.n) {
      const uint32_t m = (uint32_t)st.m;
      const uint32_t q = __umulhi((uint32_t)j, st.magic), c0 = (uint32_t)j - q * m;
      const uint32_t c2 = __umulhi(q, st.magic), c1 = q - c2 * m;
      v0 = strat_u<P>(v0, c0, st);
      v1 = strat_u<P>(v1, c1, st);
      v2 = strat_u<P>(v2, c2, st);
    }
    if (v1 < v0) { s = v0; v0 = v1; v1 = s; }
    if (v2 < v1) { s = v1; v1 = v2; v2 = s; }
    if (v1 < v0) { s = v0; v0 = v1; v1 = s; }
    lam[0] = v0;
    lam[1] = A::sub(v1, v0);
    lam[2] = A::sub(v2, v1);
    lam[3] = A::sub(P(1), v2);
  }
}

// ---------------------------------------------------------------------------
// Importance sampling (Eq. mc_element_integral_operator_general with a
// non-uniform p_t): a mixture of the uniform density and the edge-bubble
// densities (d+1)(d+2) lambda_a lambda_b / |T| (Dirichlet with 2 at the
// edge's vertices a, b and 1 elsewhere), which follow the P1 interpolation
// error that the control-variate residual is at alpha = 1. Component
// probabilities: 2D uniform 1/4, each of the 3 edges 1/4; 3D uniform 1/4,
// each of the 6 edges 1/8; so |T| p_t = 1/4 + 3 sum_{a<b} lambda_a lambda_b
// (2D) or 1/4 + 5/2 sum (3D), and the sample weight w = 1 / (|T| p_t) <= 4.
// Sample j: Philox blocks (j, t, stream, 6) = a and (j, t, stream, 7) = b.
// The top bits of a.x pick the component (2D: a.x >> 30, 0 uniform, 1..3 the
// edges (0,1), (0,2), (1,2); 3D: a.x >> 29, 0..1 uniform, 2..7 the edges
// (0,1), (0,2), (0,3), (1,2), (1,3), (2,3)). Uniform: the Osada map of
// a.y, a.z (2D) or the sorted spacings of a.y, a.z, a.w (3D). Edge (ea, eb):
// the d + 2 uniforms a.y, a.z, a.w, b.x (, b.y) sorted, spacings s_0..s_{d+2}
// (s_0 = v_0, s_i = v_i - v_{i-1}, s_{d+2} = 1 - v_{d+1}); lambda_ea =
// s_0 + s_1, lambda_eb = s_2 + s_3, the other vertices in increasing order
// s_4 (, s_5). One rounding per operation in P.
// ---------------------------------------------------------------------------
template <typename P>
__device__ __forceinline__ void cswap(P& x, P& y) {
  const P lo = y < x ? y : x, hi = y < x ? x : y;
  x = lo;
  y = hi;
}

template <int D, typename P>
__device__ __forceinline__ P importance_lambda(const uint4& a, const uint4& b, P lam[D + 1]) {
  using A = Ar<P>;
  const uint32_t c = D == 2 ? (a.x >> 30) : (a.x >> 29);
  if (D == 2 ? c == 0u : c < 2u) {
    if constexpr (D == 2) {
      const P s = A::sqrt(A::u01(a.y)), eta = A::u01(a.z);
      lam[0] = A::sub(P(1), s);
      lam[1] = A::mul(s, A::sub(P(1), eta));
      lam[2] = A::mul(s, eta);
    } else {
      P v0 = A::u01(a.y), v1 = A::u01(a.z), v2 = A::u01(a.w);
      cswap(v0, v1); cswap(v1, v2); cswap(v0, v1);
      lam[0] = v0;
      lam[1] = A::sub(v1, v0);
      lam[2] = A::sub(v2, v1);
      lam[3] = A::sub(P(1), v2);
    }
  } else {
    P v[D + 2];
    v[0] = A::u01(a.y); v[1] = A::u01(a.z); v[2] = A::u01(a.w); v[3] = A::u01(b.x);
    if constexpr (D == 2) {
      cswap(v[0], v[1]); cswap(v[2], v[3]); cswap(v[0], v[2]); cswap(v[1], v[3]); cswap(v[1], v[2]);
    } else {
      v[4] = A::u01(b.y);
      cswap(v[0], v[1]); cswap(v[3], v[4]); cswap(v[2], v[4]); cswap(v[2], v[3]); cswap(v[0], v[3]);
      cswap(v[0], v[2]); cswap(v[1], v[4]); cswap(v[1], v[3]); cswap(v[1], v[2]);
    }
    P sp[D + 3];
    sp[0] = v[0];
#pragma unroll
    for (int i = 1; i < D + 2; ++i) sp[i] = A::sub(v[i], v[i - 1]);
    sp[D + 2] = A::sub(P(1), v[D + 1]);
    const P la = A::add(sp[0], sp[1]), lb = A::add(sp[2], sp[3]);
    // the edge's vertices (ea < eb) and the others in increasing order
    int ea, eb;
    if constexpr (D == 2) {
      ea = c == 3u ? 1 : 0;
      eb = c == 1u ? 1 : 2;
    } else {
      const int e = (int)c - 2;   // (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
      ea = e < 3 ? 0 : (e < 5 ? 1 : 2);
      eb = e < 3 ? e + 1 : (e < 5 ? e - 1 : 3);
    }
    // the vertices off the edge, in increasing order: o1 (and o2 in 3D)
    const int o1 = ea > 0 ? 0 : (eb > 1 ? 1 : 2);
    const int o2 = D == 2 ? o1 : 6 - ea - eb - o1;
#pragma unroll
    for (int m = 0; m <= D; ++m) {
      P x = sp[4];
      if constexpr (D == 3) x = m == o2 ? sp[5] : x;
      x = m == o1 ? sp[4] : x;
      x = m == eb ? lb : x;
      lam[m] = m == ea ? la : x;
    }
  }
  P bub = P(0);
#pragma unroll
  for (int x = 0; x <= D; ++x)
#pragma unroll
    for (int y = x + 1; y <= D; ++y) bub = A::add(bub, A::mul(lam[x], lam[y]));
  const P tp = A::add(P(0.25), A::mul(D == 2 ? P(3) : P(2.5), bub));
  return A::div(P(1), tp);
}

// X = sum_m lam_m x_m, accumulated left to right, one rounding per operation
template <int D, typename P>
__device__ __forceinline__ void map_point(const P lam[D + 1], const P xv[D + 1][D], P X[D]) {
  using A = Ar<P>;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    P x = A::mul(lam[0], xv[0][a]);
#pragma unroll
    for (int m = 1; m <= D; ++m) x = A::add(x, A::mul(lam[m], xv[m][a]));
    X[a] = x;
  }
}

// ---------------------------------------------------------------------------
// Uniform grid (Sec. 5.3): per axis origin lo, scale inv = n / extent (rounded
// to P once), n cells. cell(x) = clamp(floor((x - lo) * inv), 0, n - 1) is
// monotone in x.
// ---------------------------------------------------------------------------
template <typename P> struct GridP {
  P lo[3];
  P inv[3];
  P h[3];      // cell size (extent / n, rounded to P): cell centres lo + (i + 1/2) h
  int32_t n[3];
};

// cell_axis(x) = clamp(floor((x - lo) * inv), 0, n - 1). The floor is taken
// without a conversion instruction: for 0 <= s <= 2^22 (2^51 in FP64),
// s + 2^23 (2^52) rounded toward zero is 2^23 + floor(s), whose bit pattern
// minus that of 2^23 is floor(s). NaN and negative s clamp to 0 (fmax
// returns the non-NaN operand), large s to n - 1 (n < 2^22 is checked on
// the host). Same result as floor + clamp.
template <typename P>
__device__ __forceinline__ int32_t cell_axis(P x, P lo, P inv, int32_t n);

template <>
__device__ __forceinline__ int32_t cell_axis<float>(float x, float lo, float inv, int32_t n) {
  float s = __fmul_rn(__fsub_rn(x, lo), inv);
  s = fminf(fmaxf(s, 0.0f), 4194304.0f);
  const float t = __fadd_rz(s, 8388608.0f);
  const int32_t c = (int32_t)(__float_as_uint(t) - 0x4B000000u);
  return c < n - 1 ? c : n - 1;
}

template <>
__device__ __forceinline__ int32_t cell_axis<double>(double x, double lo, double inv, int32_t n) {
  double s = __dmul_rn(__dsub_rn(x, lo), inv);
  s = fmin(fmax(s, 0.0), 2251799813685248.0);
  const double t = __dadd_rz(s, 4503599627370496.0);
  const int64_t c = (int64_t)((uint64_t)__double_as_longlong(t) - 0x4330000000000000ull);
  return c < (int64_t)(n - 1) ? (int32_t)c : n - 1;
}

template <int D, typename P>
__device__ __forceinline__ int32_t cell_of(const GridP<P>& g, const P X[D]) {
  int32_t c = cell_axis<P>(X[D - 1], g.lo[D - 1], g.inv[D - 1], g.n[D - 1]);
#pragma unroll
  for (int a = D - 2; a >= 0; --a) c = c * g.n[a] + cell_axis<P>(X[a], g.lo[a], g.inv[a], g.n[a]);
  return c;
}

// ---------------------------------------------------------------------------
// Location record of a source element in precision P: the first vertex a and
// the rows of the inverse affine map (formed in FP64, rounded to P once).
// 2D: {ax, ay, i00, i01, i10, i11, 0, 0}; 3D: {ax, ay, az, r00..r22}.
// mu_1.. = J^-1 (X - a), mu_0 = 1 - sum; accept when min(mu) >= 0.
// ---------------------------------------------------------------------------
template <int D> struct RecLen { static constexpr int value = D == 2 ? 8 : 12; };

template <int D, typename P>
__device__ __forceinline__ void bary_from_record(const P* __restrict__ rec, const P X[D], P mu[D + 1]) {
  using A = Ar<P>;
  if constexpr (D == 2) {
    const P dx = A::sub(X[0], rec[0]), dy = A::sub(X[1], rec[1]);
    const P m1 = A::fma(rec[3], dy, A::mul(rec[2], dx));
    const P m2 = A::fma(rec[5], dy, A::mul(rec[4], dx));
    mu[0] = A::sub(A::sub(P(1), m1), m2);
    mu[1] = m1;
    mu[2] = m2;
  } else {
    const P dx = A::sub(X[0], rec[0]), dy = A::sub(X[1], rec[1]), dz = A::sub(X[2], rec[2]);
    P m[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
      m[q] = A::fma(rec[3 + 3 * q + 2], dz, A::fma(rec[3 + 3 * q + 1], dy, A::mul(rec[3 + 3 * q], dx)));
    mu[0] = A::sub(A::sub(A::sub(P(1), m[0]), m[1]), m[2]);
    mu[1] = m[0];
    mu[2] = m[1];
    mu[3] = m[2];
  }
}

// vectorised record load (records are 16-byte aligned)
template <int D, typename P>
__device__ __forceinline__ void load_record(const P* __restrict__ recs, int32_t e, P r[RecLen<D>::value]) {
  constexpr int L = RecLen<D>::value;
  if constexpr (sizeof(P) == 4) {
    const float4* p = reinterpret_cast<const float4*>(recs + (int64_t)e * L);
#pragma unroll
    for (int q = 0; q < L / 4; ++q) {
      const float4 v = __ldg(p + q);
      r[4 * q] = v.x; r[4 * q + 1] = v.y; r[4 * q + 2] = v.z; r[4 * q + 3] = v.w;
    }
  } else {
    const double2* p = reinterpret_cast<const double2*>(recs + (int64_t)e * L);
#pragma unroll
    for (int q = 0; q < L / 2; ++q) {
      const double2 v = __ldg(p + q);
      r[2 * q] = v.x; r[2 * q + 1] = v.y;
    }
  }
}

// predicate evaluations of the walk before the cell's list is scanned
constexpr int kWalkSteps = 12;

// The fallback of the location below: every candidate of cell c is tested
// at X = (x0, x1, x2) and the one with the largest min(mu) wins, ties to the
// lowest id (an accepting one whenever any accepts, else the nearest); -1 for
// an empty list. In 3D it runs out of line (scan_cell, fed by value): the
// walk almost always succeeds, and the inlined loop raised the register
// pressure of the 3D assembly kernel (tet5m launch 2.110 ms inlined, 1.858
// out of line); in 2D the inlined form is faster (tri4m 1.276 against 1.327).
template <typename P>
struct ScanHit {
  int32_t e;
  int status;
  P mu[4];
};

template <int D, typename P>
__device__ __forceinline__ ScanHit<P> scan_cell_body(int32_t c, P x0, P x1, P x2,
                                                     const int32_t* __restrict__ cell_start,
                                                     const int32_t* __restrict__ cell_items,
                                                     const P* __restrict__ recs) {
  constexpr int L = RecLen<D>::value;
  const P X[3] = {x0, x1, x2};
  const int32_t p0 = __ldg(cell_start + c), p1 = __ldg(cell_start + c + 1);
  int32_t best = -1;
  P best_score = P(0);
  for (int32_t p = p0; p < p1; ++p) {
    const int32_t e = __ldg(cell_items + p);
    P r[L];
    load_record<D, P>(recs, e, r);
    P m[D + 1];
    bary_from_record<D, P>(r, X, m);
    P mn = m[0];
#pragma unroll
    for (int q = 1; q <= D; ++q) mn = m[q] < mn ? m[q] : mn;
    if (best < 0 || mn > best_score || (mn == best_score && e < best)) { best = e; best_score = mn; }
  }
  ScanHit<P> h;
  h.e = best;
#pragma unroll
  for (int q = 0; q < 4; ++q) h.mu[q] = P(0);
  if (best < 0) {  // an empty list (cell_first is -1 there; kept safe)
    h.status = 2;
    return h;
  }
  h.status = best_score >= P(0) ? 0 : 1;
  P r[L];
  load_record<D, P>(recs, best, r);
  bary_from_record<D, P>(r, X, h.mu);
  return h;
}

template <int D, typename P>
__device__ __noinline__ ScanHit<P> scan_cell(int32_t c, P x0, P x1, P x2, const int32_t* __restrict__ cell_start,
                                             const int32_t* __restrict__ cell_items, const P* __restrict__ recs) {
  return scan_cell_body<D, P>(c, x0, x1, x2, cell_start, cell_items, recs);
}

// Locate X. A walk through face neighbours starts at the element deepest at
// the centre of X's cell (cell_first, ties to the lowest id): at element e
// the predicate's mu is evaluated; all mu >= 0 accepts e, otherwise the walk
// moves to the element across the face opposite the vertex with the smallest
// mu (the first on ties: the face X lies farthest outside of). adj[e][m] is
// that neighbour, -1 on the boundary. The walk gives up at a boundary face or
// after kWalkSteps evaluations and hands over to scan_cell. No rule depends on
// the order of the cell's list.
// status: 0 accepted, 1 nearest candidate, 2 empty cell. mu is the returned
// element's barycentric vector. A point inside one element gets that element
// whichever way it is found; the walk decides only between elements that all
// accept a point on their shared face.
template <int D, typename P>
__device__ __forceinline__ int32_t locate_point(const GridP<P>& g, const int32_t* __restrict__ cell_start,
                                                const int32_t* __restrict__ cell_items,
                                                const int32_t* __restrict__ cell_first,
                                                const P* __restrict__ recs, const int32_t* __restrict__ adj,
                                                const P X[D], P mu[D + 1], int& status) {
  constexpr int L = RecLen<D>::value;
  const int32_t c = cell_of<D, P>(g, X);
  int32_t e = __ldg(cell_first + c);
  if (e < 0) {  // an empty cell
    status = 2;
#pragma unroll
    for (int q = 0; q <= D; ++q) mu[q] = P(0);
    return -1;
  }
  for (int s = 0; s < kWalkSteps; ++s) {
    P r[L];
    load_record<D, P>(recs, e, r);
    // 3D: the element's neighbour row (16 B) is loaded beside its record, so
    // a step waits for one cache latency instead of two (record, then the
    // neighbour it selects): tet5m launch 1.858 -> 1.755 ms. In 2D the row is
    // 12 B and the extra loads cost more than they hide (1.276 -> 1.292 ms).
    int32_t nb[D + 1];
    if constexpr (D == 3) {
      const int4 a4 = __ldg(reinterpret_cast<const int4*>(adj) + e);
      nb[0] = a4.x; nb[1] = a4.y; nb[2] = a4.z; nb[3] = a4.w;
    }
    P m[D + 1];
    bary_from_record<D, P>(r, X, m);
    P mn = m[0];
    int am = 0;
    int32_t nx = 0;
    if constexpr (D == 3) nx = nb[0];
#pragma unroll
    for (int q = 1; q <= D; ++q)
      if (m[q] < mn) {
        mn = m[q];
        am = q;
        if constexpr (D == 3) nx = nb[q];
      }
    if (mn >= P(0)) {
#pragma unroll
      for (int q = 0; q <= D; ++q) mu[q] = m[q];
      status = 0;
      return e;
    }
    if constexpr (D == 2) nx = __ldg(adj + (int64_t)e * (D + 1) + am);
    if (nx < 0) break;
    e = nx;
  }
  // the walk gave up (boundary or step limit)
  ScanHit<P> h;
  if constexpr (D == 2) h = scan_cell_body<D, P>(c, X[0], X[1], P(0), cell_start, cell_items, recs);
  else h = scan_cell<D, P>(c, X[0], X[1], X[D - 1], cell_start, cell_items, recs);
  status = h.status;
#pragma unroll
  for (int q = 0; q <= D; ++q) mu[q] = h.mu[q];
  return h.e;
}

// P1 value of field f in element e from the per-element copy of its nodal
// values (vals: [ne][snf][4] in P, snf = the source's field count, so the
// fields of one element are contiguous; slot 3 unused in 2D)
template <int D, typename P>
__device__ __forceinline__ P eval_p1(const P* __restrict__ vals, int snf, int f, int32_t e, const P mu[D + 1]) {
  using A = Ar<P>;
  const P* v = vals + ((int64_t)e * snf + f) * 4;
  P fv[4];
  if constexpr (sizeof(P) == 4) {
    const float4 q = __ldg(reinterpret_cast<const float4*>(v));
    fv[0] = q.x; fv[1] = q.y; fv[2] = q.z; fv[3] = q.w;
  } else {
    const double2 q0 = __ldg(reinterpret_cast<const double2*>(v));
    const double2 q1 = __ldg(reinterpret_cast<const double2*>(v) + 1);
    fv[0] = q0.x; fv[1] = q0.y; fv[2] = q1.x; fv[3] = q1.y;
  }
  P s = A::mul(mu[0], fv[0]);
#pragma unroll
  for (int m = 1; m <= D; ++m) s = A::fma(mu[m], fv[m], s);
  return s;
}

// ---------------------------------------------------------------------------
// Packed FP32 pairs (sm_100 family f32x2 instructions): each lane is rounded
// exactly as the scalar operation (round to nearest, no flush; measured equal
// bit for bit on 1 M random pairs with subnormals), with half the
// instructions. A packed product that feeds a packed add can be contracted
// into one fused multiply-add (measured), so where the separate roundings
// matter the product is formed with scalar __fmul_rn.
__device__ __forceinline__ uint64_t f2_pack(float a, float b) {
  uint64_t r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(uint64_t r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// ---------------------------------------------------------------------------
// error-free transformation: Knuth's TwoSum
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float ap = __fsub_rn(s, bp);
  e = __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp));
}
// two_sum of both lanes of packed pairs (the same operations in the same order)
__device__ __forceinline__ void two_sum2(uint64_t a, uint64_t b, uint64_t& s, uint64_t& e) {
  s = f2_add(a, b);
  const uint64_t bp = f2_sub(s, a);
  const uint64_t ap = f2_sub(s, bp);
  e = f2_add(f2_sub(a, ap), f2_sub(b, bp));
}

// device error words (kernel-side status reported to the host)
enum DevErr : int32_t {
  DEV_OK = 0,
  DEV_BARRIER_TIMEOUT = 1,
  DEV_BAD_INDEX = 2,
  DEV_VALENCE = 3,
  DEV_BAD_ELEMENT = 4,
  DEV_NONFINITE = 5,
  DEV_BAD_DIAGONAL = 6
};

}  // namespace sft
