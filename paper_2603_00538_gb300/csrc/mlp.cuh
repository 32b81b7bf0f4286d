// The surrogate source network: x in R^3 -> 256 -> 256 -> 256 -> 256 -> 1
// with SiLU, BF16 weights of the three 256x256 layers and BF16 hidden
// activations, FP32 accumulation in tensor memory. Device pieces shared by
// the forward kernel, the training kernels and the fused surrogate assembly.
//
// Parameter vector (FP32, kNParam): W1 [256][3], c1 [256], W2 [256][256],
// c2, W3, c3, W4, c4, w5 [256], c5 [1]; weights row-major [out][in].
#pragma once
#include <cuda_bf16.h>
#include "internal.hpp"
#include "tc.cuh"
#include "util.cuh"

namespace sft {

constexpr int kH = 256;
constexpr int kTileM = 128;
constexpr int kKC = 64;  // K chunk of a streamed weight block (training GEMM)
constexpr int kKF = 32;  // K chunk of a streamed weight block (forward tile)
constexpr int kTPR = 2;  // forward tile: threads per activation row (each owns half the columns)
constexpr int64_t kOffW1 = 0, kOffC1 = kH * 3, kOffW2 = kOffC1 + kH, kOffC2 = kOffW2 + kH * kH,
                  kOffW3 = kOffC2 + kH, kOffC3 = kOffW3 + kH * kH, kOffW4 = kOffC3 + kH,
                  kOffC4 = kOffW4 + kH * kH, kOffW5 = kOffC4 + kH, kOffC5 = kOffW5 + kH,
                  kNParam = kOffC5 + 1;

// shared memory of a forward tile: activation tile (128 x 256 BF16), two
// weight chunks (256 x 32 BF16), the first layer as float4 {w0, w1, w2, c}
// per output, the two halves' partial outputs, one mbarrier, the TMEM
// address slot and a status word. About 101 KB: two CTAs fit on one SM.
constexpr uint32_t kSmemA = kTileM * kH * 2;        // 64 KiB
constexpr uint32_t kSmemB = kH * kKC * 2;           // 32 KiB (training GEMM chunk)
constexpr uint32_t kSmemBF = kH * kKF * 2;          // 16 KiB
constexpr uint32_t kSmemW1 = kH * 16;               // 4 KiB
constexpr uint32_t kSmemY = kTPR * kTileM * 4;      // 1 KiB
constexpr uint32_t kSmemFwd = kSmemA + 2 * kSmemBF + kSmemW1 + kSmemY + 64;
constexpr uint32_t kIdesc = tc::idesc_bf16_f32(kTileM, kH);

// SiLU z sigma(z), sigma(z) = 1 / (1 + e^-z): one exponential and one
// reciprocal on the special-function unit. (The one-operation form
// u + u tanh(u), u = z/2, loses accuracy to cancellation for z << 0: its
// absolute error |u| 2^-11 exceeds the BF16 rounding of the activation.)
__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.0f + __expf(-z)); }
// d silu / dz = sigma(z) (1 + z (1 - sigma(z)))
__device__ __forceinline__ float silu_grad(float z) {
  const float sg = __fdividef(1.0f, 1.0f + __expf(-z));
  return sg * __fmaf_rn(z, 1.0f - sg, 1.0f);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void store_bf16x8(unsigned char* dst, const float* v) {
  __align__(16) __nv_bfloat16 h[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) h[i] = __float2bfloat16_rn(v[i]);
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(h);
}

// stage rows n = 0..255, k = kc*kKF .. kc*kKF+kKF-1 of a [256][256] BF16
// weight matrix (K-major) into a no-swizzle K-major smem block (K = kKF)
__device__ __forceinline__ void load_weight_chunk(unsigned char* dst, const __nv_bfloat16* __restrict__ W, int kc) {
  constexpr int Q = kKF / 8;  // 16-byte pieces per row
  for (int c = threadIdx.x; c < kH * Q; c += blockDim.x) {
    const int n = c / Q, kq = c - n * Q;
    tc::cp_async16(dst + tc::kmajor_offset(n, kq * 8, kKF), W + (int64_t)n * kH + kc * kKF + kq * 8);
  }
  tc::cp_async_commit();
}

// One hidden 256x256 layer on the tensor cores: TMEM[128 x 256] = A (smem,
// 128 x 256) * W^T, W streamed in kKF-wide K chunks through two buffers.
// Thread 0 issues chunk kc's MMAs and commits them to mbarrier kc % 2; the
// buffer of chunk kc+1 is refilled once the MMAs of chunk kc-1 (its last
// reader) have completed, so chunk kc's MMAs run while chunk kc+1 loads.
// At most one commit per barrier is outstanding; `phase` holds the parity
// bit of each barrier. Only thread 0 polls (bounded); the CTA then meets at
// a barrier, so every thread takes the same branch. Returns false if a wait
// expired (error recorded in *err); TMEM holds the layer's accumulators on
// true.
__device__ __forceinline__ bool tc_layer(unsigned char* A, unsigned char* B0, unsigned char* B1, uint64_t* bar,
                                         uint32_t& phase, uint32_t taddr, const __nv_bfloat16* __restrict__ W,
                                         int32_t* err, int* s_ok) {
  constexpr int NK = kH / kKF;
  unsigned char* Bb[2] = {B0, B1};
  load_weight_chunk(Bb[0], W, 0);
  for (int kc = 0; kc < NK; ++kc) {
    tc::cp_async_wait_all();
    tc::fence_async_smem();
    __syncthreads();
    const bool refill = kc + 1 < NK;
    const int rb = (kc + 1) & 1;           // buffer of chunk kc+1 (last read by chunk kc-1)
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kKF / 16; ++kk) {
        const uint64_t ad = tc::smem_desc(tc::smem_addr(A) + (uint32_t)((kc * kKF + kk * 16) / 8) * 128u, 128u,
                                          (uint32_t)kH * 16u);
        const uint64_t bd = tc::smem_desc(tc::smem_addr(Bb[kc & 1]) + (uint32_t)kk * 256u, 128u, (uint32_t)kKF * 16u);
        tc::mma_bf16(taddr, ad, bd, kIdesc, (kc | kk) != 0);
      }
      tc::mma_commit(bar + (kc & 1));
      bool ok = true;
      if (refill && kc >= 1) {
        ok = tc::mbar_wait(bar + rb, (phase >> rb) & 1u, err);
      } else if (!refill) {
        // end of the layer: the last two commits (chunks NK-2 and NK-1)
        ok = tc::mbar_wait(bar + rb, (phase >> rb) & 1u, err);
        ok = ok && tc::mbar_wait(bar + (kc & 1), (phase >> (kc & 1)) & 1u, err);
      }
      *s_ok = ok ? 1 : 0;
    }
    if (refill && kc >= 1) phase ^= 1u << rb;
    if (!refill) phase ^= 3u;
    if (kc >= 1 || !refill) {
      __syncthreads();
      tc::fence_after_sync();
      if (!*s_ok) {
        tc::cp_async_wait_all();
        return false;
      }
    }
    if (refill) load_weight_chunk(Bb[rb], W, kc + 1);
  }
  return true;
}

// shared-memory carve-up of one 128-row network tile
struct MlpSmem {
  unsigned char* A;   // activation tile [128][256] BF16, K-major core matrices
  unsigned char* B0;  // weight chunk buffers [256][kKF] BF16
  unsigned char* B1;
  float4* w1;         // first layer: {W1[o][0], W1[o][1], W1[o][2], c1[o]}
  float* ypart;       // [kTPR][128] partial outputs of the column halves
  uint64_t* bar;      // two MMA completion mbarriers (one per weight buffer)
  uint32_t* slot;     // TMEM base address
  int* s_ok;          // result of thread 0's bounded wait
};
__device__ __forceinline__ MlpSmem mlp_smem(unsigned char* sm) {
  MlpSmem S;
  S.A = sm;
  S.B0 = sm + kSmemA;
  S.B1 = S.B0 + kSmemBF;
  S.w1 = reinterpret_cast<float4*>(S.B1 + kSmemBF);
  S.ypart = reinterpret_cast<float*>(S.B1 + kSmemBF + kSmemW1);
  S.bar = reinterpret_cast<uint64_t*>(S.B1 + kSmemBF + kSmemW1 + kSmemY);
  S.slot = reinterpret_cast<uint32_t*>(S.bar + 2);
  S.s_ok = reinterpret_cast<int*>(S.slot + 1);
  return S;
}

// Per-CTA setup of a network tile loop: TMEM allocation (256 columns), the
// mbarrier and the first-layer table. Every thread calls it.
__device__ __forceinline__ uint32_t mlp_setup(const MlpSmem& S, const float* __restrict__ P) {
  if ((threadIdx.x >> 5) == 0) {
    tc::tmem_alloc(S.slot, kH);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    tc::mbar_init(S.bar, 1);
    tc::mbar_init(S.bar + 1, 1);
  }
  for (int o = threadIdx.x; o < kH; o += blockDim.x)
    S.w1[o] = make_float4(__ldg(P + kOffW1 + o * 3), __ldg(P + kOffW1 + o * 3 + 1), __ldg(P + kOffW1 + o * 3 + 2),
                          __ldg(P + kOffC1 + o));
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  return *S.slot;
}
__device__ __forceinline__ void mlp_teardown(uint32_t taddr) {
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(taddr, kH);
}

// The whole network on one 128-row tile with kTPR * 128 threads: thread t
// owns row t % 128 and the column half t / 128 (TMEM lanes of warp w are
// 32 (w % 4) .. +31). Every thread passes its row's input x and gets y.
// Layer 1 (3 -> 256) on the FMA pipe into the BF16 activation tile, three
// 256x256 layers on the tensor cores with bias + SiLU epilogues from TMEM,
// the last layer (256 -> 1) as FMA dots over each half, the halves added in
// a fixed order. False if a tensor-core wait expired.
__device__ __forceinline__ bool mlp_tile(const MlpSmem& S, const float* __restrict__ P,
                                         const __nv_bfloat16* __restrict__ W2, const __nv_bfloat16* __restrict__ W3,
                                         const __nv_bfloat16* __restrict__ W4, const float x[3], uint32_t taddr,
                                         uint32_t& phase, int32_t* err, float& y_out) {
  constexpr int kCols = kH / kTPR;
  const int row = threadIdx.x & (kTileM - 1);
  const int half = threadIdx.x / kTileM;
  const int c0 = half * kCols;
  const uint32_t trow = taddr + ((uint32_t)(32 * ((threadIdx.x >> 5) & 3)) << 16);
  for (int o = c0; o < c0 + kCols; o += 8) {
    float h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float4 w = S.w1[o + q];
      h[q] = silu_f(__fmaf_rn(w.z, x[2], __fmaf_rn(w.y, x[1], __fmaf_rn(w.x, x[0], w.w))));
    }
    store_bf16x8(S.A + tc::kmajor_offset(row, o, kH), h);
  }
  tc::fence_async_smem();
  __syncthreads();
  const __nv_bfloat16* Ws[3] = {W2, W3, W4};
  const int64_t offC[3] = {kOffC2, kOffC3, kOffC4};
  float y = 0.f;
  for (int l = 0; l < 3; ++l) {
    if (!tc_layer(S.A, S.B0, S.B1, S.bar, phase, taddr, Ws[l], err, S.s_ok)) return false;
    // epilogue: bias + SiLU from TMEM, this thread's row and column half
    for (int cc = c0; cc < c0 + kCols; cc += 32) {
      float v[32];
      tc::tmem_ld32(trow + (uint32_t)cc, v);
      const float4* b4 = reinterpret_cast<const float4*>(P + offC[l] + cc);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float4 b = __ldg(b4 + i);
        v[4 * i] = silu_f(v[4 * i] + b.x);
        v[4 * i + 1] = silu_f(v[4 * i + 1] + b.y);
        v[4 * i + 2] = silu_f(v[4 * i + 2] + b.z);
        v[4 * i + 3] = silu_f(v[4 * i + 3] + b.w);
      }
      if (l < 2) {
#pragma unroll
        for (int q = 0; q < 4; ++q) store_bf16x8(S.A + tc::kmajor_offset(row, cc + q * 8, kH), v + q * 8);
      } else {
        const float4* w4 = reinterpret_cast<const float4*>(P + kOffW5 + cc);
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const float4 w = __ldg(w4 + i);
          y = __fmaf_rn(bf16r(v[4 * i]), w.x, y);
          y = __fmaf_rn(bf16r(v[4 * i + 1]), w.y, y);
          y = __fmaf_rn(bf16r(v[4 * i + 2]), w.z, y);
          y = __fmaf_rn(bf16r(v[4 * i + 3]), w.w, y);
        }
      }
    }
    if (l == 2) S.ypart[half * kTileM + row] = y;
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  float yy = S.ypart[row];
#pragma unroll
  for (int h = 1; h < kTPR; ++h) yy += S.ypart[h * kTileM + row];
  y_out = yy + __ldg(P + kOffC5);
  return true;
}

}  // namespace sft

struct sft_mlp_s {
  float* P = nullptr;                                  // FP32 parameters (master)
  __nv_bfloat16* W[3] = {nullptr, nullptr, nullptr};   // BF16 copies of W2, W3, W4 ([out][in])
  __nv_bfloat16* WT[3] = {nullptr, nullptr, nullptr};  // BF16 transposes ([in][out]) for the backward pass
  float* grad = nullptr;                               // FP32 gradient of the mean loss
  float* m1 = nullptr;                                 // Adam moments
  float* m2 = nullptr;
  int64_t step = 0;
  cudaStream_t stream = nullptr;
};

namespace sft {
sft_status mlp_forward_dev(sft_mlp_s* m, int64_t n, const float* pts, float* out, cudaStream_t st, int32_t* d_err);
}  // namespace sft
