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
constexpr int kKC = 64;  // K chunk of a streamed weight block
constexpr int64_t kOffW1 = 0, kOffC1 = kH * 3, kOffW2 = kOffC1 + kH, kOffC2 = kOffW2 + kH * kH,
                  kOffW3 = kOffC2 + kH, kOffC3 = kOffW3 + kH * kH, kOffW4 = kOffC3 + kH,
                  kOffC4 = kOffW4 + kH * kH, kOffW5 = kOffC4 + kH, kOffC5 = kOffW5 + kH,
                  kNParam = kOffC5 + 1;

// shared memory of the forward kernel: activation tile (128 x 256 BF16),
// two weight chunks (256 x 64 BF16), one mbarrier, the TMEM address slot
constexpr uint32_t kSmemA = kTileM * kH * 2;        // 64 KiB
constexpr uint32_t kSmemB = kH * kKC * 2;           // 32 KiB
constexpr uint32_t kSmemFwd = kSmemA + 2 * kSmemB + 64;
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

// stage rows n = 0..255, k = kc*64 .. kc*64+63 of a [256][256] BF16 weight
// matrix (K-major) into a no-swizzle K-major smem block (K = 64)
__device__ __forceinline__ void load_weight_chunk(unsigned char* dst, const __nv_bfloat16* __restrict__ W, int kc) {
  for (int c = threadIdx.x; c < kH * (kKC / 8); c += blockDim.x) {
    const int n = c >> 3, kq = c & 7;
    tc::cp_async16(dst + tc::kmajor_offset(n, kq * 8, kKC), W + (int64_t)n * kH + kc * kKC + kq * 8);
  }
  tc::cp_async_commit();
}

// One hidden 256x256 layer on the tensor cores: TMEM[128 x 256] = A (smem,
// 128 x 256) * W^T, W streamed in four 64-wide K chunks (double buffered).
// Thread 0 issues the MMAs and alone polls the mbarrier (bounded); the CTA
// then meets at a barrier, so every thread takes the same branch. Returns
// false if the wait expired (error recorded in *err).
__device__ __forceinline__ bool tc_layer(unsigned char* A, unsigned char* B0, unsigned char* B1, uint64_t* bar,
                                         uint32_t& phase, uint32_t taddr, const __nv_bfloat16* __restrict__ W,
                                         int32_t* err, int* s_ok) {
  unsigned char* Bb[2] = {B0, B1};
  load_weight_chunk(Bb[0], W, 0);
  for (int kc = 0; kc < kH / kKC; ++kc) {
    tc::cp_async_wait_all();
    tc::fence_async_smem();
    __syncthreads();
    if (kc + 1 < kH / kKC) {
      // the MMAs reading buffer (kc+1)&1 (chunk kc-1) completed at the last wait
      load_weight_chunk(Bb[(kc + 1) & 1], W, kc + 1);
    }
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kKC / 16; ++kk) {
        const uint64_t ad = tc::smem_desc(tc::smem_addr(A) + (uint32_t)((kc * kKC + kk * 16) / 8) * 128u, 128u,
                                          (uint32_t)kH * 16u);
        const uint64_t bd = tc::smem_desc(tc::smem_addr(Bb[kc & 1]) + (uint32_t)kk * 256u, 128u, (uint32_t)kKC * 16u);
        tc::mma_bf16(taddr, ad, bd, kIdesc, (kc | kk) != 0);
      }
      tc::mma_commit(bar);
      *s_ok = tc::mbar_wait(bar, phase, err) ? 1 : 0;
    }
    phase ^= 1u;
    __syncthreads();
    tc::fence_after_sync();
    if (!*s_ok) {
      tc::cp_async_wait_all();
      return false;
    }
  }
  return true;
}

// shared-memory carve-up of one 128-row network tile
struct MlpSmem {
  unsigned char* A;   // activation tile [128][256] BF16, K-major core matrices
  unsigned char* B0;  // weight chunk buffers [256][64] BF16
  unsigned char* B1;
  uint64_t* bar;      // MMA completion mbarrier
  uint32_t* slot;     // TMEM base address
  int* s_ok;          // result of thread 0's bounded wait
};
__device__ __forceinline__ MlpSmem mlp_smem(unsigned char* sm) {
  MlpSmem S;
  S.A = sm;
  S.B0 = sm + kSmemA;
  S.B1 = S.B0 + kSmemB;
  S.bar = reinterpret_cast<uint64_t*>(S.B1 + kSmemB);
  S.slot = reinterpret_cast<uint32_t*>(S.bar + 1);
  S.s_ok = reinterpret_cast<int*>(S.slot + 1);
  return S;
}

// The whole network on one 128-row tile; thread r (of 128) owns row r and
// passes its input x, gets y. Every thread of the CTA must call it. Layer 1
// (3 -> 256) on the FMA pipe into the BF16 activation tile, three 256x256
// layers on the tensor cores with bias + SiLU epilogues from TMEM, the last
// layer (256 -> 1) as an FMA dot. False if a tensor-core wait expired.
__device__ __forceinline__ bool mlp_tile(const MlpSmem& S, const float* __restrict__ P,
                                         const __nv_bfloat16* __restrict__ W2, const __nv_bfloat16* __restrict__ W3,
                                         const __nv_bfloat16* __restrict__ W4, const float x[3], uint32_t taddr,
                                         uint32_t& phase, int32_t* err, float& y_out) {
  const int row = threadIdx.x;
  const int warp = threadIdx.x >> 5;
  const uint32_t trow = taddr + ((uint32_t)(32 * warp) << 16);
  for (int o = 0; o < kH; o += 8) {
    float h[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int oo = o + q;
      const float z = __fmaf_rn(__ldg(P + kOffW1 + oo * 3 + 2), x[2],
                                __fmaf_rn(__ldg(P + kOffW1 + oo * 3 + 1), x[1],
                                          __fmaf_rn(__ldg(P + kOffW1 + oo * 3), x[0], __ldg(P + kOffC1 + oo))));
      h[q] = silu_f(z);
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
    // epilogue: bias + SiLU from TMEM; rows 32*warp .. +31 (this thread: its row)
    for (int cc = 0; cc < kH / 32; ++cc) {
      float v[32];
      tc::tmem_ld32(trow + (uint32_t)(cc * 32), v);
#pragma unroll
      for (int i = 0; i < 32; ++i) v[i] = silu_f(v[i] + __ldg(P + offC[l] + cc * 32 + i));
      if (l < 2) {
#pragma unroll
        for (int q = 0; q < 4; ++q) store_bf16x8(S.A + tc::kmajor_offset(row, cc * 32 + q * 8, kH), v + q * 8);
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) y = __fmaf_rn(bf16r(v[i]), __ldg(P + kOffW5 + cc * 32 + i), y);
      }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
  }
  y_out = y + __ldg(P + kOffC5);
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
