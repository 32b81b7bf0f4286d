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
constexpr int kKF = 16;  // K chunk of a streamed weight block (forward tile): one MMA
constexpr int kStages = 4;  // weight chunk buffers of the forward tile
constexpr int kTPR = 2;  // forward tile: threads per activation row (each owns half the columns)
constexpr int64_t kOffW1 = 0, kOffC1 = kH * 3, kOffW2 = kOffC1 + kH, kOffC2 = kOffW2 + kH * kH,
                  kOffW3 = kOffC2 + kH, kOffC3 = kOffW3 + kH * kH, kOffW4 = kOffC3 + kH,
                  kOffC4 = kOffW4 + kH * kH, kOffW5 = kOffC4 + kH, kOffC5 = kOffW5 + kH,
                  kNParam = kOffC5 + 1;

// shared memory of a forward tile: activation tile (128 x 256 BF16),
// kStages weight chunks (256 x 16 BF16), the first layer as float4
// {w0, w1, w2, c} per output, the two halves' partial outputs, the
// mbarriers, the TMEM address slot and a status word. About 101 KB: two
// CTAs fit on one SM.
constexpr uint32_t kSmemA = kTileM * kH * 2;        // 64 KiB
constexpr uint32_t kSmemB = kH * kKC * 2;           // 32 KiB (training GEMM chunk)
constexpr uint32_t kSmemBF = kH * kKF * 2;          // 8 KiB
constexpr uint32_t kSmemW1 = kH * 16;               // 4 KiB
constexpr uint32_t kSmemY = kTPR * kTileM * 4;      // 1 KiB
constexpr uint32_t kSmemBias = 4 * kH * 4;          // 4 KiB: c2, c3, c4, w5
constexpr uint32_t kSmemBar = 128;                  // 2 kStages + 1 mbarriers, slot, status
constexpr uint32_t kSmemFwd = kSmemA + kStages * kSmemBF + kSmemW1 + kSmemBias + kSmemY + kSmemBar;
constexpr int kChunksPerLayer = kH / kKF;

// byte offset of weight (n, k) of a 256x256 layer in the chunked layout the
// forward tile streams: chunk k / kKF is one contiguous [256][kKF] block in
// the no-swizzle K-major core-matrix order of its shared-memory image
__host__ __device__ constexpr uint32_t wchunk_offset(int n, int k) {
  return (uint32_t)(k / kKF) * kSmemBF + tc::kmajor_offset(n, k % kKF, kKF);
}
constexpr uint32_t kIdesc = tc::idesc_bf16_f32(kTileM, kH);

// special-function-unit approximations (PTX ex2.approx / rcp.approx):
// relative errors near 2^-22, far below the BF16 rounding of an activation
__device__ __forceinline__ float ex2_sfu(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_sfu(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float kNegLog2e = -1.4426950408889634f;
// sigma(z) = 1 / (1 + 2^(-z log2 e)); the limits are exact: 2^(+big) = inf
// gives 1/inf = 0, 2^(-big) = 0 gives 1. (The one-operation form
// u + u tanh(u), u = z/2, loses accuracy to cancellation for z << 0: its
// absolute error |u| 2^-11 exceeds the BF16 rounding of the activation.)
__device__ __forceinline__ float sigmoid_f(float z) { return rcp_sfu(1.0f + ex2_sfu(kNegLog2e * z)); }
// SiLU z sigma(z): two special-function operations per activation
__device__ __forceinline__ float silu_f(float z) { return z * sigmoid_f(z); }
// d silu / dz = sigma(z) (1 + z (1 - sigma(z)))
__device__ __forceinline__ float silu_grad(float z) {
  const float sg = sigmoid_f(z);
  return sg * __fmaf_rn(z, 1.0f - sg, 1.0f);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ void store_bf16x8(unsigned char* dst, const float* v) {
  __align__(16) __nv_bfloat16 h[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) h[i] = __float2bfloat16_rn(v[i]);
  *reinterpret_cast<uint4*>(dst) = *reinterpret_cast<const uint4*>(h);
}

// The weight stream of a forward CTA: chunk g (g = 0, 1, ... over the
// CTA's tiles, 3 layers of kChunksPerLayer chunks each) goes to buffer
// g % kStages by one bulk copy whose bytes complete full[b]; its MMA commits
// to mdone[b]. Thread 0 consumes chunk g (wait full, MMA, commit), then waits
// for chunk g-1's MMA (its buffer is the one chunk g+kStages-1 goes to; the
// MMA of chunk g stays queued behind it, so the tensor pipe does not idle)
// and issues that copy. The next layer's first chunks thus load during the
// current layer's epilogue. Every commit to mdone[b] is waited exactly once,
// before its buffer is refilled; parity of the k-th use of a buffer is k & 1.
struct WStream {
  int64_t next_use = 0, next_copy = 0, total = 0;
};

__device__ __forceinline__ const unsigned char* wchunk_src(const unsigned char* const Wc[3], int64_t g) {
  const int64_t per_tile = 3 * kChunksPerLayer;
  const int l = (int)((g % per_tile) / kChunksPerLayer);
  const int kc = (int)(g % kChunksPerLayer);
  return Wc[l] + (size_t)kc * kSmemBF;
}

// thread 0: copy chunk ws.next_copy (buffer free: its previous reader's MMA
// was waited by the caller, or the buffer is unused yet)
__device__ __forceinline__ void ws_copy(WStream& ws, unsigned char* B, uint64_t* full,
                                        const unsigned char* const Wc[3]) {
  const int64_t g = ws.next_copy++;
  const int b = (int)(g % kStages);
  tc::mbar_arrive_expect_tx(full + b, kSmemBF);
  tc::bulk_g2s(B + (size_t)b * kSmemBF, wchunk_src(Wc, g), kSmemBF, full + b);
}

// one 256x256 layer: TMEM[128 x 256] = A (smem, 128 x 256) * W^T. Only
// thread 0 works; ends with a commit to lbar and a bounded wait on it.
// Returns false if a wait expired (error recorded in *err).
__device__ __forceinline__ bool tc_layer_issue(WStream& ws, unsigned char* A, unsigned char* B, uint64_t* full,
                                               uint64_t* mdone, uint64_t* lbar, uint32_t& lphase,
                                               const unsigned char* const Wc[3], uint32_t taddr, int32_t* err) {
  tc::fence_after_sync();
  for (int kc = 0; kc < kChunksPerLayer; ++kc) {
    const int64_t g = ws.next_use++;
    const int b = (int)(g % kStages);
    if (!tc::mbar_wait(full + b, (uint32_t)((g / kStages) & 1), err)) return false;
    const uint64_t ad = tc::smem_desc(tc::smem_addr(A) + (uint32_t)(kc * kKF / 8) * 128u, 128u, (uint32_t)kH * 16u);
    const uint64_t bd = tc::smem_desc(tc::smem_addr(B + (size_t)b * kSmemBF), 128u, (uint32_t)kKF * 16u);
    tc::mma_bf16(taddr, ad, bd, kIdesc, kc != 0);
    tc::mma_commit(mdone + b);
    if (ws.next_copy < ws.total) {
      if (g >= 1) {
        const int64_t gp = g - 1;  // last reader of the buffer chunk next_copy goes to
        if (!tc::mbar_wait(mdone + (gp % kStages), (uint32_t)((gp / kStages) & 1), err)) return false;
      }
      ws_copy(ws, B, full, Wc);
    }
  }
  tc::mma_commit(lbar);
  const bool ok = tc::mbar_wait(lbar, lphase, err);
  lphase ^= 1u;
  return ok;
}

// shared-memory carve-up of one 128-row network tile
struct MlpSmem {
  unsigned char* A;   // activation tile [128][256] BF16, K-major core matrices
  unsigned char* B;   // kStages weight chunk buffers [256][kKF] BF16
  float4* w1;         // first layer: {W1[o][0], W1[o][1], W1[o][2], c1[o]}
  float* bias;        // [4][256]: c2, c3, c4 and the output weights w5
  float* ypart;       // [kTPR][128] partial outputs of the column halves
  uint64_t* full;     // [kStages] chunk landed (bulk-copy transaction bytes)
  uint64_t* mdone;    // [kStages] MMAs reading the chunk completed
  uint64_t* lbar;     // all MMAs of a layer completed
  uint32_t* slot;     // TMEM base address
  int* s_ok;          // result of thread 0's bounded waits
};
__device__ __forceinline__ MlpSmem mlp_smem(unsigned char* sm) {
  MlpSmem S;
  S.A = sm;
  S.B = sm + kSmemA;
  S.w1 = reinterpret_cast<float4*>(S.B + kStages * kSmemBF);
  S.bias = reinterpret_cast<float*>(S.B + kStages * kSmemBF + kSmemW1);
  S.ypart = reinterpret_cast<float*>(S.B + kStages * kSmemBF + kSmemW1 + kSmemBias);
  S.full = reinterpret_cast<uint64_t*>(S.B + kStages * kSmemBF + kSmemW1 + kSmemBias + kSmemY);
  S.mdone = S.full + kStages;
  S.lbar = S.mdone + kStages;
  S.slot = reinterpret_cast<uint32_t*>(S.lbar + 1);
  S.s_ok = reinterpret_cast<int*>(S.slot + 1);
  return S;
}

// Per-CTA setup of a network tile loop over `ntiles` tiles: TMEM allocation
// (256 columns), the mbarriers, the first-layer table and the first
// kStages - 1 weight chunk copies. Every thread calls it.
__device__ __forceinline__ uint32_t mlp_setup(const MlpSmem& S, const float* __restrict__ P,
                                              const unsigned char* const Wc[3], int64_t ntiles, WStream& ws) {
  if ((threadIdx.x >> 5) == 0) {
    tc::tmem_alloc(S.slot, kH);
    tc::tmem_relinquish();
  }
  ws.total = ntiles * 3 * kChunksPerLayer;
  if (threadIdx.x == 0) {
    for (int b = 0; b < kStages; ++b) {
      tc::mbar_init(S.full + b, 1);
      tc::mbar_init(S.mdone + b, 1);
    }
    tc::mbar_init(S.lbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    while (ws.next_copy < ws.total && ws.next_copy < kStages - 1) ws_copy(ws, S.B, S.full, Wc);
  }
  for (int o = threadIdx.x; o < kH; o += blockDim.x) {
    S.w1[o] = make_float4(__ldg(P + kOffW1 + o * 3), __ldg(P + kOffW1 + o * 3 + 1), __ldg(P + kOffW1 + o * 3 + 2),
                          __ldg(P + kOffC1 + o));
    S.bias[o] = __ldg(P + kOffC2 + o);
    S.bias[kH + o] = __ldg(P + kOffC3 + o);
    S.bias[2 * kH + o] = __ldg(P + kOffC4 + o);
    S.bias[3 * kH + o] = __ldg(P + kOffW5 + o);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  return *S.slot;
}
// End of the tile loop: thread 0 waits (bounded) for copies it issued that
// no MMA consumed (after an expired wait), then TMEM is released.
__device__ __forceinline__ void mlp_teardown(const MlpSmem& S, uint32_t taddr, WStream& ws, int32_t* err) {
  if (threadIdx.x == 0) {
    for (int64_t g = ws.next_use; g < ws.next_copy; ++g)
      if (!tc::mbar_wait(S.full + (g % kStages), (uint32_t)((g / kStages) & 1), err, 200000000ull)) break;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(taddr, kH);
}

// tiles a persistent CTA visits (tile = blockIdx.x + k gridDim.x < ntiles)
__device__ __forceinline__ int64_t cta_tiles(int64_t ntiles) {
  return blockIdx.x < ntiles ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
}

// 32 columns cc .. cc+31 of hidden layer l (accumulators in r) for this
// thread's row: bias + SiLU, then into the activation tile (l < 2) or the
// output dot product y
__device__ __forceinline__ void tile_columns(const MlpSmem& S, int l, int row, int cc, const uint32_t (&r)[32],
                                             float& y) {
  const float4* b4 = reinterpret_cast<const float4*>(S.bias + l * kH + cc);
  float v[32];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 b = b4[i];
    v[4 * i] = silu_f(__uint_as_float(r[4 * i]) + b.x);
    v[4 * i + 1] = silu_f(__uint_as_float(r[4 * i + 1]) + b.y);
    v[4 * i + 2] = silu_f(__uint_as_float(r[4 * i + 2]) + b.z);
    v[4 * i + 3] = silu_f(__uint_as_float(r[4 * i + 3]) + b.w);
  }
  if (l < 2) {
#pragma unroll
    for (int q = 0; q < 4; ++q) store_bf16x8(S.A + tc::kmajor_offset(row, cc + q * 8, kH), v + q * 8);
  } else {
    const float4* w4 = reinterpret_cast<const float4*>(S.bias + 3 * kH + cc);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const float4 w = w4[i];
      y = __fmaf_rn(bf16r(v[4 * i]), w.x, y);
      y = __fmaf_rn(bf16r(v[4 * i + 1]), w.y, y);
      y = __fmaf_rn(bf16r(v[4 * i + 2]), w.z, y);
      y = __fmaf_rn(bf16r(v[4 * i + 3]), w.w, y);
    }
  }
}

// The whole network on one 128-row tile with kTPR * 128 threads: thread t
// owns row t % 128 and the column half t / 128 (TMEM lanes of warp w are
// 32 (w % 4) .. +31). Every thread passes its row's input x and gets y.
// Layer 1 (3 -> 256) on the FMA pipe into the BF16 activation tile, three
// 256x256 layers on the tensor cores with bias + SiLU epilogues from TMEM,
// the last layer (256 -> 1) as FMA dots over each half, the halves added in
// a fixed order. False if a tensor-core wait expired.
__device__ __forceinline__ bool mlp_tile(const MlpSmem& S, const float* __restrict__ P,
                                         const unsigned char* const Wc[3], WStream& ws, const float x[3],
                                         uint32_t taddr, uint32_t& phase, int32_t* err, float& y_out) {
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
  float y = 0.f;
  for (int l = 0; l < 3; ++l) {
    if (threadIdx.x == 0) *S.s_ok = tc_layer_issue(ws, S.A, S.B, S.full, S.mdone, S.lbar, phase, Wc, taddr, err);
    __syncthreads();
    tc::fence_after_sync();
    if (!*S.s_ok) return false;
    // epilogue: bias + SiLU from TMEM, this thread's row and column half;
    // TMEM loads double buffered (the next 32 columns load while the
    // current ones are processed)
    uint32_t ra[32], rb[32];
    tc::tmem_ld32_issue(trow + (uint32_t)c0, ra);
    tc::tmem_ld_wait();
#pragma unroll 1
    for (int cc = c0; cc < c0 + kCols; cc += 64) {
      tc::tmem_ld32_issue(trow + (uint32_t)(cc + 32), rb);
      tile_columns(S, l, row, cc, ra, y);
      tc::tmem_ld_wait();
      if (cc + 64 < c0 + kCols) tc::tmem_ld32_issue(trow + (uint32_t)(cc + 64), ra);
      tile_columns(S, l, row, cc + 32, rb, y);
      tc::tmem_ld_wait();
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
  unsigned char* Wc[3] = {nullptr, nullptr, nullptr};  // BF16 in the forward tile's chunked layout
  float* grad = nullptr;                               // FP32 gradient of the mean loss
  float* m1 = nullptr;                                 // Adam moments
  float* m2 = nullptr;
  int64_t step = 0;
  cudaStream_t stream = nullptr;
};

namespace sft {
sft_status mlp_forward_dev(sft_mlp_s* m, int64_t n, const float* pts, float* out, cudaStream_t st, int32_t* d_err);
}  // namespace sft
