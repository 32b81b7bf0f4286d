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

// (packed FP32 pair helpers f2_*: common.cuh)
// silu_f of both lanes of z2 (the same operations in the same order)
__device__ __forceinline__ void silu_pair(uint64_t z2, float& h0, float& h1) {
  float t0, t1;
  f2_unpack(f2_mul(z2, f2_pack(kNegLog2e, kNegLog2e)), t0, t1);
  float d0, d1;
  f2_unpack(f2_add(f2_pack(1.0f, 1.0f), f2_pack(ex2_sfu(t0), ex2_sfu(t1))), d0, d1);
  f2_unpack(f2_mul(z2, f2_pack(rcp_sfu(d0), rcp_sfu(d1))), h0, h1);
}
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

// The first layer in shared memory, pair-interleaved for the packed FMAs:
// outputs 2m and 2m + 1 take entries 2m = {W1[2m][0], W1[2m+1][0], W1[2m][1],
// W1[2m+1][1]} and 2m + 1 = {W1[2m][2], W1[2m+1][2], c1[2m], c1[2m+1]}.
__device__ __forceinline__ void w1_table_entry(float4* w1, const float* __restrict__ P, int o) {
  const int m = o >> 1, odd = o & 1;
  float* e0 = reinterpret_cast<float*>(w1 + 2 * m);
  float* e1 = reinterpret_cast<float*>(w1 + 2 * m + 1);
  e0[odd] = __ldg(P + kOffW1 + o * 3);
  e0[2 + odd] = __ldg(P + kOffW1 + o * 3 + 1);
  e1[odd] = __ldg(P + kOffW1 + o * 3 + 2);
  e1[2 + odd] = __ldg(P + kOffC1 + o);
}
// first-layer outputs o .. o + 7 (o even) of the point x: SiLU(W1 x + c1),
// the FMAs in the order fma(w2, x2, fma(w1, x1, fma(w0, x0, c)))
__device__ __forceinline__ void layer1_outputs8(const float4* w1, int o, const float x[3], float h[8]) {
  const uint64_t X0 = f2_pack(x[0], x[0]), X1 = f2_pack(x[1], x[1]), X2 = f2_pack(x[2], x[2]);
#pragma unroll
  for (int q = 0; q < 8; q += 2) {
    const float4 a = w1[o + q], b = w1[o + q + 1];
    const uint64_t z = f2_fma(f2_pack(b.x, b.y), X2, f2_fma(f2_pack(a.z, a.w), X1,
                                                           f2_fma(f2_pack(a.x, a.y), X0, f2_pack(b.z, b.w))));
    silu_pair(z, h[q], h[q + 1]);
  }
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
  float4* w1;         // first layer, pair-interleaved (w1_table_entry)
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
    w1_table_entry(S.w1, P, o);
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
__device__ __forceinline__ void tile_columns_a(unsigned char* A, const float* bias, int l, int row, int cc,
                                               const uint32_t (&r)[32], float& y) {
  const float4* b4 = reinterpret_cast<const float4*>(bias + l * kH + cc);
  float v[32];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const float4 b = b4[i];
    // silu_f(acc + bias) on pairs of columns
    silu_pair(f2_add(f2_pack(__uint_as_float(r[4 * i]), __uint_as_float(r[4 * i + 1])), f2_pack(b.x, b.y)),
              v[4 * i], v[4 * i + 1]);
    silu_pair(f2_add(f2_pack(__uint_as_float(r[4 * i + 2]), __uint_as_float(r[4 * i + 3])), f2_pack(b.z, b.w)),
              v[4 * i + 2], v[4 * i + 3]);
  }
  if (l < 2) {
#pragma unroll
    for (int q = 0; q < 4; ++q) store_bf16x8(A + tc::kmajor_offset(row, cc + q * 8, kH), v + q * 8);
  } else {
    const float4* w4 = reinterpret_cast<const float4*>(bias + 3 * kH + cc);
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

__device__ __forceinline__ void tile_columns(const MlpSmem& S, int l, int row, int cc, const uint32_t (&r)[32],
                                             float& y) {
  tile_columns_a(S.A, S.bias, l, row, cc, r, y);
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
    layer1_outputs8(S.w1, o, x, h);
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

// ---------------------------------------------------------------------------
// Two-group forward tile (the fused surrogate assembly): one CTA per SM,
// 2 x 256 threads. Group g (threads 256 g .. 256 g + 255) runs its own
// 128-row tiles exactly as mlp_tile does one (same arithmetic, bit-identical
// outputs), with its own activation tile, TMEM accumulator (columns
// 256 g .. +255) and named barrier. The two groups' layers take turns on the
// tensor cores in a fixed order - tile pair j: T0 L1, T1 L1, T0 L2, T1 L2,
// T0 L3, T1 L3; a group without a partner tile at the end runs its layers
// alone - so one group's epilogue overlaps the other's MMAs, and both read
// one ring of kStagesPP weight chunks fed in that order (chunk c = 16 s + k:
// K-slice k of the layer of slot s). Per slot 1 + kCopiers threads of its
// group work at once: thread 0 issues the 16 MMAs as their chunks land
// (descriptors formed once, so an MMA costs a few adds), and kCopiers
// threads each refill one class of buffers (chunk c mod kCopiers) as soon as
// the MMA that read a buffer completes (the chunk kStagesPP ahead). One
// thread doing both spent about 1,000 cycles per chunk on issue work, five
// times the MMA's own time (sur3d fused kernel 258 ms against 132 ms for two
// independent CTAs per SM); with one copier 132 ms, two 122 ms. Turn counters in shared memory
// (bounded waits) keep the slots' MMA issue and their copies each in slot
// order; the copies of slot s wait for slot s - 1's copier, so every
// mbarrier phase is waited only after the phase before it completed.
// ---------------------------------------------------------------------------
constexpr int kStagesPP = 8;                    // power of two
constexpr int kGroupThreads = kTPR * kTileM;    // 256
constexpr int kCopiers = 4;      // ring refill threads per group: 32 (1 + p) handles chunks = p (mod kCopiers)
constexpr int kCopierLane = 32;
constexpr uint32_t kSmemBarPP = 256;            // mbarriers, TMEM slot, flags, turn counters, stream state
constexpr uint32_t kSmemPP = 2 * kSmemA + kStagesPP * kSmemBF + kSmemW1 + kSmemBias + 2 * kSmemY + kSmemBarPP;
static_assert((kStagesPP & (kStagesPP - 1)) == 0 && kStagesPP <= kChunksPerLayer, "ring size");
static_assert(kStagesPP % kCopiers == 0 && kCopierLane * kCopiers < kGroupThreads, "copier classes");

struct StreamPP {
  int32_t total;         // chunks of the CTA's stream
  int32_t tail0;         // first slot of the unpaired tiles (6 x the paired tiles of a group)
  int32_t next_use;      // chunks whose MMA was issued
  int32_t next_copy[kCopiers];  // chunk c of class c % kCopiers was copied iff c < next_copy[c % kCopiers]
};

struct MlpSmemPP {
  unsigned char* A[2];
  unsigned char* B;   // kStagesPP weight chunk buffers [256][kKF] BF16
  float4* w1;
  float* bias;
  float* ypart[2];
  uint64_t* full;     // [kStagesPP]
  uint64_t* mdone;    // [kStagesPP]
  uint64_t* lbar;     // [2]: all MMAs of a group's layer completed
  uint32_t* slot;     // TMEM base address
  int* s_ok;          // [2]: MMA issue of the group's current slot succeeded
  int* s_okc;         // [2][kCopiers]: its copies of each class succeeded
  volatile int* issued;  // layer slots whose MMAs were issued
  volatile int* copied;  // [kCopiers]: layer slots whose copies of each class were issued
  StreamPP* st;
};
__device__ __forceinline__ MlpSmemPP mlp_smem_pp(unsigned char* sm) {
  MlpSmemPP S;
  S.A[0] = sm;
  S.A[1] = sm + kSmemA;
  S.B = sm + 2 * kSmemA;
  unsigned char* q = S.B + kStagesPP * kSmemBF;
  S.w1 = reinterpret_cast<float4*>(q);
  q += kSmemW1;
  S.bias = reinterpret_cast<float*>(q);
  q += kSmemBias;
  S.ypart[0] = reinterpret_cast<float*>(q);
  S.ypart[1] = reinterpret_cast<float*>(q + kSmemY);
  q += 2 * kSmemY;
  S.full = reinterpret_cast<uint64_t*>(q);
  S.mdone = S.full + kStagesPP;
  S.lbar = S.mdone + kStagesPP;
  S.slot = reinterpret_cast<uint32_t*>(S.lbar + 2);
  S.s_ok = reinterpret_cast<int*>(S.slot + 1);
  S.s_okc = S.s_ok + 2;
  S.issued = reinterpret_cast<volatile int*>(S.s_okc + 2 * kCopiers);
  S.copied = S.issued + 1;
  S.st = reinterpret_cast<StreamPP*>(q + 224);
  return S;
}
static_assert(2 * kStagesPP * 8 + 2 * 8 + 4 + 8 + 8 * kCopiers + 4 + 4 * kCopiers <= 224,
              "barrier block overlaps the stream state");
static_assert(224 + sizeof(StreamPP) <= kSmemBarPP, "stream state outside its block");

__device__ __forceinline__ void group_sync(int grp) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + grp), "r"(kGroupThreads) : "memory");
}

// bounded wait until *ctr == v (false and *err set if it did not come)
__device__ __forceinline__ bool turn_wait(volatile int* ctr, int v, int32_t* err,
                                          uint64_t timeout_ns = 2000000000ull) {
  if (*ctr == v) return true;
  const uint64_t t0 = globaltimer_ns();
  while (*ctr != v) {
    if (globaltimer_ns() - t0 > timeout_ns) {
      set_error(err, DEV_BARRIER_TIMEOUT);
      return false;
    }
  }
  return true;
}

// layer of slot s in the two-group order
__device__ __forceinline__ int slot_layer(int s, int tail0) { return s < tail0 ? (s % 6) >> 1 : (s - tail0) % 3; }

// the weights of layer l (a select, not an indexed local array)
__device__ __forceinline__ const unsigned char* layer_weights(const unsigned char* const Wc[3], int l) {
  return l == 0 ? Wc[0] : (l == 1 ? Wc[1] : Wc[2]);
}
__device__ __forceinline__ void copy_chunk_pp(const MlpSmemPP& S, const unsigned char* layer_w, int c) {
  const int b = c & (kStagesPP - 1);
  tc::mbar_arrive_expect_tx(S.full + b, kSmemBF);
  tc::bulk_g2s(S.B + (size_t)b * kSmemBF, layer_w + (size_t)(c & (kChunksPerLayer - 1)) * kSmemBF, kSmemBF,
               S.full + b);
}

// Setup over the CTA's `units` work units of `nsub` tiles each, split between
// the groups (group 0 the even ones): TMEM (512 columns), mbarriers, the
// stream state and its first kStagesPP copies, the first-layer table.
// Every thread calls it.
__device__ __forceinline__ uint32_t mlp_setup_pp(const MlpSmemPP& S, const float* __restrict__ P,
                                                 const unsigned char* const Wc[3], int64_t units, int nsub) {
  if ((threadIdx.x >> 5) == 0) {
    tc::tmem_alloc(S.slot, 2 * kH);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) {
    for (int b = 0; b < kStagesPP; ++b) {
      tc::mbar_init(S.full + b, 1);
      tc::mbar_init(S.mdone + b, 1);
    }
    tc::mbar_init(S.lbar, 1);
    tc::mbar_init(S.lbar + 1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    StreamPP& st = *S.st;
    st.total = (int32_t)(units * nsub * 3 * kChunksPerLayer);
    st.tail0 = (int32_t)(6 * (units / 2) * nsub);
    st.next_use = 0;
    *S.issued = 0;
    S.s_ok[0] = S.s_ok[1] = 1;
    for (int q2 = 0; q2 < 2 * kCopiers; ++q2) S.s_okc[q2] = 1;
    const unsigned char* w0 = layer_weights(Wc, slot_layer(0, st.tail0));
    int c = 0;
    for (; c < st.total && c < kStagesPP; ++c) copy_chunk_pp(S, w0, c);
    for (int q2 = 0; q2 < kCopiers; ++q2) {
      S.copied[q2] = 0;
      st.next_copy[q2] = c + ((q2 - c) % kCopiers + kCopiers) % kCopiers;  // first chunk of class q2 not copied
    }
  }
  for (int o = threadIdx.x; o < kH; o += blockDim.x) {
    w1_table_entry(S.w1, P, o);
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

// End of both groups' tile loops (every thread calls it): thread 0 waits
// (bounded) for copies that no MMA consumed, then TMEM is released.
__device__ __forceinline__ void mlp_teardown_pp(const MlpSmemPP& S, uint32_t taddr, int32_t* err) {
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x == 0) {
    const StreamPP& st = *S.st;
    int hi = st.next_copy[0];
    for (int q2 = 1; q2 < kCopiers; ++q2) hi = st.next_copy[q2] > hi ? st.next_copy[q2] : hi;
    for (int c = st.next_use; c < hi; ++c)
      if (c < st.next_copy[c % kCopiers] &&
          !tc::mbar_wait(S.full + (c & (kStagesPP - 1)), ((uint32_t)c / kStagesPP) & 1u, err, 200000000ull))
        break;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(taddr, 2 * kH);
}

// MMAs of layer slot `slot` (group grp's thread 0): after the previous slot's
// MMAs were issued, one MMA per chunk as it lands, a commit per chunk
// (mdone: its buffer may be refilled) and one for the layer (lbar[grp]); the
// turn is handed on before the bounded wait for the layer's MMAs.
__device__ __forceinline__ bool tc_layer_issue_pp(const MlpSmemPP& S, int grp, uint32_t taddr_g, int slot,
                                                  uint32_t& lphase, int32_t* err) {
  if (!turn_wait(S.issued, slot, err)) return false;
  __threadfence_block();
  tc::fence_after_sync();
  const uint64_t a0 = tc::smem_desc(tc::smem_addr(S.A[grp]), 128u, (uint32_t)kH * 16u);
  const uint64_t b0 = tc::smem_desc(tc::smem_addr(S.B), 128u, (uint32_t)kKF * 16u);
  const int c0 = slot * kChunksPerLayer;
  for (int kc = 0; kc < kChunksPerLayer; ++kc) {
    const int c = c0 + kc;
    const int b = c & (kStagesPP - 1);
    if (!tc::mbar_wait(S.full + b, ((uint32_t)c / kStagesPP) & 1u, err)) return false;
    // descriptor start address in 16-byte units: K-slice kc of A is 256 bytes
    // on, buffer b of the ring kSmemBF bytes on
    tc::mma_bf16(taddr_g, a0 + (uint64_t)(kc * (kKF * 16 / 16)), b0 + (uint64_t)(b * (kSmemBF / 16)), kIdesc,
                 kc != 0);
    tc::mma_commit(S.mdone + b);
  }
  tc::mma_commit(S.lbar + grp);
  S.st->next_use = c0 + kChunksPerLayer;
  __threadfence_block();
  *S.issued = slot + 1;
  const bool ok = tc::mbar_wait(S.lbar + grp, lphase, err);
  lphase ^= 1u;
  return ok;
}

// Copies of layer slot `slot`, chunks of class par = c mod kCopiers (group
// grp's thread kCopierLane (1 + par)): after the same class's copier of the
// previous slot, chunk u + kStagesPP into buffer u's slot as soon as MMA u
// (u in this slot) completed. A class's chunks live in its own buffers only,
// so each buffer sees its mbarrier phases in order.
__device__ __forceinline__ bool copy_slot_pp(const MlpSmemPP& S, const unsigned char* const Wc[3], int slot, int par,
                                             int32_t* err) {
  if (!turn_wait(S.copied + par, slot, err)) return false;
  __threadfence_block();
  StreamPP& st = *S.st;
  const int c0 = slot * kChunksPerLayer;
  const int total = st.total;
  // chunks c0 + kStagesPP .. c0 + 15 belong to this slot's layer, the rest
  // to the next slot's
  const unsigned char* w_this = layer_weights(Wc, slot_layer(slot, st.tail0));
  const unsigned char* w_next = layer_weights(Wc, slot_layer(slot + 1, st.tail0));
  for (int kc = par; kc < kChunksPerLayer; kc += kCopiers) {
    const int u = c0 + kc;  // the MMA whose buffer the next chunk reuses
    const int c = u + kStagesPP;
    if (c >= total) break;
    if (!tc::mbar_wait(S.mdone + (u & (kStagesPP - 1)), ((uint32_t)u / kStagesPP) & 1u, err)) return false;
    copy_chunk_pp(S, kc + kStagesPP < kChunksPerLayer ? w_this : w_next, c);
    st.next_copy[par] = c + kCopiers;
  }
  __threadfence_block();
  S.copied[par] = slot + 1;
  return true;
}

// The network on group grp's 128-row tile (lt = thread index in the group):
// the arithmetic of mlp_tile, layer slots slot0, slot0 + step, slot0 + 2 step.
// hook(lt) runs on the group's other threads while the first layer's MMAs
// are issued and computed (the caller's prefetch of its next tile).
template <class Hook>
__device__ __forceinline__ bool mlp_tile_pp(const MlpSmemPP& S, const float* __restrict__ P,
                                            const unsigned char* const Wc[3], int grp, int lt, const float x[3],
                                            uint32_t taddr, uint32_t& lphase, int64_t slot0, int step,
                                            int32_t* err, float& y_out, Hook&& hook) {
  constexpr int kCols = kH / kTPR;
  const int row = lt & (kTileM - 1);
  const int half = lt / kTileM;
  const int c0 = half * kCols;
  const uint32_t tcol = taddr + (uint32_t)(grp * kH);
  const uint32_t trow = tcol + ((uint32_t)(32 * ((lt >> 5) & 3)) << 16);
  unsigned char* A = S.A[grp];
  for (int o = c0; o < c0 + kCols; o += 8) {
    float h[8];
    layer1_outputs8(S.w1, o, x, h);
    store_bf16x8(A + tc::kmajor_offset(row, o, kH), h);
  }
  tc::fence_async_smem();
  group_sync(grp);
  float y = 0.f;
  for (int l = 0; l < 3; ++l) {
    const int slot = (int)(slot0 + (int64_t)l * step);
    if (lt == 0) {
      S.s_ok[grp] = tc_layer_issue_pp(S, grp, tcol, slot, lphase, err);
    } else if (lt % kCopierLane == 0 && lt <= kCopierLane * kCopiers) {
      const int par = lt / kCopierLane - 1;
      S.s_okc[grp * kCopiers + par] = copy_slot_pp(S, Wc, slot, par, err);
    } else if (l == 0) {
      hook(lt);
    }
    group_sync(grp);
    tc::fence_after_sync();
    bool good = S.s_ok[grp];
#pragma unroll
    for (int q = 0; q < kCopiers; ++q) good = good && S.s_okc[grp * kCopiers + q];
    if (!good) return false;
    uint32_t ra[32], rb[32];
    tc::tmem_ld32_issue(trow + (uint32_t)c0, ra);
    tc::tmem_ld_wait();
#pragma unroll 1
    for (int cc = c0; cc < c0 + kCols; cc += 64) {
      tc::tmem_ld32_issue(trow + (uint32_t)(cc + 32), rb);
      tile_columns_a(A, S.bias, l, row, cc, ra, y);
      tc::tmem_ld_wait();
      if (cc + 64 < c0 + kCols) tc::tmem_ld32_issue(trow + (uint32_t)(cc + 64), ra);
      tile_columns_a(A, S.bias, l, row, cc + 32, rb, y);
      tc::tmem_ld_wait();
    }
    if (l == 2) S.ypart[grp][half * kTileM + row] = y;
    tc::fence_async_smem();
    tc::fence_before_sync();
    group_sync(grp);
    tc::fence_after_sync();
  }
  float yy = S.ypart[grp][row];
#pragma unroll
  for (int h = 1; h < kTPR; ++h) yy += S.ypart[grp][h * kTileM + row];
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
