// The surrogate source network (spec item 4): a learned black-box
// field x in R^3 -> 256 -> 256 -> 256 -> 256 -> 1 with SiLU, BF16 weights of
// the three 256x256 layers and BF16 hidden activations, FP32 accumulation.
// The 256x256 layers run on the 5th-generation tensor cores (tcgen05.mma,
// accumulators in tensor memory); the 3->256 and 256->1 layers are FP32 FMA.
//
// Parameter vector (FP32, MLP_NPARAM): W1 [256][3], c1 [256], W2 [256][256],
// c2, W3, c3, W4, c4, w5 [256], c5 [1]; weights row-major [out][in].
#include <cstring>
#include <vector>
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

__device__ __forceinline__ float silu_f(float z) { return __fdividef(z, 1.0f + __expf(-z)); }
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

// Forward of the network on n points (x,y,z) [n][3] FP32 -> out [n] FP32.
// One CTA of 128 threads per SM; thread i owns row i of each 128-point tile.
__global__ void __launch_bounds__(128, 1) k_mlp_forward(const float* __restrict__ P, const __nv_bfloat16* __restrict__ W2,
                                                        const __nv_bfloat16* __restrict__ W3,
                                                        const __nv_bfloat16* __restrict__ W4, int64_t n,
                                                        const float* __restrict__ pts, float* __restrict__ out,
                                                        int32_t* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* A = sm;
  unsigned char* B0 = sm + kSmemA;
  unsigned char* B1 = B0 + kSmemB;
  uint64_t* bar = reinterpret_cast<uint64_t*>(B1 + kSmemB);
  uint32_t* slot = reinterpret_cast<uint32_t*>(bar + 1);
  int* s_ok = reinterpret_cast<int*>(slot + 1);
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    tc::tmem_alloc(slot, kH);
    tc::tmem_relinquish();
  }
  if (threadIdx.x == 0) tc::mbar_init(bar, 1);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t taddr = *slot;
  const uint32_t trow = taddr + ((uint32_t)(32 * warp) << 16);
  uint32_t phase = 0;
  const __nv_bfloat16* Ws[3] = {W2, W3, W4};
  const int64_t offC[3] = {kOffC2, kOffC3, kOffC4};
  bool ok = true;
  for (int64_t tile = blockIdx.x; ok && tile * kTileM < n; tile += gridDim.x) {
    const int row = threadIdx.x;
    const int64_t gi = tile * kTileM + row;
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    if (gi < n) {
      x0 = pts[gi * 3];
      x1 = pts[gi * 3 + 1];
      x2 = pts[gi * 3 + 2];
    }
    // layer 1 (3 -> 256) on the FMA pipe, BF16 into the activation tile
    for (int o = 0; o < kH; o += 8) {
      float h[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int oo = o + q;
        const float z = __fmaf_rn(__ldg(P + kOffW1 + oo * 3 + 2), x2,
                                  __fmaf_rn(__ldg(P + kOffW1 + oo * 3 + 1), x1,
                                            __fmaf_rn(__ldg(P + kOffW1 + oo * 3), x0, __ldg(P + kOffC1 + oo))));
        h[q] = silu_f(z);
      }
      store_bf16x8(A + tc::kmajor_offset(row, o, kH), h);
    }
    tc::fence_async_smem();
    __syncthreads();
    float y = 0.f;
    for (int l = 0; l < 3 && ok; ++l) {
      ok = tc_layer(A, B0, B1, bar, phase, taddr, Ws[l], err, s_ok);
      if (!ok) break;
      // epilogue: bias + SiLU from TMEM; rows 32*warp .. +31 (this thread: its row)
      for (int cc = 0; cc < kH / 32; ++cc) {
        float v[32];
        tc::tmem_ld32(trow + (uint32_t)(cc * 32), v);
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = silu_f(v[i] + __ldg(P + offC[l] + cc * 32 + i));
        if (l < 2) {
#pragma unroll
          for (int q = 0; q < 4; ++q) store_bf16x8(A + tc::kmajor_offset(row, cc * 32 + q * 8, kH), v + q * 8);
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
    if (ok && gi < n) out[gi] = y + __ldg(P + kOffC5);
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(taddr, kH);
}

__global__ void k_to_bf16(const float* __restrict__ in, __nv_bfloat16* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = __float2bfloat16_rn(in[i]);
}

}  // namespace sft

struct sft_mlp_s {
  float* P = nullptr;                 // FP32 parameters (master)
  __nv_bfloat16* W[3] = {nullptr, nullptr, nullptr};  // BF16 copies of W2, W3, W4
  cudaStream_t stream = nullptr;
};

namespace sft {

static sft_status refresh_bf16(sft_mlp_s* m, cudaStream_t st) {
  const int64_t offW[3] = {kOffW2, kOffW3, kOffW4};
  for (int l = 0; l < 3; ++l) {
    ::sft::note_launch(), k_to_bf16<<<64, 256, 0, st>>>(m->P + offW[l], m->W[l], (int64_t)kH * kH);
    SFT_CUDA(cudaGetLastError());
  }
  return SFT_OK;
}

sft_status mlp_forward_dev(sft_mlp_s* m, int64_t n, const float* pts, float* out, cudaStream_t st, int32_t* d_err) {
  if (n <= 0) return SFT_OK;
  static bool attr_done = false;
  if (!attr_done) {
    SFT_CUDA(cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemFwd));
    attr_done = true;
  }
  int dev = 0, sms = 0;
  SFT_CUDA(cudaGetDevice(&dev));
  SFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t tiles = (n + kTileM - 1) / kTileM;
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, sms);
  ::sft::note_launch(), k_mlp_forward<<<grid, 128, kSmemFwd, st>>>(m->P, m->W[0], m->W[1], m->W[2], n, pts, out, d_err);
  SFT_CUDA(cudaGetLastError());
  return SFT_OK;
}

}  // namespace sft

using namespace sft;

extern "C" {

int64_t sft_mlp_nparam(void) { return kNParam; }

sft_status sft_mlp_create(const float* params, int32_t device_ptrs, void* cuda_stream, sft_mlp* out) {
  (void)device_ptrs;
  if (!out || !params) return fail(SFT_ERR_ARG, "null argument");
  *out = nullptr;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  auto* m = new sft_mlp_s();
  m->stream = st;
  sft_status r = SFT_OK;
  do {
    cudaError_t e = dalloc(&m->P, (size_t)kNParam, st);
    if (e != cudaSuccess) { r = cuda_fail(e, "alloc"); break; }
    e = cudaMemcpyAsync(m->P, params, sizeof(float) * kNParam, cudaMemcpyDefault, st);
    if (e != cudaSuccess) { r = cuda_fail(e, "copy"); break; }
    for (auto& w : m->W) {
      e = dalloc(&w, (size_t)kH * kH, st);
      if (e != cudaSuccess) { r = cuda_fail(e, "alloc"); break; }
    }
    if (r) break;
    if ((r = refresh_bf16(m, st))) break;
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) r = cuda_fail(e, "sync");
  } while (0);
  if (r) {
    sft_mlp_destroy(m);
    return r;
  }
  *out = m;
  return SFT_OK;
}

void sft_mlp_destroy(sft_mlp m) {
  if (!m) return;
  dfree(m->P, m->stream);
  for (auto& w : m->W) dfree(w, m->stream);
  delete m;
}

sft_status sft_mlp_params(sft_mlp m, float* out, int32_t out_device, void* cuda_stream) {
  if (!m || !out) return fail(SFT_ERR_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  SFT_CUDA(cudaMemcpyAsync(out, m->P, sizeof(float) * kNParam,
                           out_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  return SFT_OK;
}

sft_status sft_mlp_forward(sft_mlp m, int64_t n, const float* pts, float* out, int32_t device_ptrs,
                           void* cuda_stream) {
  if (!m || (n > 0 && (!pts || !out))) return fail(SFT_ERR_ARG, "null argument");
  if (n <= 0) return SFT_OK;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  float* dp = const_cast<float*>(pts);
  float* dout = out;
  std::vector<void*> tmp;
  if (!device_ptrs) {
    SFT_CUDA(dalloc(&dp, (size_t)n * 3, st));
    SFT_CUDA(dalloc(&dout, (size_t)n, st));
    SFT_CUDA(cudaMemcpyAsync(dp, pts, sizeof(float) * 3 * n, cudaMemcpyHostToDevice, st));
  }
  int32_t* d_err = nullptr;
  SFT_CUDA(dalloc(&d_err, 1, st));
  SFT_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int32_t), st));
  sft_status r = mlp_forward_dev(m, n, dp, dout, st, d_err);
  int32_t herr = 0;
  if (!r) {
    SFT_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (!device_ptrs) SFT_CUDA(cudaMemcpyAsync(out, dout, sizeof(float) * n, cudaMemcpyDeviceToHost, st));
    SFT_CUDA(cudaStreamSynchronize(st));
  }
  dfree(d_err, st);
  if (!device_ptrs) {
    dfree(dp, st);
    dfree(dout, st);
  }
  if (r) return r;
  if (herr) return fail(SFT_ERR_DEVICE_STATUS, "tensor-core wait expired in the network forward");
  return SFT_OK;
}

}  // extern "C"
