// The surrogate source network (spec item 4): a learned black-box
// field x in R^3 -> 256 -> 256 -> 256 -> 256 -> 1 with SiLU, BF16 weights of
// the three 256x256 layers and BF16 hidden activations, FP32 accumulation.
// The 256x256 layers run on the 5th-generation tensor cores (tcgen05.mma,
// accumulators in tensor memory); the 3->256 and 256->1 layers are FP32 FMA.
//
// Parameter vector (FP32, MLP_NPARAM): W1 [256][3], c1 [256], W2 [256][256],
// c2, W3, c3, W4, c4, w5 [256], c5 [1]; weights row-major [out][in].
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>
#include "mlp.cuh"

namespace sft {

// Forward of the network on n points (x,y,z) [n][3] FP32 -> out [n] FP32.
// Persistent CTAs of 256 threads (two per SM): each 128-point tile is
// shared by the two column halves (mlp_tile).
__global__ void __launch_bounds__(kTPR * kTileM, 2) k_mlp_forward(const float* __restrict__ P,
                                                                  const unsigned char* __restrict__ W2,
                                                                  const unsigned char* __restrict__ W3,
                                                                  const unsigned char* __restrict__ W4, int64_t n,
                                                                  const float* __restrict__ pts,
                                                                  float* __restrict__ out, int32_t* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const MlpSmem S = mlp_smem(sm);
  const unsigned char* const Wc[3] = {W2, W3, W4};
  WStream ws;
  const uint32_t taddr = mlp_setup(S, P, Wc, cta_tiles((n + kTileM - 1) / kTileM), ws);
  uint32_t phase = 0;
  bool ok = true;
  const int row = threadIdx.x & (kTileM - 1);
  for (int64_t tile = blockIdx.x; ok && tile * kTileM < n; tile += gridDim.x) {
    const int64_t gi = tile * kTileM + row;
    float x[3] = {0.f, 0.f, 0.f};
    if (gi < n) {
      x[0] = pts[gi * 3];
      x[1] = pts[gi * 3 + 1];
      x[2] = pts[gi * 3 + 2];
    }
    float y = 0.f;
    ok = mlp_tile(S, P, Wc, ws, x, taddr, phase, err, y);
    if (ok && gi < n && threadIdx.x < kTileM) out[gi] = y;
  }
  mlp_teardown(S, taddr, ws, err);
}

// ---------------------------------------------------------------------------
// Training: a tcgen05 "TN" GEMM  C[M x 256] = A[M x K] * B[256 x K]^T  (both
// operands BF16, rows K-contiguous), M multiple of 128, K multiple of 64,
// split over K by blockIdx.y, with fused epilogues.
// ---------------------------------------------------------------------------
enum : int { EPI_FWD = 0, EPI_BWD = 1, EPI_ACC = 2 };

struct GemmEpi {
  const float* bias;            // FWD: [256]
  __nv_bfloat16* z;             // FWD: pre-activation [M][256]
  __nv_bfloat16* h;             // FWD: activation [M][256]
  __nv_bfloat16* hT;            // FWD: activation transposed [256][ldT] (may be null)
  const __nv_bfloat16* zprev;   // BWD: pre-activation of the layer below [M][256]
  __nv_bfloat16* dz;            // BWD: [M][256]
  __nv_bfloat16* dzT;           // BWD: [256][ldT]
  float* C;                     // ACC: C[M][256] += result (FP32 atomics)
  int64_t ldT;
};

constexpr uint32_t kGemmA = kTileM * kKC * 2;   // 16 KiB per A chunk
constexpr uint32_t kSmemGemm = 2 * kGemmA + 2 * kSmemB + 64;


template <int EPI>
__global__ void __launch_bounds__(128, 1) k_gemm_tn(int64_t M, int64_t K, int64_t klen,
                                                    const __nv_bfloat16* __restrict__ A, int64_t lda,
                                                    const __nv_bfloat16* __restrict__ B, int64_t ldb, GemmEpi e,
                                                    int32_t* err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char* As[2] = {sm, sm + kGemmA};
  unsigned char* Bs[2] = {sm + 2 * kGemmA, sm + 2 * kGemmA + kSmemB};
  uint64_t* bar = reinterpret_cast<uint64_t*>(sm + 2 * kGemmA + 2 * kSmemB);
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
  const int64_t m0 = (int64_t)blockIdx.x * kTileM;
  const int64_t kb = (int64_t)blockIdx.y * klen;
  const int64_t ke = min(K, kb + klen);
  const int nch = (int)((ke - kb) / kKC);
  auto load = [&](int buf, int64_t k0) {
    for (int c = threadIdx.x; c < kTileM * (kKC / 8); c += blockDim.x) {
      const int r = c >> 3, kq = c & 7;
      tc::cp_async16(As[buf] + tc::kmajor_offset(r, kq * 8, kKC), A + (m0 + r) * lda + k0 + kq * 8);
    }
    for (int c = threadIdx.x; c < kH * (kKC / 8); c += blockDim.x) {
      const int r = c >> 3, kq = c & 7;
      tc::cp_async16(Bs[buf] + tc::kmajor_offset(r, kq * 8, kKC), B + (int64_t)r * ldb + k0 + kq * 8);
    }
    tc::cp_async_commit();
  };
  uint32_t phase = 0;
  bool ok = nch > 0;
  if (ok) load(0, kb);
  for (int c = 0; ok && c < nch; ++c) {
    tc::cp_async_wait_all();
    tc::fence_async_smem();
    __syncthreads();
    if (c + 1 < nch) load((c + 1) & 1, kb + (int64_t)(c + 1) * kKC);
    if (threadIdx.x == 0) {
      tc::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < kKC / 16; ++kk) {
        const uint64_t ad = tc::smem_desc(tc::smem_addr(As[c & 1]) + (uint32_t)kk * 256u, 128u, (uint32_t)kKC * 16u);
        const uint64_t bd = tc::smem_desc(tc::smem_addr(Bs[c & 1]) + (uint32_t)kk * 256u, 128u, (uint32_t)kKC * 16u);
        tc::mma_bf16(taddr, ad, bd, kIdesc, (c | kk) != 0);
      }
      tc::mma_commit(bar);
      *s_ok = tc::mbar_wait(bar, phase, err) ? 1 : 0;
    }
    phase ^= 1u;
    __syncthreads();
    tc::fence_after_sync();
    ok = *s_ok != 0;
  }
  tc::cp_async_wait_all();
  if (ok) {
    const int r = threadIdx.x;
    const int64_t m = m0 + r;
    const uint32_t trow = taddr + ((uint32_t)(32 * warp) << 16);
    for (int cc = 0; cc < kH / 32; ++cc) {
      float v[32];
      tc::tmem_ld32(trow + (uint32_t)(cc * 32), v);
      if (m < M) {
        if constexpr (EPI == EPI_FWD) {
          float hh[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float z = v[i] + __ldg(e.bias + cc * 32 + i);
            v[i] = z;
            hh[i] = silu_f(z);
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            store_bf16x8(reinterpret_cast<unsigned char*>(e.z + m * kH + cc * 32 + q * 8), v + q * 8);
            store_bf16x8(reinterpret_cast<unsigned char*>(e.h + m * kH + cc * 32 + q * 8), hh + q * 8);
          }
          if (e.hT)
#pragma unroll
            for (int i = 0; i < 32; ++i) e.hT[(int64_t)(cc * 32 + i) * e.ldT + m] = __float2bfloat16_rn(hh[i]);
        } else if constexpr (EPI == EPI_BWD) {
#pragma unroll
          for (int i = 0; i < 32; ++i)
            v[i] = v[i] * silu_grad(__bfloat162float(e.zprev[m * kH + cc * 32 + i]));
#pragma unroll
          for (int q = 0; q < 4; ++q)
            store_bf16x8(reinterpret_cast<unsigned char*>(e.dz + m * kH + cc * 32 + q * 8), v + q * 8);
#pragma unroll
          for (int i = 0; i < 32; ++i) e.dzT[(int64_t)(cc * 32 + i) * e.ldT + m] = __float2bfloat16_rn(v[i]);
        } else {
#pragma unroll
          for (int i = 0; i < 32; ++i) atomicAdd(e.C + m * kH + cc * 32 + i, v[i]);
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(taddr, kH);
}

// layer 1 of a training batch (rows >= n are padding: x = 0)
__global__ void k_train_layer1(const float* __restrict__ P, const float* __restrict__ pts, int64_t n, int64_t rows,
                               __nv_bfloat16* __restrict__ z1, __nv_bfloat16* __restrict__ h1,
                               __nv_bfloat16* __restrict__ h1T) {
  const int64_t total = rows * kH;
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = k % rows;
    const int o = (int)(k / rows);
    float x0 = 0.f, x1 = 0.f, x2 = 0.f;
    if (r < n) { x0 = pts[r * 3]; x1 = pts[r * 3 + 1]; x2 = pts[r * 3 + 2]; }
    const float z = __fmaf_rn(P[kOffW1 + o * 3 + 2], x2, __fmaf_rn(P[kOffW1 + o * 3 + 1], x1,
                                                                  __fmaf_rn(P[kOffW1 + o * 3], x0, P[kOffC1 + o])));
    const float h = silu_f(z);
    z1[r * kH + o] = __float2bfloat16_rn(z);
    h1[r * kH + o] = __float2bfloat16_rn(h);
    h1T[(int64_t)o * rows + r] = __float2bfloat16_rn(h);
  }
}

// output layer, loss and its gradient for one batch: y = w5.h4 + c5,
// dL/dy = 2 (y - t) / n_total; dW5 += sum_r dy h4, dc5 += sum dy,
// dz4 = dy w5 * silu'(z4). One block of 256 threads per 128 rows.
__global__ void k_train_head(const float* __restrict__ P, const __nv_bfloat16* __restrict__ z4,
                             const __nv_bfloat16* __restrict__ h4, const float* __restrict__ t, int64_t n,
                             int64_t rows, double inv_ntot, float* __restrict__ grad, __nv_bfloat16* __restrict__ dz4,
                             __nv_bfloat16* __restrict__ dz4T, double* __restrict__ loss) {
  __shared__ float s_dy[kTileM];
  __shared__ double s_red[8];
  const int64_t r0 = (int64_t)blockIdx.x * kTileM;
  double le = 0.0;
  if (threadIdx.x < kTileM) {
    const int64_t r = r0 + threadIdx.x;
    float dy = 0.f;
    if (r < n) {
      float y = P[kOffC5];
      for (int i = 0; i < kH; ++i) y = __fmaf_rn(__bfloat162float(h4[r * kH + i]), P[kOffW5 + i], y);
      const float e = y - t[r];
      le = (double)e * (double)e;
      dy = (float)(2.0 * (double)e * inv_ntot);
    }
    s_dy[threadIdx.x] = dy;
  }
  le = warp_sum<double>(le);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = le;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    float sdy = 0.f;
    for (int w = 0; w < 8; ++w) a += s_red[w];
    for (int r = 0; r < kTileM; ++r) sdy += s_dy[r];
    atomicAdd(loss, a);
    atomicAdd(grad + kOffC5, sdy);
  }
  const int o = threadIdx.x;  // one column per thread
  const float w5 = P[kOffW5 + o];
  float gw = 0.f;
  for (int r = 0; r < kTileM; ++r) {
    const int64_t rr = r0 + r;
    if (rr >= rows) break;
    const float dy = s_dy[r];
    gw = __fmaf_rn(dy, __bfloat162float(h4[rr * kH + o]), gw);
    const float d = dy * w5 * silu_grad(__bfloat162float(z4[rr * kH + o]));
    dz4[rr * kH + o] = __float2bfloat16_rn(d);
    dz4T[(int64_t)o * rows + rr] = __float2bfloat16_rn(d);
  }
  atomicAdd(grad + kOffW5 + o, gw);
}

// bias gradients (column sums of dz) and, for layer 1, dW1 = dz1^T x
__global__ void k_train_colsum(const __nv_bfloat16* __restrict__ dz, int64_t rows, float* __restrict__ gc,
                               const float* __restrict__ pts, int64_t n, float* __restrict__ gW1) {
  const int o = threadIdx.x;
  const int64_t r0 = (int64_t)blockIdx.x * kTileM;
  float s = 0.f, w0 = 0.f, w1 = 0.f, w2 = 0.f;
  for (int r = 0; r < kTileM; ++r) {
    const int64_t rr = r0 + r;
    if (rr >= rows) break;
    const float d = __bfloat162float(dz[rr * kH + o]);
    s += d;
    if (gW1 && rr < n) {
      w0 = __fmaf_rn(d, pts[rr * 3], w0);
      w1 = __fmaf_rn(d, pts[rr * 3 + 1], w1);
      w2 = __fmaf_rn(d, pts[rr * 3 + 2], w2);
    }
  }
  atomicAdd(gc + o, s);
  if (gW1) {
    atomicAdd(gW1 + o * 3, w0);
    atomicAdd(gW1 + o * 3 + 1, w1);
    atomicAdd(gW1 + o * 3 + 2, w2);
  }
}

// Adam (Kingma & Ba) on the FP32 parameters
__global__ void k_adam(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m1,
                       float* __restrict__ m2, int64_t np, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.f - b1) * gi;
    const float b = b2 * m2[i] + (1.f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    P[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
  }
}

// BF16 copies of a 256x256 layer: W (K-major [out][in]), W^T ([in][out])
// and the forward tile's chunked layout
__global__ void k_weights_bf16(const float* __restrict__ Wf, __nv_bfloat16* __restrict__ W,
                               __nv_bfloat16* __restrict__ WT, unsigned char* __restrict__ Wc) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < kH * kH; k += gridDim.x * blockDim.x) {
    const int o = k / kH, i = k % kH;
    const __nv_bfloat16 v = __float2bfloat16_rn(Wf[k]);
    W[k] = v;
    if (WT) WT[i * kH + o] = v;
    *reinterpret_cast<__nv_bfloat16*>(Wc + wchunk_offset(o, i)) = v;
  }
}

static sft_status refresh_bf16(sft_mlp_s* m, cudaStream_t st) {
  const int64_t offW[3] = {kOffW2, kOffW3, kOffW4};
  for (int l = 0; l < 3; ++l) {
    ::sft::note_launch(), k_weights_bf16<<<64, 256, 0, st>>>(m->P + offW[l], m->W[l], m->WT[l], m->Wc[l]);
    SFT_CUDA(cudaGetLastError());
  }
  return SFT_OK;
}

// device error word of one call, freed on every return path
struct ErrWord {
  int32_t* p = nullptr;
  cudaStream_t st = nullptr;
  ~ErrWord() { dfree(p, st); }
  cudaError_t init(cudaStream_t s) {
    st = s;
    cudaError_t e = dalloc(&p, 1, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p, 0, sizeof(int32_t), s);
    return e;
  }
};

// per-batch activations of a training pass (rows = batch padded to 128)
struct TrainWs {
  int64_t rows = 0;
  __nv_bfloat16 *z[4] = {}, *h[4] = {}, *hT[3] = {}, *dz[2] = {}, *dzT = nullptr;
  double* loss = nullptr;
  cudaStream_t st = nullptr;
  ~TrainWs() {
    for (auto& p : z) dfree(p, st);
    for (auto& p : h) dfree(p, st);
    for (auto& p : hT) dfree(p, st);
    for (auto& p : dz) dfree(p, st);
    dfree(dzT, st);
    dfree(loss, st);
  }
  cudaError_t init(int64_t r, cudaStream_t s) {
    rows = r;
    st = s;
    const size_t sz = (size_t)r * kH;
    cudaError_t e = cudaSuccess;
    for (auto& p : z) if (e == cudaSuccess) e = dalloc(&p, sz, s);
    for (auto& p : h) if (e == cudaSuccess) e = dalloc(&p, sz, s);
    for (auto& p : hT) if (e == cudaSuccess) e = dalloc(&p, sz, s);
    for (auto& p : dz) if (e == cudaSuccess) e = dalloc(&p, sz, s);
    if (e == cudaSuccess) e = dalloc(&dzT, sz, s);
    if (e == cudaSuccess) e = dalloc(&loss, 1, s);
    return e;
  }
};

static sft_status gemm_attrs() {
  static bool done = false;
  if (done) return SFT_OK;
  SFT_CUDA(cudaFuncSetAttribute(k_gemm_tn<EPI_FWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemGemm));
  SFT_CUDA(cudaFuncSetAttribute(k_gemm_tn<EPI_BWD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemGemm));
  SFT_CUDA(cudaFuncSetAttribute(k_gemm_tn<EPI_ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemGemm));
  done = true;
  return SFT_OK;
}

template <int EPI>
static sft_status gemm(int64_t M, int64_t K, int64_t klen, const __nv_bfloat16* A, int64_t lda,
                       const __nv_bfloat16* B, int64_t ldb, const GemmEpi& e, cudaStream_t st, int32_t* err) {
  const dim3 grid((unsigned)((M + kTileM - 1) / kTileM), (unsigned)((K + klen - 1) / klen));
  ::sft::note_launch(), k_gemm_tn<EPI><<<grid, 128, kSmemGemm, st>>>(M, K, klen, A, lda, B, ldb, e, err);
  SFT_CUDA(cudaGetLastError());
  return SFT_OK;
}

// forward + backward of one batch (n valid rows of ws.rows) accumulating the
// gradient of loss / n_total into m->grad and sum (y - t)^2 into *ws.loss
static sft_status batch_grad(sft_mlp_s* m, TrainWs& ws, const float* pts, const float* t, int64_t n,
                             double inv_ntot, cudaStream_t st, int32_t* err) {
  const int64_t R = ws.rows;
  const int64_t offW[3] = {kOffW2, kOffW3, kOffW4}, offC[3] = {kOffC2, kOffC3, kOffC4};
  ::sft::note_launch(), k_train_layer1<<<(unsigned)std::min<int64_t>((R * kH + 255) / 256, 152 * 32), 256, 0, st>>>(
      m->P, pts, n, R, ws.z[0], ws.h[0], ws.hT[0]);
  SFT_CUDA(cudaGetLastError());
  for (int l = 0; l < 3; ++l) {
    GemmEpi e{};
    e.bias = m->P + offC[l];
    e.z = ws.z[l + 1];
    e.h = ws.h[l + 1];
    e.hT = l < 2 ? ws.hT[l + 1] : nullptr;
    e.ldT = R;
    if (sft_status r = gemm<EPI_FWD>(R, kH, kH, ws.h[l], kH, m->W[l], kH, e, st, err)) return r;
  }
  ::sft::note_launch(), k_train_head<<<(unsigned)(R / kTileM), 256, 0, st>>>(
      m->P, ws.z[3], ws.h[3], t, n, R, inv_ntot, m->grad, ws.dz[1], ws.dzT, ws.loss);
  SFT_CUDA(cudaGetLastError());
  int cur = 1;  // dz of layer l+1 lives in ws.dz[cur]
  for (int l = 2; l >= 0; --l) {  // weight matrix W_{l+2}, input activation h[l]
    GemmEpi ea{};
    ea.C = m->grad + offW[l];
    // split K (the batch rows) so that the two 128-row output tiles fill the SMs
    const int64_t klen = std::min<int64_t>(R, std::max<int64_t>(kKC, (R / 76 + kKC - 1) / kKC * kKC));
    if (sft_status r = gemm<EPI_ACC>(kH, R, klen, ws.dzT, R, ws.hT[l], R, ea, st, err)) return r;
    ::sft::note_launch(), k_train_colsum<<<(unsigned)(R / kTileM), 256, 0, st>>>(ws.dz[cur], R, m->grad + offC[l],
                                                                                 nullptr, 0, nullptr);
    SFT_CUDA(cudaGetLastError());
    GemmEpi eb{};
    eb.zprev = ws.z[l];
    eb.dz = ws.dz[cur ^ 1];
    eb.dzT = ws.dzT;
    eb.ldT = R;
    if (sft_status r = gemm<EPI_BWD>(R, kH, kH, ws.dz[cur], kH, m->WT[l], kH, eb, st, err)) return r;
    cur ^= 1;
  }
  ::sft::note_launch(), k_train_colsum<<<(unsigned)(R / kTileM), 256, 0, st>>>(ws.dz[cur], R, m->grad + kOffC1,
                                                                               pts, n, m->grad + kOffW1);
  SFT_CUDA(cudaGetLastError());
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
  const unsigned grid = (unsigned)std::min<int64_t>(tiles, 2 * (int64_t)sms);
  ::sft::note_launch(), k_mlp_forward<<<grid, kTPR * kTileM, kSmemFwd, st>>>(m->P, m->Wc[0], m->Wc[1], m->Wc[2], n,
                                                                             pts, out, d_err);
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
    for (int l = 0; l < 3 && e == cudaSuccess; ++l) {
      e = dalloc(&m->W[l], (size_t)kH * kH, st);
      if (e == cudaSuccess) e = dalloc(&m->WT[l], (size_t)kH * kH, st);
      if (e == cudaSuccess) e = dalloc(&m->Wc[l], (size_t)kH * kH * 2, st);
    }
    if (e != cudaSuccess) { r = cuda_fail(e, "alloc"); break; }
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
  for (auto& w : m->WT) dfree(w, m->stream);
  for (auto& w : m->Wc) dfree(w, m->stream);
  dfree(m->grad, m->stream);
  dfree(m->m1, m->stream);
  dfree(m->m2, m->stream);
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

static sft_status ensure_train_state(sft_mlp m, cudaStream_t st) {
  if (m->grad) return SFT_OK;
  SFT_CUDA(dalloc(&m->grad, (size_t)kNParam, st));
  SFT_CUDA(dalloc(&m->m1, (size_t)kNParam, st));
  SFT_CUDA(dalloc(&m->m2, (size_t)kNParam, st));
  SFT_CUDA(cudaMemsetAsync(m->m1, 0, sizeof(float) * kNParam, st));
  SFT_CUDA(cudaMemsetAsync(m->m2, 0, sizeof(float) * kNParam, st));
  return SFT_OK;
}

sft_status sft_mlp_loss_grad(sft_mlp m, int64_t n, const float* pts, const float* targets, float* grad_out,
                             double* loss_out, int32_t device_ptrs, void* cuda_stream) {
  if (!m || n < 1 || !pts || !targets || !grad_out) return fail(SFT_ERR_ARG, "null argument or n < 1");
  if (!device_ptrs) return fail(SFT_ERR_ARG, "sft_mlp_loss_grad takes device pointers");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (sft_status r = gemm_attrs()) return r;
  if (sft_status r = ensure_train_state(m, st)) return r;
  const int64_t B = std::min<int64_t>(16384, (n + kTileM - 1) / kTileM * kTileM);
  TrainWs ws;
  SFT_CUDA(ws.init(B, st));
  ErrWord ew;
  SFT_CUDA(ew.init(st));
  int32_t* d_err = ew.p;
  SFT_CUDA(cudaMemsetAsync(m->grad, 0, sizeof(float) * kNParam, st));
  SFT_CUDA(cudaMemsetAsync(ws.loss, 0, sizeof(double), st));
  for (int64_t b0 = 0; b0 < n; b0 += B) {
    const int64_t nb = std::min<int64_t>(B, n - b0);
    if (sft_status r = batch_grad(m, ws, pts + b0 * 3, targets + b0, nb, 1.0 / (double)n, st, d_err)) return r;
  }
  double hl = 0.0;
  int32_t herr = 0;
  SFT_CUDA(cudaMemcpyAsync(grad_out, m->grad, sizeof(float) * kNParam, cudaMemcpyDeviceToDevice, st));
  SFT_CUDA(cudaMemcpyAsync(&hl, ws.loss, sizeof(double), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  if (herr) return fail(SFT_ERR_DEVICE_STATUS, "tensor-core wait expired in the network backward");
  if (loss_out) *loss_out = hl / (double)n;
  return SFT_OK;
}

sft_status sft_mlp_train(sft_mlp m, int64_t n, const float* pts, const float* targets, int32_t epochs, int32_t batch,
                         float lr, float lr_final, double* loss_history, int32_t device_ptrs, void* cuda_stream) {
  if (!m || n < 1 || !pts || !targets || epochs < 1 || batch < 1) return fail(SFT_ERR_ARG, "bad training arguments");
  if (!device_ptrs) return fail(SFT_ERR_ARG, "sft_mlp_train takes device pointers");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  if (sft_status r = gemm_attrs()) return r;
  if (sft_status r = ensure_train_state(m, st)) return r;
  const int64_t B = std::min<int64_t>((int64_t)(batch + kTileM - 1) / kTileM * kTileM,
                                      (n + kTileM - 1) / kTileM * kTileM);
  TrainWs ws;
  SFT_CUDA(ws.init(B, st));
  ErrWord ew;
  SFT_CUDA(ew.init(st));
  int32_t* d_err = ew.p;
  const int64_t nbatch = (n + B - 1) / B;
  const int64_t total_steps = (int64_t)epochs * nbatch;
  int64_t s_step = 0;
  for (int ep = 0; ep < epochs; ++ep) {
    SFT_CUDA(cudaMemsetAsync(ws.loss, 0, sizeof(double), st));
    for (int64_t bi = 0; bi < nbatch; ++bi) {
      const int64_t b0 = bi * B, nb = std::min<int64_t>(B, n - b0);
      SFT_CUDA(cudaMemsetAsync(m->grad, 0, sizeof(float) * kNParam, st));
      if (sft_status r = batch_grad(m, ws, pts + b0 * 3, targets + b0, nb, 1.0 / (double)nb, st, d_err)) return r;
      // learning rate: geometric decay from lr to lr_final over the run
      const double frac = total_steps > 1 ? (double)(s_step++) / (double)(total_steps - 1) : 0.0;
      const float lr_t = (float)((double)lr * std::pow((double)lr_final / (double)lr, std::min(1.0, frac)));
      m->step += 1;
      const float c1 = (float)(1.0 - std::pow(0.9, (double)m->step));
      const float c2 = (float)(1.0 - std::pow(0.999, (double)m->step));
      ::sft::note_launch(), k_adam<<<256, 256, 0, st>>>(m->P, m->grad, m->m1, m->m2, kNParam, lr_t, 0.9f, 0.999f,
                                                        1e-8f, c1, c2);
      SFT_CUDA(cudaGetLastError());
      if (sft_status r = refresh_bf16(m, st)) return r;
    }
    if (loss_history) {
      double hl = 0.0;
      SFT_CUDA(cudaMemcpyAsync(&hl, ws.loss, sizeof(double), cudaMemcpyDeviceToHost, st));
      SFT_CUDA(cudaStreamSynchronize(st));
      loss_history[ep] = hl / (double)n;
    }
  }
  int32_t herr = 0;
  SFT_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  if (herr) return fail(SFT_ERR_DEVICE_STATUS, "tensor-core wait expired in training");
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
