// Device-wide exclusive scan (three phases: per-block scan, recursive scan of
// the block totals, add-back) and small conversion kernels.
#include "util.cuh"

#include <cstdint>
#include <mutex>
#include "internal.hpp"

namespace sft {

// one memory pool per device, made on first use with a release threshold of
// "never": blocks freed in stream order stay with the pool for the next
// allocation (the default pool returns them to the driver at every
// synchronisation, and remapping them costs tenths of a millisecond per call)
static std::mutex g_pool_mu;
static cudaMemPool_t g_pool[64] = {};

static cudaMemPool_t library_pool(int dev) {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;  // the device's default pool then
    }
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pool[dev] = pool;
  }
  return g_pool[dev];
}

cudaError_t pool_alloc(void** p, size_t bytes, cudaStream_t s) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool = dev >= 0 && dev < 64 ? library_pool(dev) : nullptr;
  if (!pool) return cudaMallocAsync(p, bytes, s);
  return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

void trim_pools() {
  std::lock_guard<std::mutex> lk(g_pool_mu);
  for (auto& pool : g_pool)
    if (pool) cudaMemPoolTrimTo(pool, 0);
}

namespace {
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;                         // per thread
constexpr int kScanTile = kScanThreads * kScanItems;  // per block

template <typename TIn>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const TIn* __restrict__ in, int64_t* __restrict__ out,
                                                             int64_t n, int64_t* __restrict__ tile_sums) {
  __shared__ int64_t warp_tot[kScanThreads / kWarp];
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t run = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i;
    v[i] = idx < n ? (int64_t)in[idx] : 0;
    run += v[i];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t incl = warp_inclusive_scan<int64_t>(run, lane);
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < kScanThreads / kWarp ? warp_tot[lane] : 0;
    w = warp_inclusive_scan<int64_t>(w, lane);
    if (lane < kScanThreads / kWarp) warp_tot[lane] = w;
  }
  __syncthreads();
  int64_t pre = (warp > 0 ? warp_tot[warp - 1] : 0) + incl - run;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const int64_t idx = base + i;
    if (idx < n) out[idx] = pre;
    pre += v[i];
  }
  if (threadIdx.x == kScanThreads - 1) tile_sums[blockIdx.x] = warp_tot[kScanThreads / kWarp - 1];
}

__global__ void k_add_tile_offsets(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ offs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] += offs[i / kScanTile];
}

__global__ void k_narrow(const int64_t* __restrict__ in, int32_t* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (int32_t)in[i];
}

// exclusive scan of n values into out[0..n) plus total at out[n]
template <typename TIn>
cudaError_t scan_rec(const TIn* in, int64_t* out, int64_t n, cudaStream_t s) {
  const int64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 0) return cudaMemsetAsync(out, 0, sizeof(int64_t), s);
  int64_t* sums = nullptr;
  cudaError_t e = pool_alloc(reinterpret_cast<void**>(&sums), sizeof(int64_t) * (tiles + 1), s);
  if (e != cudaSuccess) return e;
  ::sft::note_launch(), k_scan_tiles<TIn><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, sums);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (tiles == 1) {
    // out[n] = tile total; offsets are zero
    e = cudaMemcpyAsync(out + n, sums, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
  } else {
    int64_t* sums_scan = nullptr;
    e = pool_alloc(reinterpret_cast<void**>(&sums_scan), sizeof(int64_t) * (tiles + 1), s);
    if (e != cudaSuccess) return e;
    e = scan_rec<int64_t>(sums, sums_scan, tiles, s);
    if (e == cudaSuccess) {
      ::sft::note_launch(), k_add_tile_offsets<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, n, sums_scan);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out + n, sums_scan + tiles, sizeof(int64_t), cudaMemcpyDeviceToDevice, s);
    cudaFreeAsync(sums_scan, s);
  }
  cudaFreeAsync(sums, s);
  return e;
}
}  // namespace

cudaError_t exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  return scan_rec<int32_t>(in, out, n, s);
}

// err <- code (first error wins) when any of x[0..n) is not finite: one
// coalesced pass on the device (a host loop over the coordinates of a
// multi-million-node mesh took milliseconds per create)
template <typename T>
__global__ void k_check_finite(const T* __restrict__ x, int64_t n, int32_t* __restrict__ err, int32_t code) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    bad = bad || !isfinite(__ldg(x + i));
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) set_error(err, code);
}

cudaError_t check_finite(const void* x, int64_t n, bool is_double, int32_t* err, int32_t code, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (n + 255) / 256;
  const unsigned blocks = (unsigned)(want < 8LL * sms ? want : 8LL * sms);
  if (is_double)
    ::sft::note_launch(), k_check_finite<double><<<blocks, 256, 0, s>>>((const double*)x, n, err, code);
  else
    ::sft::note_launch(), k_check_finite<float><<<blocks, 256, 0, s>>>((const float*)x, n, err, code);
  return cudaGetLastError();
}

cudaError_t narrow_i64_to_i32(const int64_t* in, int32_t* out, int64_t n, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ::sft::note_launch(), k_narrow<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
  return cudaGetLastError();
}

}  // namespace sft
