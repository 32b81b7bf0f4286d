// Shared device utilities: warp/block reductions and scans, a grid-wide
// barrier with a bounded wait (for cooperative launches), error-flag helpers.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "common.cuh"

namespace sft {

constexpr int kWarp = 32;

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void set_error(int32_t* err, int32_t code) {
  if (err) atomicCAS(err, 0, code);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// inclusive warp scan
template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v, int lane) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// inner FP32 solver of the mixed-precision solves: 1 = Chebyshev iteration
// on the proven spectrum bounds of A (one SpMV and one grid barrier per step,
// no dot products), 0 = CG (two grid barriers and two reductions per step)
#ifndef SFT_MIX_CHEBYSHEV
#define SFT_MIX_CHEBYSHEV 1
#endif
constexpr bool kMixCheb = SFT_MIX_CHEBYSHEV != 0;

// Chebyshev iteration on A y = c (A the Jacobi-scaled P1 mass matrix) with
// the spectrum of A inside [a, b] (a = 1/2, b = 2 or 5/2, widened by 1e-3
// relative for the FP32 rounding of A's entries): theta = (a + b) / 2,
// delta = (b - a) / 2, s1 = theta / delta.
// From y0 = 0, r0 = c, d0 = c / theta, rho0 = 1 / s1, each step takes
//   y += d, r -= A d, rho' = 1 / (2 s1 - rho), d' = rho' rho d + (2 rho' / delta) r
// and leaves r_k = P_k(A) c with max |P_k| on [a, b] = 1 / T_k(s1) (the
// scaled Chebyshev polynomial of degree k; Saad, Iterative Methods for Sparse
// Linear Systems, Sec. 12.3). So ||r_k|| <= eta ||c|| after
// k = ceil(acosh(1 / eta) / acosh(s1)) steps: 12 for eta = 1e-5 on
// triangles, 13 on tetrahedra.
struct ChebCoef {
  float theta, delta, s1;
};
__host__ __device__ inline ChebCoef cheb_coef(float lmax) {
  const float a = 0.5f * (1.f - 1e-3f), b = lmax * (1.f + 1e-3f);
  ChebCoef c;
  c.theta = 0.5f * (a + b);
  c.delta = 0.5f * (b - a);
  c.s1 = c.theta / c.delta;
  return c;
}
__device__ inline int cheb_steps(double eta, float s1) {
  const int k = (int)ceil(acosh(1.0 / eta) / acosh((double)s1));
  return k < 1 ? 1 : k;
}

// limit of a device wait (grid barrier, mbarrier phase) unless the caller
// sets another (sft_target_set_wait_limit for the solves on a target)
constexpr uint64_t kDefaultWaitNs = 2000000000ull;

// Grid-wide barrier for a cooperative launch (all blocks co-resident).
// Sense by generation counter; the wait gives up after `timeout_ns`, sets
// DEV_BARRIER_TIMEOUT in *err and returns false (callers then return). A
// block that finds the error word set while it waits leaves at once, so after
// one expired wait every block leaves at the next barrier it waits at.
struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};

__device__ __forceinline__ bool grid_sync(GridBarrier* bar, unsigned int nblocks, int32_t* err,
                                          uint64_t timeout_ns = kDefaultWaitNs) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned int* vgen = &bar->gen;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&bar->count, 1u);
    if (arrived == nblocks - 1) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const uint64_t t0 = globaltimer_ns();
      while (*vgen == g) {
        if (*reinterpret_cast<volatile int32_t*>(err) != 0) { ok = 0; break; }
        if (globaltimer_ns() - t0 > timeout_ns) {
          set_error(err, DEV_BARRIER_TIMEOUT);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

}  // namespace sft

// host-side helpers implemented in util.cu / api.cu
namespace sft {
// counts every kernel this library launches (exported as sft_kernel_launches)
void note_launch();
// kernels recorded into a graph are counted when the graph is launched:
// capture subtracts them (note_launches(-k)), every replay adds k
void note_launches(int64_t n);
int64_t launch_count();
// exclusive scan of int32 counts [n] into int64 offsets [n+1] (out[n] = total)
cudaError_t exclusive_scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, cudaStream_t s);
// narrow int64 -> int32 (caller checked the range)
cudaError_t narrow_i64_to_i32(const int64_t* in, int32_t* out, int64_t n, cudaStream_t s);
}  // namespace sft
