// Mesh intersection in 2D on the GPU (Sec. 3, Intersection-Based Galerkin
// Projection: the target elements are partitioned by the source elements,
// Eq. partition_ts, and each piece is integrated exactly): the exact P1
// load vector b_i = int psi_i f^s of a P1 mesh source, and the supermesh L2
// error of a target field (Eq. relative_L2_error). It is the exact judge of
// the Monte Carlo transfer at scale and the paper's comparison method.
//
// One thread per target triangle t, all arithmetic FP64:
//   1. locate t's centroid in the source (the location walk): the first
//      source triangle s0 overlaps t with positive area;
//   2. breadth-first over source face neighbours from s0: each visited source
//      triangle is clipped against t (Sutherland-Hodgman, the source triangle
//      against t's three edge half-planes in edge order); a piece of positive
//      area is split into a fan from its first vertex, every fan triangle is
//      integrated with the edge-midpoint rule (exact for the degree-2
//      products of two functions linear on the piece), and the neighbours of
//      s are queued. Source triangles overlapping t with positive area form
//      a face-connected set (they tile the convex t), so the walk reaches
//      all of them and touches only their face neighbours besides;
//   3. b: three FP64 atomics per target triangle; L2: per-block partial sums.
// Up to kMiQueue source triangles are visited per target triangle; beyond
// that the kernel sets DEV_VALENCE and the call reports SFT_ERR_UNSUPPORTED.
#include <algorithm>
#include <cmath>
#include <vector>
#include "internal.hpp"
#include "util.cuh"

namespace sft {

constexpr int kMiQueue = 256;
constexpr int kMiThreads = 128;

struct P2 { double x, y; };

__device__ __forceinline__ double cross3(P2 o, P2 a, P2 b) {
  return __dsub_rn(__dmul_rn(__dsub_rn(a.x, o.x), __dsub_rn(b.y, o.y)),
                   __dmul_rn(__dsub_rn(a.y, o.y), __dsub_rn(b.x, o.x)));
}

// clip the polygon in[0..n) by the half-plane left of the directed edge
// (p, q); returns the new vertex count (at most n + 1)
__device__ __forceinline__ int clip_edge(const P2* in, int n, P2 p, P2 q, P2* out) {
  int m = 0;
  for (int i = 0; i < n; ++i) {
    const P2 a = in[i], b = in[i + 1 == n ? 0 : i + 1];
    const double sa = cross3(p, q, a), sb = cross3(p, q, b);
    if (sa >= 0.0) out[m++] = a;
    if ((sa >= 0.0) != (sb >= 0.0)) {
      const double t = __ddiv_rn(sa, __dsub_rn(sa, sb));
      out[m++] = P2{__dadd_rn(a.x, __dmul_rn(t, __dsub_rn(b.x, a.x))), __dadd_rn(a.y, __dmul_rn(t, __dsub_rn(b.y, a.y)))};
    }
  }
  return m;
}

__device__ __forceinline__ void bary2(const P2 v[3], P2 x, double mu[3]) {
  const double area = cross3(v[0], v[1], v[2]);
  mu[1] = __ddiv_rn(cross3(v[0], x, v[2]), area);
  mu[2] = __ddiv_rn(cross3(v[0], v[1], x), area);
  mu[0] = __dsub_rn(__dsub_rn(1.0, mu[1]), mu[2]);
}

template <bool L2>
__global__ void __launch_bounds__(kMiThreads) k_mi_2d(
    const double* __restrict__ sx, const int32_t* __restrict__ sconn, const int32_t* __restrict__ adj,
    const double* __restrict__ svals, int snf, int field, const GridP<double>* __restrict__ gp,
    const int32_t* __restrict__ cell_start, const int32_t* __restrict__ cell_items,
    const int32_t* __restrict__ cell_first, const double* __restrict__ recs, const double* __restrict__ tx, const int32_t* __restrict__ tconn, int64_t net, const double* __restrict__ u,
    double* __restrict__ b, double* __restrict__ part, int32_t* err) {
  const GridP<double> g = *gp;
  double e2 = 0.0, n2 = 0.0;
  int32_t queue[kMiQueue];
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < net; t += (int64_t)gridDim.x * blockDim.x) {
    P2 tv[3];
    int32_t tn[3];
    double ut[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      tn[m] = __ldg(tconn + t * 3 + m);
      tv[m] = P2{__ldg(tx + (int64_t)tn[m] * 2), __ldg(tx + (int64_t)tn[m] * 2 + 1)};
      if (L2) ut[m] = __ldg(u + tn[m]);
    }
    // the centroid lies strictly inside t: the source triangle holding it
    // overlaps t with positive area
    double c[2] = {__ddiv_rn(__dadd_rn(__dadd_rn(tv[0].x, tv[1].x), tv[2].x), 3.0),
                   __ddiv_rn(__dadd_rn(__dadd_rn(tv[0].y, tv[1].y), tv[2].y), 3.0)};
    double mu0[3];
    int status = 0;
    const int32_t s0 = locate_point<2, double>(g, cell_start, cell_items, cell_first, recs, adj, c, mu0, status);
    if (s0 < 0) {
      set_error(err, DEV_BAD_INDEX);
      continue;
    }
    double bt[3] = {0.0, 0.0, 0.0};
    int n = 1, head = 0;
    queue[0] = s0;
    while (head < n) {
      const int32_t s = queue[head++];
      P2 sv[3];
      double fv[3];
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const int32_t v = __ldg(sconn + (int64_t)s * 3 + m);
        sv[m] = P2{__ldg(sx + (int64_t)v * 2), __ldg(sx + (int64_t)v * 2 + 1)};
        fv[m] = __ldg(svals + ((int64_t)s * snf + field) * 4 + m);
      }
      P2 poly[12], tmp[12];
      int k = 3;
#pragma unroll
      for (int m = 0; m < 3; ++m) poly[m] = sv[m];
#pragma unroll
      for (int ed = 0; ed < 3; ++ed) {
        if (k == 0) break;
        k = clip_edge(poly, k, tv[ed], tv[ed == 2 ? 0 : ed + 1], tmp);
        for (int i = 0; i < k; ++i) poly[i] = tmp[i];
      }
      bool overlap = false;
      for (int i = 1; i + 1 < k; ++i) {  // fan from the anchor poly[0]
        const P2 tri[3] = {poly[0], poly[i], poly[i + 1]};
        const double area = __dmul_rn(0.5, cross3(tri[0], tri[1], tri[2]));
        if (!(area > 0.0)) continue;
        overlap = true;
        const double w = __ddiv_rn(area, 3.0);
#pragma unroll
        for (int e = 0; e < 3; ++e) {      // edge midpoints, weight area / 3
          const P2 mp{__dmul_rn(0.5, __dadd_rn(tri[e].x, tri[e == 2 ? 0 : e + 1].x)),
                      __dmul_rn(0.5, __dadd_rn(tri[e].y, tri[e == 2 ? 0 : e + 1].y))};
          double ms[3], mt[3];
          bary2(sv, mp, ms);
          bary2(tv, mp, mt);
          double fs = 0.0;
#pragma unroll
          for (int m = 0; m < 3; ++m) fs = __dadd_rn(fs, __dmul_rn(ms[m], fv[m]));
          if (L2) {
            double ft = 0.0;
#pragma unroll
            for (int m = 0; m < 3; ++m) ft = __dadd_rn(ft, __dmul_rn(mt[m], ut[m]));
            const double d = __dsub_rn(fs, ft);
            e2 = __dadd_rn(e2, __dmul_rn(w, __dmul_rn(d, d)));
            n2 = __dadd_rn(n2, __dmul_rn(w, __dmul_rn(fs, fs)));
          } else {
#pragma unroll
            for (int m = 0; m < 3; ++m) bt[m] = __dadd_rn(bt[m], __dmul_rn(__dmul_rn(w, fs), mt[m]));
          }
        }
      }
      if (!overlap) continue;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const int32_t nb = __ldg(adj + (int64_t)s * 3 + m);
        if (nb < 0) continue;
        bool seen = false;
        for (int i = 0; i < n; ++i) seen = seen || queue[i] == nb;
        if (seen) continue;
        if (n == kMiQueue) {
          set_error(err, DEV_VALENCE);
          head = n;  // stop this element; the call reports the overflow
          break;
        }
        queue[n++] = nb;
      }
    }
    if (!L2) {
#pragma unroll
      for (int m = 0; m < 3; ++m) atomicAdd(b + tn[m], bt[m]);
    }
  }
  if (L2) {
    __shared__ double sh[2][kMiThreads / 32];
    e2 = warp_sum<double>(e2);
    n2 = warp_sum<double>(n2);
    if ((threadIdx.x & 31) == 0) {
      sh[0][threadIdx.x >> 5] = e2;
      sh[1][threadIdx.x >> 5] = n2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a = 0.0, c = 0.0;
      for (int w = 0; w < kMiThreads / 32; ++w) {
        a += sh[0][w];
        c += sh[1][w];
      }
      part[blockIdx.x * 2] = a;
      part[blockIdx.x * 2 + 1] = c;
    }
  }
}

// b (load) or the L2 error (L2 = true) of field `field`
sft_status mesh_intersection_2d(sft_source_s* s, sft_target_s* t, int field, const double* u, double* b,
                                double* err_out, double* norm_out, cudaStream_t st) {
  if (s->dim != 2 || t->dim != 2) return fail(SFT_ERR_UNSUPPORTED, "mesh intersection is 2D only");
  if (field < 0 || field >= s->nf) return fail(SFT_ERR_ARG, "field out of range");
  DevBuf<int32_t> d_err(st);
  SFT_CUDA(d_err.alloc(1));
  SFT_CUDA(cudaMemsetAsync(d_err.p, 0, sizeof(int32_t), st));
  if (sft_status r = build_locator(s, SFT_PREC_FP64, st, d_err.p)) return r;
  if (sft_status r = target_coordsP(t, SFT_PREC_FP64, st)) return r;
  const Locator& L = s->loc[SFT_PREC_FP64];
  const bool l2 = u != nullptr;
  int dev = 0, sms = 0;
  SFT_CUDA(cudaGetDevice(&dev));
  SFT_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t want = (t->ne + kMiThreads - 1) / kMiThreads;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 16));
  DevBuf<double> part(st);
  SFT_CUDA(part.alloc((size_t)blocks * 2));
  if (!l2) SFT_CUDA(cudaMemsetAsync(b, 0, sizeof(double) * t->nv, st));
  auto launch = [&](auto kern) {
    ::sft::note_launch(), kern<<<blocks, kMiThreads, 0, st>>>(
        (const double*)L.coordsP, s->conn, L.adj, (const double*)L.vals, s->nf, field, (const GridP<double>*)L.grid,
        L.cell_start, L.cell_items, L.cell_first, (const double*)L.recs, (const double*)t->coordsP[SFT_PREC_FP64], t->conn,
        t->ne, u, b, part.p, d_err.p);
  };
  if (l2) launch(k_mi_2d<true>);
  else launch(k_mi_2d<false>);
  SFT_CUDA(cudaGetLastError());
  std::vector<double> hp(l2 ? (size_t)blocks * 2 : 0);
  int32_t herr = 0;
  if (l2) SFT_CUDA(cudaMemcpyAsync(hp.data(), part.p, sizeof(double) * hp.size(), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaMemcpyAsync(&herr, d_err.p, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  if (herr == DEV_VALENCE)
    return fail(SFT_ERR_UNSUPPORTED, "a target triangle overlaps more source triangles than the intersection "
                                     "walk holds (256)");
  if (herr != 0) return fail(SFT_ERR_OUTSIDE, "a target centroid lies outside the source mesh");
  if (l2) {
    double e2 = 0.0, n2 = 0.0;
    for (unsigned i = 0; i < blocks; ++i) {  // fixed order
      e2 += hp[2 * i];
      n2 += hp[2 * i + 1];
    }
    if (err_out) *err_out = std::sqrt(e2);
    if (norm_out) *norm_out = std::sqrt(n2);
  }
  return SFT_OK;
}

}  // namespace sft

using namespace sft;

extern "C" sft_status sft_mi_load_vector(sft_source s, sft_target t, int32_t field, double* b_out,
                                         int32_t out_device, void* cuda_stream) {
  if (!s || !t || !b_out) return fail(SFT_ERR_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf<double> tmp(st);
  double* bd = b_out;
  if (!out_device) {
    SFT_CUDA(tmp.alloc((size_t)t->nv));
    bd = tmp.p;
  }
  if (sft_status r = mesh_intersection_2d(s, t, field, nullptr, bd, nullptr, nullptr, st)) return r;
  if (!out_device) {
    SFT_CUDA(cudaMemcpyAsync(b_out, bd, sizeof(double) * t->nv, cudaMemcpyDeviceToHost, st));
    SFT_CUDA(cudaStreamSynchronize(st));
  }
  return SFT_OK;
}

extern "C" sft_status sft_mi_l2_error(sft_source s, sft_target t, int32_t field, const double* u,
                                      int32_t u_on_device, void* cuda_stream, double* out2) {
  if (!s || !t || !u || !out2) return fail(SFT_ERR_ARG, "null argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  DevBuf<double> tmp(st);
  const double* ud = u;
  if (!u_on_device) {
    SFT_CUDA(tmp.alloc((size_t)t->nv));
    SFT_CUDA(cudaMemcpyAsync(tmp.p, u, sizeof(double) * t->nv, cudaMemcpyHostToDevice, st));
    ud = tmp.p;
  }
  return mesh_intersection_2d(s, t, field, ud, nullptr, out2, out2 + 1, st);
}
