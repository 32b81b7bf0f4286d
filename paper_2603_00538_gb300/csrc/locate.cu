// Source side of the transfer: the uniform-grid point-location structure
// (Sec. 5.3 grid search; cells per axis int(L sqrt(#elements)) in 2D, the
// cube-root analogue in 3D), built on the GPU by a counting sort of
// (cell, element) registrations, and the standalone point-query kernel used
// for the control values g (Sec. 4 step 1) and the query entry point.
//
// Layout in HBM per precision P:
//   recs  [ne][8 | 12] P  : first vertex + inverse affine map (16-B aligned rows)
//   vals  [ne][nf][4]  P  : per-element copy of the nodal values (one 16/32-B load)
//   cell_start [ncells+1], cell_items [nitems] int32: elements of each cell
//   (in no particular order); cell_first [ncells] int32: the element deepest
//   at the cell centre (largest min barycentric coordinate there, ties to the
//   lowest id), where the location walk starts; -1 for an empty cell;
//   adj [ne][d+1] int32: face neighbours (one array per source).
#include <cmath>
#include <vector>
#include "internal.hpp"
#include "util.cuh"

namespace sft {

// cells per axis: the largest n >= 1 with n^d <= L^d * ne
static int32_t cells_per_axis(int dim, int64_t ne, double L) {
  const double target = (dim == 2 ? L * L : L * L * L) * (double)ne;
  int64_t n = (int64_t)std::floor(dim == 2 ? std::sqrt(target) : std::cbrt(target));
  if (n < 1) n = 1;
  auto pw = [dim](double x) { return dim == 2 ? x * x : x * x * x; };
  while (pw((double)(n + 1)) <= target) ++n;
  while (n > 1 && pw((double)n) > target) --n;
  return (int32_t)n;
}

template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ in, TO* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if constexpr (sizeof(TO) == 4 && sizeof(TI) == 8) out[i] = __double2float_rn(in[i]);
    else out[i] = (TO)in[i];
  }
}

sft_status convert_coords(const void* in, int in_dtype, void* out, int out_prec, int64_t n, cudaStream_t st) {
  if (n <= 0) return SFT_OK;
  const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 65535 * 8);
  if (in_dtype == SFT_F64 && out_prec == SFT_PREC_FP32)
    ::sft::note_launch(), k_convert<double, float><<<blocks, 256, 0, st>>>((const double*)in, (float*)out, n);
  else if (in_dtype == SFT_F64)
    ::sft::note_launch(), k_convert<double, double><<<blocks, 256, 0, st>>>((const double*)in, (double*)out, n);
  else if (out_prec == SFT_PREC_FP32)
    ::sft::note_launch(), k_convert<float, float><<<blocks, 256, 0, st>>>((const float*)in, (float*)out, n);
  else
    ::sft::note_launch(), k_convert<float, double><<<blocks, 256, 0, st>>>((const float*)in, (double*)out, n);
  SFT_CUDA(cudaGetLastError());
  return SFT_OK;
}

// ---------------------------------------------------------------------------
// grid box: per-block min/max, then one block combines and forms GridP
// ---------------------------------------------------------------------------
template <int D, typename P>
__global__ void k_bbox_partial(const P* __restrict__ x, int64_t nv, P* __restrict__ part) {
  P lo[D], hi[D];
#pragma unroll
  for (int a = 0; a < D; ++a) { lo[a] = P(INFINITY); hi[a] = P(-INFINITY); }
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
    for (int a = 0; a < D; ++a) {
      const P v = x[i * D + a];
      lo[a] = v < lo[a] ? v : lo[a];
      hi[a] = v > hi[a] ? v : hi[a];
    }
  }
  __shared__ P slo[D][256], shi[D][256];
#pragma unroll
  for (int a = 0; a < D; ++a) { slo[a][threadIdx.x] = lo[a]; shi[a][threadIdx.x] = hi[a]; }
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int a = 0; a < D; ++a) {
        const P l2 = slo[a][threadIdx.x + s], h2 = shi[a][threadIdx.x + s];
        if (l2 < slo[a][threadIdx.x]) slo[a][threadIdx.x] = l2;
        if (h2 > shi[a][threadIdx.x]) shi[a][threadIdx.x] = h2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < D; ++a) { part[blockIdx.x * 2 * D + a] = slo[a][0]; part[blockIdx.x * 2 * D + D + a] = shi[a][0]; }
  }
}

template <int D, typename P>
__global__ void k_grid_params(const P* __restrict__ part, int nblocks, int32_t n, GridP<P>* __restrict__ g,
                              int32_t* err) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  GridP<P> r;
#pragma unroll
  for (int a = 0; a < 3; ++a) { r.lo[a] = P(0); r.inv[a] = P(0); r.h[a] = P(0); r.n[a] = 1; }
  for (int a = 0; a < D; ++a) {
    P lo = part[a], hi = part[D + a];
    for (int b = 1; b < nblocks; ++b) {
      const P l2 = part[b * 2 * D + a], h2 = part[b * 2 * D + D + a];
      lo = l2 < lo ? l2 : lo;
      hi = h2 > hi ? h2 : hi;
    }
    if (!(hi > lo)) set_error(err, DEV_BAD_ELEMENT);
    r.lo[a] = lo;
    r.inv[a] = Ar<P>::from_d(__ddiv_rn((double)n, __dsub_rn((double)hi, (double)lo)));
    r.h[a] = Ar<P>::from_d(__ddiv_rn(__dsub_rn((double)hi, (double)lo), (double)n));
    r.n[a] = n;
  }
  *g = r;
}

// ---------------------------------------------------------------------------
// per-element location records + per-element value copies
// ---------------------------------------------------------------------------
template <int D, typename P>
__device__ __forceinline__ void elem_vertices(const P* __restrict__ x, const int32_t* __restrict__ conn, int64_t e,
                                              P xv[D + 1][D]) {
#pragma unroll
  for (int m = 0; m <= D; ++m) {
    const int32_t v = conn[e * (D + 1) + m];
#pragma unroll
    for (int a = 0; a < D; ++a) xv[m][a] = x[(int64_t)v * D + a];
  }
}

template <int D, typename P>
__device__ __forceinline__ int64_t elem_cell_range(const GridP<P>& g, const P xv[D + 1][D], int32_t c0[3], int32_t c1[3]) {
  int64_t cnt = 1;
#pragma unroll
  for (int a = 0; a < 3; ++a) { c0[a] = 0; c1[a] = 0; }
#pragma unroll
  for (int a = 0; a < D; ++a) {
    P lo = xv[0][a], hi = xv[0][a];
#pragma unroll
    for (int m = 1; m <= D; ++m) {
      lo = xv[m][a] < lo ? xv[m][a] : lo;
      hi = xv[m][a] > hi ? xv[m][a] : hi;
    }
    c0[a] = cell_axis<P>(lo, g.lo[a], g.inv[a], g.n[a]);
    c1[a] = cell_axis<P>(hi, g.lo[a], g.inv[a], g.n[a]);
    cnt *= (int64_t)(c1[a] - c0[a] + 1);
  }
  return cnt;
}

// a*d - b*c in FP32 by Kahan's algorithm (the FMA recovers the rounding error
// of b*c)
__device__ __forceinline__ float det2f(float a, float d, float b, float c) {
  const float w = __fmul_rn(b, c);
  const float e = __fmaf_rn(-b, c, w);
  const float f = __fmaf_rn(a, d, -w);
  return __fadd_rn(f, e);
}

// Inverse affine map of an element into record slots [D .. D + D*D): formed in
// P from the edge vectors, with one correctly rounded reciprocal of the
// determinant (FP32: cofactors and determinant by Kahan's 2x2 determinant).
// Returns false for a non-positive element.
template <int D, typename P>
__device__ __forceinline__ bool record_map(const P xv[D + 1][D], P* r) {
  if constexpr (sizeof(P) == 4) {
    float e[D][D];
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int a = 0; a < D; ++a) e[k][a] = __fsub_rn(xv[k + 1][a], xv[0][a]);
    if constexpr (D == 2) {
      const float det = det2f(e[0][0], e[1][1], e[1][0], e[0][1]);
      const float inv = __frcp_rn(det);
      r[2] = __fmul_rn(e[1][1], inv);
      r[3] = __fmul_rn(-e[1][0], inv);
      r[4] = __fmul_rn(-e[0][1], inv);
      r[5] = __fmul_rn(e[0][0], inv);
      return det > 0.f;
    } else {
      const float* e1 = e[0];
      const float* e2 = e[1];
      const float* e3 = e[2];
      const float c23[3] = {det2f(e2[1], e3[2], e2[2], e3[1]), det2f(e2[2], e3[0], e2[0], e3[2]),
                            det2f(e2[0], e3[1], e2[1], e3[0])};
      const float c31[3] = {det2f(e3[1], e1[2], e3[2], e1[1]), det2f(e3[2], e1[0], e3[0], e1[2]),
                            det2f(e3[0], e1[1], e3[1], e1[0])};
      const float c12[3] = {det2f(e1[1], e2[2], e1[2], e2[1]), det2f(e1[2], e2[0], e1[0], e2[2]),
                            det2f(e1[0], e2[1], e1[1], e2[0])};
      const float det = __fmaf_rn(e1[2], c23[2], __fmaf_rn(e1[1], c23[1], __fmul_rn(e1[0], c23[0])));
      const float inv = __frcp_rn(det);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        r[3 + q] = __fmul_rn(c23[q], inv);
        r[6 + q] = __fmul_rn(c31[q], inv);
        r[9 + q] = __fmul_rn(c12[q], inv);
      }
      return det > 0.f;
    }
  } else {
    double e[D][D];
#pragma unroll
    for (int k = 0; k < D; ++k)
#pragma unroll
      for (int a = 0; a < D; ++a) e[k][a] = __dsub_rn(xv[k + 1][a], xv[0][a]);
    if constexpr (D == 2) {
      const double det = __dsub_rn(__dmul_rn(e[0][0], e[1][1]), __dmul_rn(e[1][0], e[0][1]));
      const double inv = __drcp_rn(det);
      r[2] = __dmul_rn(e[1][1], inv);
      r[3] = __dmul_rn(-e[1][0], inv);
      r[4] = __dmul_rn(-e[0][1], inv);
      r[5] = __dmul_rn(e[0][0], inv);
      return det > 0.0;
    } else {
      const double* e1 = e[0];
      const double* e2 = e[1];
      const double* e3 = e[2];
      auto crs = [](const double* u, const double* w, double* o) {
        o[0] = __dsub_rn(__dmul_rn(u[1], w[2]), __dmul_rn(u[2], w[1]));
        o[1] = __dsub_rn(__dmul_rn(u[2], w[0]), __dmul_rn(u[0], w[2]));
        o[2] = __dsub_rn(__dmul_rn(u[0], w[1]), __dmul_rn(u[1], w[0]));
      };
      double c23[3], c31[3], c12[3];
      crs(e2, e3, c23);
      crs(e3, e1, c31);
      crs(e1, e2, c12);
      const double det =
          __dadd_rn(__dadd_rn(__dmul_rn(e1[0], c23[0]), __dmul_rn(e1[1], c23[1])), __dmul_rn(e1[2], c23[2]));
      const double inv = __drcp_rn(det);
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        r[3 + q] = __dmul_rn(c23[q], inv);
        r[6 + q] = __dmul_rn(c31[q], inv);
        r[9 + q] = __dmul_rn(c12[q], inv);
      }
      return det > 0.0;
    }
  }
}

template <int D, typename P, typename TV>
__global__ void k_records(const P* __restrict__ x, const int32_t* __restrict__ conn, const TV* __restrict__ values,
                          int64_t nv, int64_t ne, int nf, P* __restrict__ recs, P* __restrict__ vals, int32_t* err,
                          double* __restrict__ evol) {
  constexpr int L = RecLen<D>::value;
  
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[D + 1];
    bool ok = true;
#pragma unroll
    for (int m = 0; m <= D; ++m) {
      v[m] = conn[e * (D + 1) + m];
      ok = ok && v[m] >= 0 && v[m] < nv;
    }
    if (!ok) {
      set_error(err, DEV_BAD_INDEX);
      continue;
    }
    P xv[D + 1][D];
    elem_vertices<D, P>(x, conn, e, xv);
    P r[L];
#pragma unroll
    for (int q = 0; q < L; ++q) r[q] = P(0);
#pragma unroll
    for (int a = 0; a < D; ++a) r[a] = xv[0][a];
    if (!record_map<D, P>(xv, r)) set_error(err, DEV_BAD_ELEMENT);
#pragma unroll
    for (int q = 0; q < L; ++q) recs[e * L + q] = r[q];
    if (evol) {
      // FP64 measure of the element (exact differences of the stored coordinates)
      double xd[D + 1][D];
#pragma unroll
      for (int m = 0; m <= D; ++m)
#pragma unroll
        for (int a = 0; a < D; ++a) xd[m][a] = f2d(xv[m][a]);
      double vol;
      if constexpr (D == 2) {
        vol = 0.5 * ((xd[1][0] - xd[0][0]) * (xd[2][1] - xd[0][1]) - (xd[2][0] - xd[0][0]) * (xd[1][1] - xd[0][1]));
      } else {
        double e1[3], e2[3], e3[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) { e1[a] = xd[1][a] - xd[0][a]; e2[a] = xd[2][a] - xd[0][a]; e3[a] = xd[3][a] - xd[0][a]; }
        vol = (e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
               e1[2] * (e2[0] * e3[1] - e2[1] * e3[0])) * (1.0 / 6.0);
      }
      evol[e] = vol;
    }
    for (int f = 0; f < nf; ++f) {
#pragma unroll
      for (int m = 0; m < 4; ++m)
        vals[((int64_t)e * nf + f) * 4 + m] = m <= D ? P(values[(int64_t)f * nv + v[m]]) : P(0);
    }
  }
}

// centre of cell index i along axis a: lo + (i + 1/2) h as one FMA in P
template <typename P>
__device__ __forceinline__ P cell_centre(const GridP<P>& g, int a, int32_t i) {
  return Ar<P>::fma(Ar<P>::add((P)i, P(0.5)), g.h[a], g.lo[a]);
}

// Can the cell box (centre c, half widths w) hold a point of the element with
// location record r? Each barycentric coordinate is affine; its largest value
// over the box is its value at the centre plus sum_a |gradient_a| w_a. The
// element is left out when that value is below -2^-10 for some coordinate
// (the box lies outside a face plane by a margin far above the predicate's
// rounding, so the test never drops an element a point of the cell could be
// accepted by). Fixed evaluation order in P.
template <int D, typename P>
__device__ __forceinline__ bool cell_may_hold(const P* r, const P c[D], const P w[D]) {
  using A = Ar<P>;
  const P eps = P(0.0009765625);
  P d[D], s[D], tsum = P(0);
#pragma unroll
  for (int a = 0; a < D; ++a) d[a] = A::sub(c[a], r[a]);
#pragma unroll
  for (int m = 0; m < D; ++m) {
    const P* row = r + D + m * D;
    P t = A::mul(row[0], d[0]);
    P sp = A::mul(row[0] < P(0) ? -row[0] : row[0], w[0]);
#pragma unroll
    for (int a = 1; a < D; ++a) {
      t = A::fma(row[a], d[a], t);
      sp = A::fma(row[a] < P(0) ? -row[a] : row[a], w[a], sp);
    }
    if (A::add(t, sp) < -eps) return false;
    tsum = m == 0 ? t : A::add(tsum, t);
#pragma unroll
    for (int a = 0; a < D; ++a) s[a] = m == 0 ? row[a] : A::add(s[a], row[a]);
  }
  P S = A::mul(s[0] < P(0) ? -s[0] : s[0], w[0]);
#pragma unroll
  for (int a = 1; a < D; ++a) S = A::fma(s[a] < P(0) ? -s[a] : s[a], w[a], S);
  return !(A::add(A::sub(P(1), tsum), S) < -eps);
}

// one filled registration: the element and the depth of the cell centre in it,
// stored together so that the fill writes one scattered entry, not two
template <typename P> struct RegEntry;
template <> struct alignas(8) RegEntry<float> { int32_t id; float depth; };
template <> struct alignas(16) RegEntry<double> { int32_t id; int32_t pad; double depth; };

// one registration per (element, cell) that passes cell_may_hold: count, or
// fill the element id and the depth of the cell centre in the
// element (its min barycentric coordinate there, evaluated exactly as a
// query at that point would be), which orders the cell's list
// The count pass records which cells of the element's bounding box passed
// the test as a bit mask (bit k: the k-th box cell in x-fastest order) when
// the box has at most kMaskCells cells; the fill pass then registers exactly
// those without testing again. Larger boxes (bit 31 set) are tested again.
constexpr int kMaskCells = 31;
constexpr uint32_t kMaskRetest = 0x80000000u;

template <int D, typename P, bool FILL>
__global__ void k_register(const P* __restrict__ x, const int32_t* __restrict__ conn, const P* __restrict__ recs,
                           int64_t nv, int64_t ne, const GridP<P>* __restrict__ gp, int32_t* __restrict__ cell_count,
                           const int32_t* __restrict__ cell_start, RegEntry<P>* __restrict__ reg,
                           uint32_t* __restrict__ mask) {
  constexpr int RL = RecLen<D>::value;
  const GridP<P> g = *gp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    bool ok = true;
#pragma unroll
    for (int m = 0; m <= D; ++m) {
      const int32_t v = conn[e * (D + 1) + m];
      ok = ok && v >= 0 && v < nv;
    }
    if (!ok) continue;  // reported by k_records; never read out of range
    P xv[D + 1][D];
    elem_vertices<D, P>(x, conn, e, xv);
    int32_t c0[3], c1[3];
    const int64_t nbox = elem_cell_range<D, P>(g, xv, c0, c1);
    P r[RL];
    load_record<D, P>(recs, (int32_t)e, r);
    P w[D];
#pragma unroll
    for (int a = 0; a < D; ++a) w[a] = Ar<P>::mul(g.h[a], P(0.5));
    const bool use_mask = nbox <= kMaskCells;
    const uint32_t have = FILL ? __ldg(mask + e) : 0u;
    const bool retest = !FILL || (have & kMaskRetest) != 0u;
    uint32_t bits = 0u;
    int k = 0;
    for (int32_t iz = c0[2]; iz <= c1[2]; ++iz)
      for (int32_t iy = c0[1]; iy <= c1[1]; ++iy)
        for (int32_t ix = c0[0]; ix <= c1[0]; ++ix, ++k) {
          const int32_t idx[3] = {ix, iy, iz};
          P cc[D];
#pragma unroll
          for (int a = 0; a < D; ++a) cc[a] = cell_centre<P>(g, a, idx[a]);
          if (retest) {
            if (!cell_may_hold<D, P>(r, cc, w)) continue;
          } else if (!((have >> k) & 1u)) {
            continue;
          }
          if (!FILL && use_mask) bits |= 1u << k;
          const int64_t c = ((int64_t)iz * g.n[1] + iy) * g.n[0] + ix;
          const int32_t pos = atomicAdd(cell_count + c, 1);
          if (FILL) {
            P mu[D + 1];
            bary_from_record<D, P>(r, cc, mu);
            P mn = mu[0];
#pragma unroll
            for (int q = 1; q <= D; ++q) mn = mu[q] < mn ? mu[q] : mn;
            RegEntry<P> en;
            if constexpr (sizeof(P) == 8) en.pad = 0;
            en.id = (int32_t)e;
            en.depth = mn;
            reg[(int64_t)cell_start[c] + pos] = en;
          }
        }
    if (!FILL) mask[e] = use_mask ? bits : kMaskRetest;
  }
}

// Start element of each cell and its list of ids: the fill leaves a cell's
// entries in arbitrary order, which no rule depends on (the walk starts at
// the element deepest at the cell centre, ties to the lowest id; the
// fallback takes the best-scoring candidate whatever the order). One thread
// per cell: the argmax of (depth, -id) over its entries, and the ids copied
// into the cell's list.
template <typename P>
__global__ void k_cell_first(const int32_t* __restrict__ cell_start, const RegEntry<P>* __restrict__ reg,
                             int64_t ncells, int32_t* __restrict__ items, int32_t* __restrict__ first) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncells; c += (int64_t)gridDim.x * blockDim.x) {
    const int32_t p0 = __ldg(cell_start + c), p1 = __ldg(cell_start + c + 1);
    int32_t best = -1;
    P bd = P(0);
    for (int32_t p = p0; p < p1; ++p) {
      const RegEntry<P> en = reg[p];
      if (best < 0 || en.depth > bd || (en.depth == bd && en.id < best)) {
        best = en.id;
        bd = en.depth;
      }
      items[p] = en.id;
    }
    first[c] = best;
  }
}

// Face neighbours of every element for the location walk: adj[e][m] = the
// other element holding every vertex of the face opposite local vertex m
// (the smallest id if several), -1 on the boundary. Found through the grid:
// an element holding vertex v has v in its closure, and registration keeps
// every cell a point of the element can fall in, so it is listed in the cell
// of v. Faces m != 0 hold vertex 0 and are matched against the list of
// cell(x_0); face 0 holds vertex 1 and is matched against the list of
// cell(x_1). Two threads per element, one per list (they write different
// entries of the element's row).
template <int D, typename P>
__global__ void k_adjacency(const P* __restrict__ x, const int32_t* __restrict__ conn, int64_t nv, int64_t ne,
                            const GridP<P>* __restrict__ gp, const int32_t* __restrict__ cell_start,
                            const int32_t* __restrict__ cell_items, int32_t* __restrict__ adj) {
  constexpr int K = D + 1;
  const GridP<P> g = *gp;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < 2 * ne; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i >> 1;
    const int pass = (int)(i & 1);
    int32_t v[K];
    bool ok = true;
#pragma unroll
    for (int m = 0; m < K; ++m) {
      v[m] = __ldg(conn + e * K + m);
      ok = ok && v[m] >= 0 && v[m] < nv;
    }
    int32_t best[K];
#pragma unroll
    for (int m = 0; m < K; ++m) best[m] = INT32_MAX;
    if (ok) {
      P X[D];
      const int32_t vp = pass == 0 ? v[0] : v[1];
#pragma unroll
      for (int a = 0; a < D; ++a) X[a] = __ldg(x + (int64_t)vp * D + a);
      const int32_t c = cell_of<D, P>(g, X);
      const int32_t p1 = __ldg(cell_start + c + 1);
#pragma unroll 2
      for (int32_t p = __ldg(cell_start + c); p < p1; ++p) {
        const int32_t e2 = __ldg(cell_items + p);
        if (e2 == (int32_t)e) continue;
        int32_t w[K];
#pragma unroll
        for (int r = 0; r < K; ++r) w[r] = __ldg(conn + (int64_t)e2 * K + r);
        int shared = 0, miss = 0;
#pragma unroll
        for (int m = 0; m < K; ++m) {
          bool in = false;
#pragma unroll
          for (int r = 0; r < K; ++r) in = in || w[r] == v[m];
          shared += in;
          miss = in ? miss : m;
        }
        if (shared != D || (pass == 0) == (miss == 0)) continue;
#pragma unroll
        for (int m = 0; m < K; ++m)
          if (m == miss && e2 < best[m]) best[m] = e2;
      }
    }
    // pass 0 owns faces 1..D, pass 1 face 0
#pragma unroll
    for (int m = 0; m < K; ++m)
      if ((m == 0) == (pass == 1)) adj[e * K + m] = best[m] == INT32_MAX ? -1 : best[m];
  }
}

static unsigned grid_for(int64_t n, int threads = 256) {
  int64_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

template <int D, typename P>
static sft_status build_locator_t(sft_source_s* s, int prec, cudaStream_t st, int32_t* d_err) {
  Locator& L = s->loc[prec];
  constexpr int RL = RecLen<D>::value;
  // coordinates in P
  P* xP = nullptr;
  SFT_CUDA(dalloc(&xP, (size_t)s->nv * D, st));
  L.coordsP = xP;
  if (sft_status r = convert_coords(s->coords, s->dtype, xP, prec, s->nv * D, st)) return r;
  // grid box and parameters
  const int32_t n = cells_per_axis(D, s->ne, s->L);
  if (n >= (1 << 22)) return fail(SFT_ERR_UNSUPPORTED, "grid too fine (cells per axis >= 2^22)");
  L.n[0] = L.n[1] = L.n[2] = 1;
  L.ncells = 1;
  for (int a = 0; a < D; ++a) { L.n[a] = n; L.ncells *= n; }
  const unsigned nb = 256;
  P* part = nullptr;
  SFT_CUDA(dalloc(&part, (size_t)nb * 2 * D, st));
  ::sft::note_launch(), k_bbox_partial<D, P><<<nb, 256, 0, st>>>(xP, s->nv, part);
  GridP<P>* g = nullptr;
  SFT_CUDA(dalloc(&g, 1, st));
  L.grid = g;
  ::sft::note_launch(), k_grid_params<D, P><<<1, 32, 0, st>>>(part, nb, n, g, d_err);
  SFT_CUDA(cudaGetLastError());
  dfree(part, st);
  // location records and value copies
  P* recs = nullptr;
  P* vals = nullptr;
  SFT_CUDA(dalloc(&recs, (size_t)s->ne * RL, st));
  SFT_CUDA(dalloc(&vals, (size_t)s->nf * s->ne * 4, st));
  L.recs = recs;
  L.vals = vals;
  // the first locator (the source's own precision, at create) also records
  // every element's FP64 measure for the source integrals
  double* evol = nullptr;
  if (!s->evol) {
    SFT_CUDA(dalloc(&s->evol, (size_t)s->ne, st));
    evol = s->evol;
  }
  if (s->dtype == SFT_F64)
    ::sft::note_launch(), k_records<D, P, double><<<grid_for(s->ne), 256, 0, st>>>(xP, s->conn, (const double*)s->values, s->nv, s->ne,
                                                             s->nf, recs, vals, d_err, evol);
  else
    ::sft::note_launch(), k_records<D, P, float><<<grid_for(s->ne), 256, 0, st>>>(xP, s->conn, (const float*)s->values, s->nv, s->ne,
                                                            s->nf, recs, vals, d_err, evol);
  SFT_CUDA(cudaGetLastError());
  // count registrations per cell, then total (int64) -> int32 offsets must suffice
  // (temporaries freed in stream order on every return)
  DevBuf<int32_t> cell_count(st);
  DevBuf<int64_t> start64(st);
  DevBuf<uint32_t> mask(st);
  DevBuf<RegEntry<P>> reg(st);
  SFT_CUDA(cell_count.alloc((size_t)L.ncells));
  SFT_CUDA(start64.alloc((size_t)L.ncells + 1));
  SFT_CUDA(mask.alloc((size_t)s->ne));
  SFT_CUDA(cudaMemsetAsync(cell_count.p, 0, sizeof(int32_t) * L.ncells, st));
  ::sft::note_launch(), k_register<D, P, false><<<grid_for(s->ne), 256, 0, st>>>(xP, s->conn, recs, s->nv, s->ne, g,
                                                                               cell_count.p, nullptr, nullptr, mask.p);
  SFT_CUDA(cudaGetLastError());
  SFT_CUDA(exclusive_scan_i32_to_i64(cell_count.p, start64.p, L.ncells, st));
  int32_t herr = 0;
  int64_t total = 0;
  SFT_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaMemcpyAsync(&total, start64.p + L.ncells, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  if (herr != 0)
    return fail(SFT_ERR_MESH, herr == DEV_NONFINITE  ? "non-finite source coordinate"
                              : herr == DEV_BAD_INDEX ? "source connectivity index out of range"
                                                      : "source mesh has a non-positive element or a degenerate box");
  if (total >= (int64_t)INT32_MAX) return fail(SFT_ERR_UNSUPPORTED, "grid registrations exceed 2^31");
  L.nitems = total;
  SFT_CUDA(dalloc(&L.cell_start, (size_t)L.ncells + 1, st));
  SFT_CUDA(narrow_i64_to_i32(start64.p, L.cell_start, L.ncells + 1, st));
  // fill (arbitrary order within a cell), then each cell's start element
  SFT_CUDA(reg.alloc((size_t)total));
  SFT_CUDA(dalloc(&L.cell_items, (size_t)total, st));
  SFT_CUDA(cudaMemsetAsync(cell_count.p, 0, sizeof(int32_t) * L.ncells, st));
  ::sft::note_launch(), k_register<D, P, true><<<grid_for(s->ne), 256, 0, st>>>(xP, s->conn, recs, s->nv, s->ne, g,
                                                                              cell_count.p, L.cell_start, reg.p, mask.p);
  SFT_CUDA(cudaGetLastError());
  SFT_CUDA(dalloc(&L.cell_first, (size_t)L.ncells, st));
  ::sft::note_launch(), k_cell_first<P><<<grid_for(L.ncells), 256, 0, st>>>(L.cell_start, reg.p, L.ncells, L.cell_items,
                                                                           L.cell_first);
  SFT_CUDA(cudaGetLastError());
  // face neighbours for the location walk (one array per source mesh)
  if (!s->adj) {
    SFT_CUDA(dalloc(&s->adj, (size_t)s->ne * (D + 1), st));
    ::sft::note_launch(), k_adjacency<D, P><<<grid_for(2 * s->ne), 256, 0, st>>>(xP, s->conn, s->nv, s->ne, g, L.cell_start,
                                                                           L.cell_items, s->adj);
    SFT_CUDA(cudaGetLastError());
  }
  L.adj = s->adj;
  L.built = true;
  return SFT_OK;
}

sft_status build_locator(sft_source_s* s, int prec, cudaStream_t st, int32_t* d_err) {
  if (s->loc[prec].built) return SFT_OK;
  if (s->dim == 2)
    return prec == SFT_PREC_FP32 ? build_locator_t<2, float>(s, prec, st, d_err) : build_locator_t<2, double>(s, prec, st, d_err);
  return prec == SFT_PREC_FP32 ? build_locator_t<3, float>(s, prec, st, d_err) : build_locator_t<3, double>(s, prec, st, d_err);
}

// per-element value copies from the nodal values (after a value update)
template <int D, typename P, typename TV>
__global__ void k_value_copies(const int32_t* __restrict__ conn, const TV* __restrict__ values, int64_t nv,
                               int64_t ne, int nf, P* __restrict__ vals) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[D + 1];
#pragma unroll
    for (int m = 0; m <= D; ++m) v[m] = conn[e * (D + 1) + m];
    for (int f = 0; f < nf; ++f)
#pragma unroll
      for (int m = 0; m < 4; ++m) vals[((int64_t)e * nf + f) * 4 + m] = m <= D ? P(values[(int64_t)f * nv + v[m]]) : P(0);
  }
}

sft_status refresh_value_copies(sft_source_s* s, cudaStream_t st) {
  for (int prec = 0; prec < 2; ++prec) {
    Locator& L = s->loc[prec];
    if (!L.built) continue;
    const unsigned blocks = grid_for(s->ne);
#define SFT_VC(DD, PP, TT)                                                                                  \
  ::sft::note_launch(), k_value_copies<DD, PP, TT><<<blocks, 256, 0, st>>>(s->conn, (const TT*)s->values, s->nv, \
                                                                          s->ne, s->nf, (PP*)L.vals)
    if (s->dim == 2) {
      if (prec == SFT_PREC_FP32) { if (s->dtype == SFT_F64) SFT_VC(2, float, double); else SFT_VC(2, float, float); }
      else { if (s->dtype == SFT_F64) SFT_VC(2, double, double); else SFT_VC(2, double, float); }
    } else {
      if (prec == SFT_PREC_FP32) { if (s->dtype == SFT_F64) SFT_VC(3, float, double); else SFT_VC(3, float, float); }
      else { if (s->dtype == SFT_F64) SFT_VC(3, double, double); else SFT_VC(3, double, float); }
    }
#undef SFT_VC
    SFT_CUDA(cudaGetLastError());
  }
  return SFT_OK;
}

// ---------------------------------------------------------------------------
// point queries: location + P1 evaluation of all fields
// ---------------------------------------------------------------------------
template <int D, typename P, typename TIn, typename TOut>
__global__ void __launch_bounds__(256) k_locate_points(const TIn* __restrict__ pts, int64_t n,
                                                       const GridP<P>* __restrict__ gp,
                                                       const int32_t* __restrict__ cell_start,
                                                       const int32_t* __restrict__ cell_items,
                                                       const int32_t* __restrict__ cell_first,
                                                       const P* __restrict__ recs, const int32_t* __restrict__ adj,
                                                       const P* __restrict__ vals,
                                                       int snf, int nf, int32_t* __restrict__ elem_out,
                                                       TOut* __restrict__ val_out, int64_t val_stride,
                                                       int64_t* __restrict__ counters, P* __restrict__ mu_out) {
  const GridP<P> g = *gp;
  int n_fallback = 0, n_empty = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    P X[D];
#pragma unroll
    for (int a = 0; a < D; ++a) {
      if constexpr (sizeof(P) == 4 && sizeof(TIn) == 8) X[a] = __double2float_rn(pts[i * D + a]);
      else X[a] = (P)pts[i * D + a];
    }
    P mu[D + 1];
    int status;
    const int32_t e = locate_point<D, P>(g, cell_start, cell_items, cell_first, recs, adj, X, mu, status);
    n_fallback += status == 1;
    n_empty += status == 2;
    if (elem_out) elem_out[i] = e;
    if (mu_out) {
#pragma unroll
      for (int a = 0; a < D; ++a) mu_out[a * n + i] = mu[a + 1];
    }
    if (val_out) {
      for (int f = 0; f < nf; ++f)
        val_out[(int64_t)f * val_stride + i] = e >= 0 ? (TOut)eval_p1<D, P>(vals, snf, f, e, mu) : TOut(0);
    }
  }
  if (counters) {
    const int fb = warp_sum<int>(n_fallback), em = warp_sum<int>(n_empty);
    if ((threadIdx.x & 31) == 0) {
      if (fb) atomicAdd(reinterpret_cast<unsigned long long*>(counters), (unsigned long long)fb);
      if (em) atomicAdd(reinterpret_cast<unsigned long long*>(counters + 1), (unsigned long long)em);
    }
  }
}

template <int D, typename P>
static void launch_locate(sft_source_s* s, const Locator& L, int64_t n, const void* pts, int pts_are_double,
                          int32_t* elem_out, void* val_out, int val_is_double, int64_t val_stride,
                          int64_t* counters, cudaStream_t st, int nf, void* mu_out) {
  const unsigned blocks = grid_for(n);
  const GridP<P>* g = (const GridP<P>*)L.grid;
  const P* recs = (const P*)L.recs;
  const P* vals = (const P*)L.vals;
#define SFT_LOC(TIN, TOUT)                                                                                      \
  ::sft::note_launch(), k_locate_points<D, P, TIN, TOUT><<<blocks, 256, 0, st>>>((const TIN*)pts, n, g, L.cell_start, L.cell_items, \
                                                           L.cell_first,                                    \
                                                           recs, L.adj, vals, s->nf, nf, elem_out,          \
                                                           (TOUT*)val_out,                                   \
                                                           val_stride, counters, (P*)mu_out)
  if (pts_are_double) {
    if (val_is_double) SFT_LOC(double, double); else SFT_LOC(double, P);
  } else {
    if (val_is_double) SFT_LOC(P, double); else SFT_LOC(P, P);
  }
#undef SFT_LOC
}

sft_status locate_points(sft_source_s* s, int prec, int64_t n, const void* pts, int pts_are_double,
                         int32_t* elem_out, void* val_out, int val_is_double, int64_t val_stride,
                         int64_t* d_counters, cudaStream_t st, int nf_out, void* mu_out) {
  const Locator& L = s->loc[prec];
  const int nf = nf_out < 0 ? s->nf : nf_out;
  if (!L.built) return fail(SFT_ERR_ARG, "locator not built");
  if (n <= 0) return SFT_OK;
  if (s->dim == 2) {
    if (prec == SFT_PREC_FP32) launch_locate<2, float>(s, L, n, pts, pts_are_double, elem_out, val_out, val_is_double, val_stride, d_counters, st, nf, mu_out);
    else launch_locate<2, double>(s, L, n, pts, pts_are_double, elem_out, val_out, val_is_double, val_stride, d_counters, st, nf, mu_out);
  } else {
    if (prec == SFT_PREC_FP32) launch_locate<3, float>(s, L, n, pts, pts_are_double, elem_out, val_out, val_is_double, val_stride, d_counters, st, nf, mu_out);
    else launch_locate<3, double>(s, L, n, pts, pts_are_double, elem_out, val_out, val_is_double, val_stride, d_counters, st, nf, mu_out);
  }
  SFT_CUDA(cudaGetLastError());
  return SFT_OK;
}

// ---------------------------------------------------------------------------
// exact P1 integral of every source field: sum_e |e| mean(f over vertices)
// ---------------------------------------------------------------------------
template <int D, typename TI>
__global__ void k_p1_integral_partial(const double* __restrict__ evol, const int32_t* __restrict__ conn,
                                      const TI* __restrict__ values, int64_t nv, int64_t ne, int nf,
                                      double* __restrict__ part) {
  double acc[kMaxFields];
  for (int f = 0; f < kMaxFields; ++f) acc[f] = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    int32_t v[D + 1];
#pragma unroll
    for (int m = 0; m <= D; ++m) v[m] = __ldg(conn + e * (D + 1) + m);
    const double vol = __ldg(evol + e);
    // sum |e| (f_0 + ... + f_d); the 1 / (d + 1) is applied once per thread
    for (int f = 0; f < nf; ++f) {
      double m = 0.0;
#pragma unroll
      for (int q = 0; q <= D; ++q) m += f2d(values[(int64_t)f * nv + v[q]]);
      acc[f] = fma(vol, m, acc[f]);
    }
  }
  for (int f = 0; f < nf; ++f) acc[f] *= 1.0 / (D + 1);
  __shared__ double sh[kMaxFields][8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int f = 0; f < nf; ++f) {
    const double w = warp_sum<double>(acc[f]);
    if (lane == 0) sh[f][warp] = w;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int f = 0; f < nf; ++f) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += sh[f][w];
      part[(int64_t)blockIdx.x * kMaxFields + f] = t;
    }
  }
}

sft_status source_integrals_launch(sft_source_s* s, double* part, cudaStream_t st) {
  const unsigned nb = kIntegralBlocks;
  if (!s->evol) return fail(SFT_ERR_ARG, "source has no element measures");
  if (s->dim == 2) {
    if (s->dtype == SFT_F64) ::sft::note_launch(), k_p1_integral_partial<2, double><<<nb, 256, 0, st>>>(s->evol, s->conn, (const double*)s->values, s->nv, s->ne, s->nf, part);
    else ::sft::note_launch(), k_p1_integral_partial<2, float><<<nb, 256, 0, st>>>(s->evol, s->conn, (const float*)s->values, s->nv, s->ne, s->nf, part);
  } else {
    if (s->dtype == SFT_F64) ::sft::note_launch(), k_p1_integral_partial<3, double><<<nb, 256, 0, st>>>(s->evol, s->conn, (const double*)s->values, s->nv, s->ne, s->nf, part);
    else ::sft::note_launch(), k_p1_integral_partial<3, float><<<nb, 256, 0, st>>>(s->evol, s->conn, (const float*)s->values, s->nv, s->ne, s->nf, part);
  }
  SFT_CUDA(cudaGetLastError());
  return SFT_OK;
}

void source_integrals_finish(sft_source_s* s, const double* hpart) {
  for (int f = 0; f < s->nf; ++f) {
    double t = 0.0;
    for (unsigned b = 0; b < kIntegralBlocks; ++b) t += hpart[(size_t)b * kMaxFields + f];
    s->integral[f] = t;
  }
  s->integral_valid = true;
}

sft_status source_integrals(sft_source_s* s, cudaStream_t st) {
  DevBuf<double> part(st);
  SFT_CUDA(part.alloc((size_t)kIntegralBlocks * kMaxFields));
  if (sft_status r = source_integrals_launch(s, part.p, st)) return r;
  std::vector<double> h((size_t)kIntegralBlocks * kMaxFields);
  SFT_CUDA(cudaMemcpyAsync(h.data(), part.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  source_integrals_finish(s, h.data());
  return SFT_OK;
}

}  // namespace sft
