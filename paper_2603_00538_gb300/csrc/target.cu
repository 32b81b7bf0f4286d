// Target side: element measures |T| and the FP64 P1 mass matrix
// M_ki = int psi_k psi_i (Eq. mass_matrix). P1 x P1 is degree 2, so exact
// quadrature gives the closed form |T| (1 + delta_ij) / ((d+1)(d+2)).
//
// CSR build without a global sort: node -> element incidence lists by a
// counting sort (atomics + per-node insertion sort, ascending element id);
// then one thread per row merges the vertices of its incident elements into a
// sorted, de-duplicated column list, summing contributions in ascending
// element order (deterministic values).
#include <vector>
#include "internal.hpp"
#include "util.cuh"

namespace sft {

constexpr int kMaxRow = 64;  // distinct neighbours (incl. self) per node

template <int D, typename TI>
__global__ void k_volumes(const TI* __restrict__ x, const int32_t* __restrict__ conn, int64_t nv, int64_t ne,
                          double* __restrict__ vol, float* __restrict__ vol32, double2* __restrict__ wfac,
                          int32_t* __restrict__ inc_count, int32_t* err) {
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
      vol[e] = 0.0;
      vol32[e] = 0.f;
      continue;
    }
    double xv[D + 1][D];
#pragma unroll
    for (int m = 0; m <= D; ++m)
#pragma unroll
      for (int a = 0; a < D; ++a) xv[m][a] = f2d(x[(int64_t)v[m] * D + a]);
    double w;
    if constexpr (D == 2) {
      w = 0.5 * ((xv[1][0] - xv[0][0]) * (xv[2][1] - xv[0][1]) - (xv[2][0] - xv[0][0]) * (xv[1][1] - xv[0][1]));
    } else {
      double e1[3], e2[3], e3[3];
#pragma unroll
      for (int a = 0; a < 3; ++a) { e1[a] = xv[1][a] - xv[0][a]; e2[a] = xv[2][a] - xv[0][a]; e3[a] = xv[3][a] - xv[0][a]; }
      w = (e1[0] * (e2[1] * e3[2] - e2[2] * e3[1]) - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0]) +
           e1[2] * (e2[0] * e3[1] - e2[1] * e3[0])) * (1.0 / 6.0);
    }
    if (!(w > 0.0) || !isfinite(w)) set_error(err, DEV_BAD_ELEMENT);
    vol[e] = w;
    vol32[e] = __double2float_rn(w);
    // mass-matrix factor |T|/((d+1)(d+2)) and lumped share |T|/(d+1), by
    // the rounded reciprocals (a division costs ~10 operations on this GPU's
    // narrow FP64 pipe; the factors are within one ulp of the quotients)
    constexpr double kMassF = 1.0 / ((D + 1) * (D + 2)), kLumpF = 1.0 / (D + 1);
    wfac[e] = make_double2(w * kMassF, w * kLumpF);
#pragma unroll
    for (int m = 0; m <= D; ++m) atomicAdd(inc_count + v[m], 1);
  }
}

// node -> element incidence, filled in arbitrary order (atomic cursor) with
// the node of every entry, then put in ascending element order by rank
template <int D>
__global__ void k_inc_fill(const int32_t* __restrict__ conn, int64_t ne, int64_t nv,
                           const int32_t* __restrict__ inc_start,
                           int32_t* __restrict__ cursor, int32_t* __restrict__ inc, int32_t* __restrict__ inc_node) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    // elements with an index out of range were not counted (k_volumes) and
    // are skipped here too: the error is reported after the counting pass
    bool ok = true;
#pragma unroll
    for (int m = 0; m <= D; ++m) {
      const int32_t v = conn[e * (D + 1) + m];
      ok = ok && v >= 0 && v < nv;
    }
    if (!ok) continue;
#pragma unroll
    for (int m = 0; m <= D; ++m) {
      const int32_t v = conn[e * (D + 1) + m];
      const int32_t pos = inc_start[v] + atomicAdd(cursor + v, 1);
      inc[pos] = (int32_t)e;
      inc_node[pos] = v;
    }
  }
}

// positions [0, inc_start[nv]) were filled (skipped elements leave the tail unused)
__global__ void k_inc_rank(const int32_t* __restrict__ inc_start, const int32_t* __restrict__ inc,
                           const int32_t* __restrict__ inc_node, int64_t nv, int32_t* __restrict__ out) {
  const int64_t n = inc_start[nv];
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int32_t v = inc_node[p];
    const int32_t p0 = inc_start[v], p1 = inc_start[v + 1];
    const int32_t e = inc[p];
    int32_t rank = 0;
    for (int32_t q = p0; q < p1; ++q) rank += inc[q] < e;
    out[p0 + rank] = e;
  }
}

// Row i of M: FILL=false writes the row length (and, when tmp_col is given,
// the row itself into an entry-major staging array [kMaxRow][nv], so that the second pass
// only copies), FILL=true writes columns, values, the Jacobi inverse diagonal
// and the lumped mass.
// CAP bounds the row buffers (local memory per thread); a counting pass with
// CAP < kMaxRow marks the rows that do not fit (row_len = -1) and a second
// pass with REDO = true and CAP = kMaxRow builds exactly those.
template <int D, bool FILL, int CAP = kMaxRow, bool REDO = false>
__global__ void k_mass_rows(const int32_t* __restrict__ conn, const double2* __restrict__ wfac,
                            const int32_t* __restrict__ inc_start, const int32_t* __restrict__ inc, int64_t nv,
                            int32_t* __restrict__ row_len, const int32_t* __restrict__ row_ptr,
                            int32_t* __restrict__ col, double* __restrict__ val, double* __restrict__ dinv,
                            double* __restrict__ lumped, int32_t* err, int32_t* __restrict__ tmp_col,
                            double* __restrict__ tmp_val, double* __restrict__ tmp_lump) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    if (REDO && row_len[i] >= 0) continue;
    int32_t cols[CAP];
    double vals[CAP];
    int cnt = 0;
    bool overflow = false;
    double lump = 0.0;
    // incident elements in chunks of kPre: their connectivity and factors are
    // loaded first (independent loads in flight together), then merged in
    // incidence order (the same sums as one element at a time)
    constexpr int kPre = 4;
    const int32_t p_end = inc_start[i + 1];
    for (int32_t p0 = inc_start[i]; p0 < p_end; p0 += kPre) {
      int32_t ce[kPre][D + 1];
      double2 wv[kPre];
#pragma unroll
      for (int u = 0; u < kPre; ++u) {
        if (p0 + u < p_end) {
          const int32_t e = __ldg(inc + p0 + u);
          wv[u] = __ldg(wfac + e);
#pragma unroll
          for (int m = 0; m <= D; ++m) ce[u][m] = __ldg(conn + (int64_t)e * (D + 1) + m);
        }
      }
#pragma unroll
      for (int u = 0; u < kPre; ++u) {
      if (p0 + u >= p_end) break;
      const double2 wf = wv[u];
      lump += wf.y;
      // 2 RN(w/den) == RN(2w/den): same values as dividing each entry
      const double wd = wf.x;
#pragma unroll
      for (int m = 0; m <= D; ++m) {
        const int32_t j = ce[u][m];
        const double c = j == i ? 2.0 * wd : wd;
        int q = 0;
        while (q < cnt && cols[q] < j) ++q;
        if (q < cnt && cols[q] == j) {
          vals[q] += c;
        } else if (cnt < CAP) {
          for (int r = cnt; r > q; --r) { cols[r] = cols[r - 1]; vals[r] = vals[r - 1]; }
          cols[q] = j;
          vals[q] = c;
          ++cnt;
        } else {
          overflow = true;
        }
      }
      }
    }
    if (overflow) {
      if (CAP < kMaxRow) {  // this row is built again with the full buffers
        row_len[i] = -1;
        continue;
      }
      set_error(err, DEV_VALENCE);
    }
    if (!FILL) {
      row_len[i] = cnt;
      if (tmp_col) {
        for (int q = 0; q < cnt; ++q) {
          // entry q of every row contiguous ([q][nv]): coalesced across a warp's rows
          tmp_col[(int64_t)q * nv + i] = cols[q];
          tmp_val[(int64_t)q * nv + i] = vals[q];
        }
        tmp_lump[i] = lump;
      }
    } else {
      const int32_t base = row_ptr[i];
      double diag = 0.0;
      for (int q = 0; q < cnt; ++q) {
        col[base + q] = cols[q];
        val[base + q] = vals[q];
        if (cols[q] == i) diag = vals[q];
      }
      dinv[i] = diag > 0.0 ? 1.0 / diag : 0.0;
      lumped[i] = lump;
    }
  }
}

// second pass from the staged rows: copy into the CSR arrays
__global__ void k_mass_copy(const int32_t* __restrict__ tmp_col, const double* __restrict__ tmp_val,
                            const double* __restrict__ tmp_lump, const int32_t* __restrict__ row_ptr, int64_t nv,
                            int32_t* __restrict__ col, double* __restrict__ val, double* __restrict__ dinv,
                            double* __restrict__ lumped) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t base = row_ptr[i], cnt = row_ptr[i + 1] - base;
    double diag = 0.0;
    for (int q = 0; q < cnt; ++q) {
      const int32_t c = tmp_col[(int64_t)q * nv + i];
      const double v = tmp_val[(int64_t)q * nv + i];
      col[base + q] = c;
      val[base + q] = v;
      if (c == i) diag = v;
    }
    dinv[i] = diag > 0.0 ? 1.0 / diag : 0.0;
    lumped[i] = tmp_lump[i];
  }
}

static unsigned blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return (unsigned)b;
}

template <int D>
static sft_status build_target_t(sft_target_s* t, cudaStream_t st, int32_t* d_err) {
  SFT_CUDA(dalloc(&t->vol, (size_t)t->ne, st));
  SFT_CUDA(dalloc(&t->vol32, (size_t)t->ne, st));
  double2* wfac = nullptr;
  SFT_CUDA(dalloc(&wfac, (size_t)t->ne, st));
  int32_t *inc_count = nullptr, *inc_start = nullptr, *inc = nullptr, *row_len = nullptr;
  int64_t* off64 = nullptr;
  SFT_CUDA(dalloc(&inc_count, (size_t)t->nv, st));
  SFT_CUDA(cudaMemsetAsync(inc_count, 0, sizeof(int32_t) * t->nv, st));
  if (t->dtype == SFT_F64)
    ::sft::note_launch(), k_volumes<D, double><<<blocks_for(t->ne), 256, 0, st>>>((const double*)t->coords, t->conn, t->nv, t->ne, t->vol, t->vol32, wfac, inc_count, d_err);
  else
    ::sft::note_launch(), k_volumes<D, float><<<blocks_for(t->ne), 256, 0, st>>>((const float*)t->coords, t->conn, t->nv, t->ne, t->vol, t->vol32, wfac, inc_count, d_err);
  SFT_CUDA(cudaGetLastError());
  int32_t herr = 0;
  // no host check here: every later kernel only follows connectivity of
  // elements whose indices are all in range, and the error flag is read with
  // the row count below
  SFT_CUDA(dalloc(&off64, (size_t)t->nv + 1, st));
  SFT_CUDA(dalloc(&inc_start, (size_t)t->nv + 1, st));
  SFT_CUDA(dalloc(&inc, (size_t)t->ne * (D + 1), st));
  int32_t *inc_raw = nullptr, *inc_node = nullptr;
  SFT_CUDA(dalloc(&inc_raw, (size_t)t->ne * (D + 1), st));
  SFT_CUDA(dalloc(&inc_node, (size_t)t->ne * (D + 1), st));
  SFT_CUDA(exclusive_scan_i32_to_i64(inc_count, off64, t->nv, st));
  SFT_CUDA(narrow_i64_to_i32(off64, inc_start, t->nv + 1, st));
  SFT_CUDA(cudaMemsetAsync(inc_count, 0, sizeof(int32_t) * t->nv, st));
  ::sft::note_launch(), k_inc_fill<D><<<blocks_for(t->ne), 256, 0, st>>>(t->conn, t->ne, t->nv, inc_start, inc_count,
                                                                       inc_raw, inc_node);
  SFT_CUDA(cudaGetLastError());
  ::sft::note_launch(), k_inc_rank<<<blocks_for(t->ne * (D + 1)), 256, 0, st>>>(inc_start, inc_raw, inc_node, t->nv,
                                                                               inc);
  SFT_CUDA(cudaGetLastError());
  dfree(inc_raw, st);
  dfree(inc_node, st);
  row_len = inc_count;  // reuse
  // rows are staged at a fixed stride when that fits comfortably (the
  // second pass then copies instead of merging the incidence lists again)
  DevBuf<int32_t> stage_col(st);
  DevBuf<double> stage_val(st), stage_lump(st);
  int32_t* tmp_col = nullptr;
  double *tmp_val = nullptr, *tmp_lump = nullptr;
  if (t->nv * kMaxRow <= (int64_t)1 << 31) {
    if (stage_col.alloc((size_t)t->nv * kMaxRow) == cudaSuccess &&
        stage_val.alloc((size_t)t->nv * kMaxRow) == cudaSuccess && stage_lump.alloc((size_t)t->nv) == cudaSuccess) {
      tmp_col = stage_col.p;
      tmp_val = stage_val.p;
      tmp_lump = stage_lump.p;
    } else {
      cudaGetLastError();  // no staging: the second pass merges again
    }
  }
  // rows of up to 16 (2D) / 32 (3D) entries in small buffers, the rest again
  // with the full ones (measured: the full-size buffers spill to L2)
  constexpr int kCapSmall = D == 2 ? 16 : 32;
  ::sft::note_launch(), k_mass_rows<D, false, kCapSmall><<<blocks_for(t->nv), 256, 0, st>>>(t->conn, wfac, inc_start, inc, t->nv, row_len, nullptr,
                                                           nullptr, nullptr, nullptr, nullptr, d_err, tmp_col,
                                                           tmp_val, tmp_lump);
  SFT_CUDA(cudaGetLastError());
  ::sft::note_launch(), k_mass_rows<D, false, kMaxRow, true><<<blocks_for(t->nv), 256, 0, st>>>(t->conn, wfac, inc_start, inc, t->nv, row_len, nullptr,
                                                           nullptr, nullptr, nullptr, nullptr, d_err, tmp_col,
                                                           tmp_val, tmp_lump);
  SFT_CUDA(cudaGetLastError());
  SFT_CUDA(exclusive_scan_i32_to_i64(row_len, off64, t->nv, st));
  int64_t nnz = 0;
  SFT_CUDA(cudaMemcpyAsync(&nnz, off64 + t->nv, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  SFT_CUDA(cudaStreamSynchronize(st));
  if (herr || nnz >= (int64_t)INT32_MAX) {
    dfree(off64, st);
    dfree(inc_start, st);
    dfree(inc, st);
    dfree(inc_count, st);
    dfree(wfac, st);
    if (herr == DEV_NONFINITE) return fail(SFT_ERR_MESH, "non-finite target coordinate");
    if (herr == DEV_BAD_INDEX) return fail(SFT_ERR_MESH, "target connectivity index out of range");
    if (herr == DEV_BAD_ELEMENT) return fail(SFT_ERR_MESH, "target mesh has a non-positive element");
    if (herr) return fail(SFT_ERR_MESH, "target node belongs to more elements than supported");
    return fail(SFT_ERR_UNSUPPORTED, "mass matrix nnz exceeds 2^31");
  }
  t->nnz = nnz;
  SFT_CUDA(dalloc(&t->row_ptr, (size_t)t->nv + 1, st));
  SFT_CUDA(narrow_i64_to_i32(off64, t->row_ptr, t->nv + 1, st));
  SFT_CUDA(dalloc(&t->col, (size_t)nnz, st));
  SFT_CUDA(dalloc(&t->val, (size_t)nnz, st));
  SFT_CUDA(dalloc(&t->dinv, (size_t)t->nv, st));
  SFT_CUDA(dalloc(&t->lumped, (size_t)t->nv, st));
  if (tmp_col) {
    ::sft::note_launch(), k_mass_copy<<<blocks_for(t->nv), 256, 0, st>>>(tmp_col, tmp_val, tmp_lump, t->row_ptr, t->nv,
                                                                        t->col, t->val, t->dinv, t->lumped);
  } else {
    ::sft::note_launch(), k_mass_rows<D, true><<<blocks_for(t->nv), 256, 0, st>>>(t->conn, wfac, inc_start, inc, t->nv, nullptr, t->row_ptr,
                                                            t->col, t->val, t->dinv, t->lumped, d_err, nullptr,
                                                            nullptr, nullptr);
  }
  SFT_CUDA(cudaGetLastError());
  dfree(off64, st);
  dfree(inc_start, st);
  dfree(inc, st);
  dfree(inc_count, st);
  dfree(wfac, st);
  return SFT_OK;
}

sft_status build_target(sft_target_s* t, cudaStream_t st, int32_t* d_err) {
  return t->dim == 2 ? build_target_t<2>(t, st, d_err) : build_target_t<3>(t, st, d_err);
}

sft_status target_coordsP(sft_target_s* t, int prec, cudaStream_t st) {
  if (t->coordsP[prec]) return SFT_OK;
  const size_t esz = prec == SFT_PREC_FP32 ? 4 : 8;
  void* p = nullptr;
  SFT_CUDA(pool_alloc(&p, esz * (size_t)(t->nv * t->dim > 0 ? t->nv * t->dim : 1), st));
  t->coordsP[prec] = p;
  return convert_coords(t->coords, t->dtype, p, prec, t->nv * t->dim, st);
}

}  // namespace sft
