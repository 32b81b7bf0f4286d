/*
 * Oracle: mass matrix (Eq. mass_matrix), Jacobi-PCG solve of the Galerkin
 * system (Eq. galerkin_system) and the control-variate Monte Carlo transfer
 * (Sec. 4, steps 1-7; Eqs. cv_element_load_residual_operator and
 * cv_load_expanded). TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Readings: P1 x P1 is a degree-2 polynomial, so the Gaussian quadrature the
 * paper uses for M and for the control term (Sec. 2, Dunavant/Keast rules) is
 * exact and equals the closed form |T| (1 + delta_ij) / ((d+1)(d+2)). The
 * solver is not named in the paper; Jacobi-preconditioned CG from x0 = 0 is
 * used, stopping at ||b - M x||_2 <= tol ||b||_2.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static double element_measure(int dim, const double* coords, const int32_t* v)
{
    if (dim == 2) {
        const double* a = coords + (int64_t)v[0] * 2;
        const double* b = coords + (int64_t)v[1] * 2;
        const double* c = coords + (int64_t)v[2] * 2;
        return 0.5 * ((b[0] - a[0]) * (c[1] - a[1]) - (c[0] - a[0]) * (b[1] - a[1]));
    }
    const double* a = coords + (int64_t)v[0] * 3;
    const double* b = coords + (int64_t)v[1] * 3;
    const double* c = coords + (int64_t)v[2] * 3;
    const double* d = coords + (int64_t)v[3] * 3;
    const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    const double e3[3] = {d[0] - a[0], d[1] - a[1], d[2] - a[2]};
    const double det = e1[0] * (e2[1] * e3[2] - e2[2] * e3[1])
                     - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0])
                     + e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
    return det / 6.0;
}

/* ------------------------------------------------------------------------ */
/* mass matrix                                                               */
/* ------------------------------------------------------------------------ */
typedef struct { int32_t r, c; double v; } triplet;

static int cmp_triplet(const void* pa, const void* pb)
{
    const triplet* a = (const triplet*)pa;
    const triplet* b = (const triplet*)pb;
    if (a->r != b->r) return a->r < b->r ? -1 : 1;
    if (a->c != b->c) return a->c < b->c ? -1 : 1;
    return 0;
}

/* all element contributions M^t_ij = |T| (1 + delta_ij) / ((d+1)(d+2)),
 * sorted by (row, column) */
static triplet* mass_triplets(int dim, const double* coords, int64_t ne,
                              const int32_t* conn, int64_t* nt_out)
{
    const int k = dim + 1;
    const double denom = (double)((dim + 1) * (dim + 2));
    const int64_t nt = ne * k * k;
    triplet* t = (triplet*)malloc(sizeof(triplet) * (size_t)(nt > 0 ? nt : 1));
    int64_t q = 0;
    for (int64_t e = 0; e < ne; ++e) {
        const int32_t* v = conn + e * k;
        const double vol = element_measure(dim, coords, v);
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                t[q].r = v[i]; t[q].c = v[j];
                t[q].v = vol * (i == j ? 2.0 : 1.0) / denom;
                ++q;
            }
    }
    qsort(t, (size_t)nt, sizeof(triplet), cmp_triplet);
    *nt_out = nt;
    return t;
}

int64_t orc_mass_nnz(int dim, int64_t nv, int64_t ne, const int32_t* conn)
{
    (void)nv;
    /* the pattern does not depend on coordinates: use a unit placeholder */
    const int k = dim + 1;
    int64_t nt = ne * k * k;
    triplet* t = (triplet*)malloc(sizeof(triplet) * (size_t)(nt > 0 ? nt : 1));
    int64_t q = 0;
    for (int64_t e = 0; e < ne; ++e)
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                t[q].r = conn[e * k + i]; t[q].c = conn[e * k + j]; t[q].v = 0; ++q;
            }
    qsort(t, (size_t)nt, sizeof(triplet), cmp_triplet);
    int64_t nnz = 0;
    for (int64_t i = 0; i < nt; ++i)
        if (i == 0 || t[i].r != t[i - 1].r || t[i].c != t[i - 1].c) ++nnz;
    free(t);
    return nnz;
}

void orc_mass_csr(int dim, int64_t nv, const double* coords, int64_t ne, const int32_t* conn,
                  int64_t* row_ptr, int32_t* col, double* val)
{
    int64_t nt;
    triplet* t = mass_triplets(dim, coords, ne, conn, &nt);
    for (int64_t i = 0; i <= nv; ++i) row_ptr[i] = 0;
    int64_t nnz = 0;
    for (int64_t i = 0; i < nt; ++i) {
        if (i == 0 || t[i].r != t[i - 1].r || t[i].c != t[i - 1].c) {
            col[nnz] = t[i].c;
            val[nnz] = t[i].v;
            row_ptr[t[i].r + 1]++;
            ++nnz;
        } else {
            val[nnz - 1] += t[i].v;
        }
    }
    for (int64_t i = 0; i < nv; ++i) row_ptr[i + 1] += row_ptr[i];
    free(t);
}

void orc_lumped_mass(int dim, int64_t nv, const double* coords, int64_t ne,
                     const int32_t* conn, double* m_out)
{
    const int k = dim + 1;
    for (int64_t i = 0; i < nv; ++i) m_out[i] = 0.0;
    for (int64_t e = 0; e < ne; ++e) {
        const double vol = element_measure(dim, coords, conn + e * k);
        for (int i = 0; i < k; ++i) m_out[conn[e * k + i]] += vol / (double)k;
    }
}

/* ------------------------------------------------------------------------ */
/* Jacobi-preconditioned conjugate gradients                                 */
/* ------------------------------------------------------------------------ */
static double dot(int64_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
    return s;
}

static void spmv(int64_t n, const int64_t* rp, const int32_t* col, const double* val,
                 const double* x, double* y)
{
    for (int64_t i = 0; i < n; ++i) {
        double s = 0.0;
        for (int64_t q = rp[i]; q < rp[i + 1]; ++q) s += val[q] * x[col[q]];
        y[i] = s;
    }
}

int orc_pcg(int64_t n, const int64_t* rp, const int32_t* col, const double* val,
            const double* b, double* x, double tol, int max_iter, double* rel_resid_out)
{
    double* r = (double*)malloc(sizeof(double) * (size_t)n);
    double* z = (double*)malloc(sizeof(double) * (size_t)n);
    double* p = (double*)malloc(sizeof(double) * (size_t)n);
    double* q = (double*)malloc(sizeof(double) * (size_t)n);
    double* dinv = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) {
        double d = 0.0;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) if (col[k] == i) d = val[k];
        dinv[i] = 1.0 / d;
        x[i] = 0.0;
        r[i] = b[i];
        z[i] = dinv[i] * r[i];
        p[i] = z[i];
    }
    const double bnorm = sqrt(dot(n, b, b));
    double rz = dot(n, r, z);
    double rnorm = bnorm;
    int it = 0;
    if (bnorm == 0.0) {
        *rel_resid_out = 0.0;
        goto done;
    }
    while (it < max_iter && rnorm > tol * bnorm) {
        spmv(n, rp, col, val, p, q);
        const double alpha = rz / dot(n, p, q);
        for (int64_t i = 0; i < n; ++i) { x[i] += alpha * p[i]; r[i] -= alpha * q[i]; }
        rnorm = sqrt(dot(n, r, r));
        ++it;
        for (int64_t i = 0; i < n; ++i) z[i] = dinv[i] * r[i];
        const double rz_new = dot(n, r, z);
        const double beta = rz_new / rz;
        rz = rz_new;
        for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];
    }
    *rel_resid_out = rnorm / bnorm;
done:
    free(r); free(z); free(p); free(q); free(dinv);
    return it;
}

/* ------------------------------------------------------------------------ */
/* the control-variate Monte Carlo transfer                                   */
/* ------------------------------------------------------------------------ */
void orc_transfer(int dim, const orc_params* p,
                  int64_t nvs, const double* src_coords, int64_t nes, const int32_t* src_conn,
                  int nf, const double* src_values,
                  int64_t nvt, const double* tgt_coords, int64_t net, const int32_t* tgt_conn,
                  double* g_out, double* bg_out, double* bres_out, double* b_out, double* u_out,
                  int32_t* sample_elem_out, orc_stats* stats)
{
    const int k = dim + 1;
    const int N = p->samples_per_elem;
    const double alpha = p->alpha;
    memset(stats, 0, sizeof(*stats));

    /* the path reads coordinates and nodal values at its precision */
    double* scoord = (double*)malloc(sizeof(double) * (size_t)(nvs * dim));
    double* svals = (double*)malloc(sizeof(double) * (size_t)(nvs * nf));
    double* tcoord = (double*)malloc(sizeof(double) * (size_t)(nvt * dim));
    for (int64_t i = 0; i < nvs * dim; ++i)
        scoord[i] = p->prec == 1 ? (double)(float)src_coords[i] : src_coords[i];
    for (int64_t i = 0; i < nvs * nf; ++i)
        svals[i] = p->prec == 1 ? (double)(float)src_values[i] : src_values[i];
    for (int64_t i = 0; i < nvt * dim; ++i)
        tcoord[i] = p->prec == 1 ? (double)(float)tgt_coords[i] : tgt_coords[i];

    orc_grid* grid = orc_grid_build(p->prec, dim, nvs, scoord, nes, src_conn, p->grid_scale_L);

    /* Step 1: control g = I_h f^s, the source evaluated at the target nodes */
    for (int64_t i = 0; i < nvt; ++i) {
        int32_t e;
        int32_t st;
        orc_grid_locate(grid, 1, tcoord + i * dim, &e, &st);
        if (st == 1) stats->fallback_queries++;
        double f[64];
        if (e < 0) {
            stats->empty_queries++;
            for (int q = 0; q < nf; ++q) f[q] = 0.0;
        } else {
            orc_eval_p1(dim, scoord, src_conn, nf, nvs, svals, e, tcoord + i * dim, f);
        }
        for (int q = 0; q < nf; ++q) g_out[(int64_t)q * nvt + i] = f[q];
    }

    /* Step 2: deterministic control contribution b_g = sum_t int_t alpha g psi_i,
     * with the exact P1 element mass matrix */
    for (int64_t i = 0; i < nvt * nf; ++i) { bg_out[i] = 0.0; bres_out[i] = 0.0; }
    const double denom = (double)((dim + 1) * (dim + 2));
    for (int64_t t = 0; t < net; ++t) {
        const int32_t* v = tgt_conn + t * k;
        const double vol = element_measure(dim, tgt_coords, v);
        for (int q = 0; q < nf; ++q) {
            const double* g = g_out + (int64_t)q * nvt;
            for (int i = 0; i < k; ++i) {
                double s = 0.0;
                for (int m = 0; m < k; ++m) s += (i == m ? 2.0 : 1.0) * g[v[m]];
                bg_out[(int64_t)q * nvt + v[i]] += alpha * vol * s / denom;
            }
        }
    }

    /* Steps 3-5: per target element, N_t samples (uniform, stratified or
     * importance; N_t = N, or the adaptive count); locate each sample in the
     * source, evaluate f^s and g there, and accumulate the residual estimate
     * |T|/N_t sum_j w_j (f^s - alpha g)(X_j) psi_i(X_j), w_j = 1 / (|T| p_t(X_j)) */
    const int adapt = p->adapt_ref_measure > 0.0;
    const int Nmax = adapt ? 8 * N : N;
    double* lam = (double*)malloc(sizeof(double) * (size_t)(Nmax * k));
    double* X = (double*)malloc(sizeof(double) * (size_t)(Nmax * dim));
    double* w = (double*)malloc(sizeof(double) * (size_t)Nmax);
    double* acc = (double*)malloc(sizeof(double) * (size_t)(nf * k));
    for (int64_t t = 0; t < net; ++t) {
        const int32_t* v = tgt_conn + t * k;
        const double vol = element_measure(dim, tgt_coords, v);
        double xyz[12];
        for (int m = 0; m < k; ++m)
            for (int a = 0; a < dim; ++a) xyz[m * dim + a] = tcoord[(int64_t)v[m] * dim + a];
        const int32_t Nt = adapt ? orc_adaptive_samples(dim, xyz, N, p->adapt_ref_measure) : N;
        stats->samples += Nt;
        orc_sample_element_w(p->prec, dim, p->seed, p->stream, t, Nt, p->sampling, xyz, lam, X, w);
        for (int i = 0; i < nf * k; ++i) acc[i] = 0.0;
        if (sample_elem_out)
            for (int j = Nt; j < Nmax; ++j) sample_elem_out[t * Nmax + j] = -1;
        for (int j = 0; j < Nt; ++j) {
            int32_t e, st;
            orc_grid_locate(grid, 1, X + (int64_t)j * dim, &e, &st);
            if (st == 1) stats->fallback_queries++;
            if (sample_elem_out) sample_elem_out[t * Nmax + j] = e;
            double fs[64];
            if (e < 0) {
                stats->empty_queries++;
                for (int q = 0; q < nf; ++q) fs[q] = 0.0;
            } else {
                orc_eval_p1(dim, scoord, src_conn, nf, nvs, svals, e, X + (int64_t)j * dim, fs);
            }
            const double* lj = lam + (int64_t)j * k;
            for (int q = 0; q < nf; ++q) {
                double gX = 0.0;     /* g is P1 on the target element: sum_m g_m psi_m(X) */
                for (int m = 0; m < k; ++m) gX += g_out[(int64_t)q * nvt + v[m]] * lj[m];
                const double r = fs[q] - alpha * gX;
                for (int i = 0; i < k; ++i) acc[q * k + i] += w[j] * r * lj[i];
            }
        }
        /* Step 6 (residual part): scatter the element-local estimate */
        for (int q = 0; q < nf; ++q)
            for (int i = 0; i < k; ++i)
                bres_out[(int64_t)q * nvt + v[i]] += vol / (double)Nt * acc[q * k + i];
    }
    free(lam); free(X); free(w); free(acc);

    /* Step 6: b = b_g + b_res */
    for (int64_t i = 0; i < nvt * nf; ++i) b_out[i] = bg_out[i] + bres_out[i];

    /* Step 7: solve M u = b (mass matrix from the target coordinates as given) */
    const int64_t nnz = orc_mass_nnz(dim, nvt, net, tgt_conn);
    int64_t* rp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nvt + 1));
    int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)nnz);
    double* val = (double*)malloc(sizeof(double) * (size_t)nnz);
    orc_mass_csr(dim, nvt, tgt_coords, net, tgt_conn, rp, col, val);
    stats->cg_iters = 0;
    stats->cg_rel_resid = 0.0;
    for (int q = 0; q < nf; ++q) {
        double rr;
        int it = orc_pcg(nvt, rp, col, val, b_out + (int64_t)q * nvt, u_out + (int64_t)q * nvt,
                         p->cg_tol, p->cg_max_iter, &rr);
        if (it > stats->cg_iters) stats->cg_iters = it;
        if (rr > stats->cg_rel_resid) stats->cg_rel_resid = rr;
    }
    free(rp); free(col); free(val);
    orc_grid_free(grid);
    free(scoord); free(svals); free(tcoord);
}

double orc_integral_p1(int dim, int64_t nv, const double* coords, int64_t ne,
                       const int32_t* conn, const double* values)
{
    (void)nv;
    const int k = dim + 1;
    double s = 0.0;
    for (int64_t e = 0; e < ne; ++e) {
        const int32_t* v = conn + e * k;
        double mean = 0.0;
        for (int m = 0; m < k; ++m) mean += values[v[m]];
        s += element_measure(dim, coords, v) * mean / (double)k;
    }
    return s;
}
