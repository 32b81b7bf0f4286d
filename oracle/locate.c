/*
 * Oracle: point location of the black-box source query (Sec. 4, step 4) in a
 * uniform grid (Sec. 5.3: nx = ny = int(L sqrt(#elements))), and P1
 * evaluation of the source field. TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Reading of the unstated parts:
 *   - cells per axis: the largest n >= 1 with n^d <= L^d * #elements (2D:
 *     int(L sqrt(#elements)) as in the paper; 3D: the cube-root analogue);
 *   - grid box: min/max of the source node coordinates; per-axis scale
 *     inv = n / (max - min) in FP64, rounded once to the path precision P;
 *   - cell of a coordinate x: clamp(floor((x - min) * inv), 0, n - 1) in P.
 *     It is monotone in x, so a point inside an element's bounding box falls
 *     in one of the cells the element is registered in;
 *   - each element is registered in the cells its bounding box overlaps,
 *     except those that one of its face planes separates from it (see
 *     cell_may_hold); a cell lists its elements by decreasing "depth" of the cell centre in
 *     them (min of the centre's barycentric coordinates, computed with the
 *     predicate below), ties by ascending id. The centre of cell i along an
 *     axis is lo + (i + 1/2) h with h = (max - min)/n formed in FP64 and
 *     rounded to P, evaluated as one fused multiply-add in P;
 *   - predicate: barycentric coordinates mu from the element's inverse affine
 *     map, formed in P from the vertex coordinates (one reciprocal of the
 *     determinant; FP32 uses Kahan's 2x2 determinant); mu is evaluated in P
 *     with fused multiply-adds in a fixed order. Accepted when all mu >= 0;
 *   - search: a walk through face neighbours, started at the first element
 *     of the point's cell (the one deepest at the cell centre). At element e
 *     the predicate's mu is evaluated; all mu >= 0 accepts e; otherwise the
 *     walk moves to the element across the face opposite the vertex with the
 *     smallest mu (the first such vertex on ties), the face where the point
 *     lies farthest outside. It gives up at a boundary face (no neighbour)
 *     or after ORC_WALK_STEPS evaluations;
 *   - neighbour across the face of e opposite its local vertex m: the other
 *     element whose vertices include the face's vertices (the smallest id if
 *     several; none on the boundary);
 *   - when the walk gives up, every candidate of the cell is tested and the
 *     one with the largest min(mu) wins (ties to the lowest id): an
 *     accepting one whenever any accepts (status 0), else the nearest
 *     (status 1); the result does not depend on the list's order. An empty
 *     cell yields -1.
 * A point inside exactly one element (the usual case) gets that element
 * whatever the search; the rule only fixes which element wins where the
 * rounded predicate accepts several (points on shared faces).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* predicate evaluations of the walk before the cell's list is scanned */
#define ORC_WALK_STEPS 12

struct orc_grid {
    int prec, dim;
    int32_t n[3];
    double lo[3];      /* grid box minimum (a P value) */
    double inv[3];     /* n / extent rounded to P */
    double h[3];       /* extent / n rounded to P (cell size) */
    int64_t ncells, nitems;
    int64_t* start;
    int32_t* items;
    /* source mesh (coordinates rounded to P) */
    int64_t nv, ne;
    double* coords;
    const int32_t* conn;
    int32_t* adj;      /* [ne][dim+1]: neighbour across the face opposite vertex m, or -1 */
};

static double to_prec(int prec, double x) { return prec == 1 ? (double)(float)x : x; }

static int32_t cells_per_axis(int dim, int64_t ne, double L)
{
    const double target = (dim == 2 ? L * L : L * L * L) * (double)ne;
    double r = dim == 2 ? sqrt(target) : cbrt(target);
    int64_t n = (int64_t)floor(r);
    if (n < 1) n = 1;
    /* exact fix-up of the floating-point root */
    for (;;) {
        double nn = (double)(n + 1);
        double p = dim == 2 ? nn * nn : nn * nn * nn;
        if (p <= target) ++n; else break;
    }
    for (;;) {
        double nn = (double)n;
        double p = dim == 2 ? nn * nn : nn * nn * nn;
        if (n > 1 && p > target) --n; else break;
    }
    return (int32_t)n;
}

static int32_t cell_axis(const orc_grid* g, int a, double x)
{
    double fl;
    if (g->prec == 1) {
        float d = (float)x - (float)g->lo[a];
        float s = d * (float)g->inv[a];
        fl = (double)floorf(s);
    } else {
        double d = x - g->lo[a];
        double s = d * g->inv[a];
        fl = floor(s);
    }
    if (!(fl >= 0.0)) return 0;
    if (fl > (double)(g->n[a] - 1)) return g->n[a] - 1;
    return (int32_t)fl;
}

/* a*d - b*c in FP32 with Kahan's algorithm (one FMA recovers the rounding
 * error of b*c), accurate to a few units in the last place */
static float det2f(float a, float d, float b, float c)
{
    const float w = b * c;
    const float e = fmaf(-b, c, w);
    const float f = fmaf(a, d, -w);
    return f + e;
}

/* The element's inverse affine map in precision P: first vertex x0[dim] and
 * rows R[m][a] (m, a < dim) with mu_{m+1}(X) = R[m] . (X - x0). Formed in P
 * from the edge vectors e_k = x_k - x_0 with one correctly rounded reciprocal
 * of the determinant (FP32: cofactors and determinant by Kahan's 2x2
 * determinant; FP64: plain products). Values are stored as doubles holding
 * P values. */
static void inverse_map(int prec, int dim, const double* coords, const int32_t* conn, int32_t e,
                        double x0[3], double R[3][3])
{
    const int k = dim + 1;
    const double* a = coords + (int64_t)conn[(int64_t)e * k + 0] * dim;
    for (int q = 0; q < dim; ++q) x0[q] = a[q];
    if (dim == 2) {
        const double* b = coords + (int64_t)conn[(int64_t)e * k + 1] * dim;
        const double* c = coords + (int64_t)conn[(int64_t)e * k + 2] * dim;
        if (prec == 1) {
            const float ax = (float)a[0], ay = (float)a[1];
            const float e1x = (float)b[0] - ax, e1y = (float)b[1] - ay;
            const float e2x = (float)c[0] - ax, e2y = (float)c[1] - ay;
            const float inv = 1.0f / det2f(e1x, e2y, e2x, e1y);
            R[0][0] = e2y * inv; R[0][1] = -e2x * inv; R[1][0] = -e1y * inv; R[1][1] = e1x * inv;
        } else {
            const double e1x = b[0] - a[0], e1y = b[1] - a[1];
            const double e2x = c[0] - a[0], e2y = c[1] - a[1];
            const double inv = 1.0 / (e1x * e2y - e2x * e1y);
            R[0][0] = e2y * inv; R[0][1] = -e2x * inv; R[1][0] = -e1y * inv; R[1][1] = e1x * inv;
        }
    } else {
        const double* b = coords + (int64_t)conn[(int64_t)e * k + 1] * dim;
        const double* c = coords + (int64_t)conn[(int64_t)e * k + 2] * dim;
        const double* d = coords + (int64_t)conn[(int64_t)e * k + 3] * dim;
        if (prec == 1) {
            float e1[3], e2[3], e3[3];
            for (int q = 0; q < 3; ++q) {
                e1[q] = (float)b[q] - (float)a[q];
                e2[q] = (float)c[q] - (float)a[q];
                e3[q] = (float)d[q] - (float)a[q];
            }
            /* rows of the inverse Jacobian: (e2 x e3, e3 x e1, e1 x e2) / det */
            const float c23[3] = {det2f(e2[1], e3[2], e2[2], e3[1]), det2f(e2[2], e3[0], e2[0], e3[2]),
                                  det2f(e2[0], e3[1], e2[1], e3[0])};
            const float c31[3] = {det2f(e3[1], e1[2], e3[2], e1[1]), det2f(e3[2], e1[0], e3[0], e1[2]),
                                  det2f(e3[0], e1[1], e3[1], e1[0])};
            const float c12[3] = {det2f(e1[1], e2[2], e1[2], e2[1]), det2f(e1[2], e2[0], e1[0], e2[2]),
                                  det2f(e1[0], e2[1], e1[1], e2[0])};
            const float inv = 1.0f / fmaf(e1[2], c23[2], fmaf(e1[1], c23[1], e1[0] * c23[0]));
            for (int q = 0; q < 3; ++q) {
                R[0][q] = c23[q] * inv; R[1][q] = c31[q] * inv; R[2][q] = c12[q] * inv;
            }
        } else {
            const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
            const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
            const double e3[3] = {d[0] - a[0], d[1] - a[1], d[2] - a[2]};
            const double c23[3] = {e2[1] * e3[2] - e2[2] * e3[1], e2[2] * e3[0] - e2[0] * e3[2],
                                   e2[0] * e3[1] - e2[1] * e3[0]};
            const double c31[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2],
                                   e3[0] * e1[1] - e3[1] * e1[0]};
            const double c12[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                   e1[0] * e2[1] - e1[1] * e2[0]};
            const double inv = 1.0 / ((e1[0] * c23[0] + e1[1] * c23[1]) + e1[2] * c23[2]);
            for (int q = 0; q < 3; ++q) {
                R[0][q] = c23[q] * inv; R[1][q] = c31[q] * inv; R[2][q] = c12[q] * inv;
            }
        }
    }
}

/* barycentric coordinates of X in element e, evaluated in precision P with
 * fused multiply-adds in a fixed order from the inverse map above */
static void predicate_mu(int prec, int dim, const double* coords, const int32_t* conn,
                         int32_t e, const double* X, double* mu)
{
    double x0[3], R[3][3];
    inverse_map(prec, dim, coords, conn, e, x0, R);
    if (prec == 1) {
        float dx[3], m[3];
        for (int q = 0; q < dim; ++q) dx[q] = (float)X[q] - (float)x0[q];
        float s = 1.0f;
        for (int r = 0; r < dim; ++r) {
            float t = (float)R[r][0] * dx[0];
            for (int q = 1; q < dim; ++q) t = fmaf((float)R[r][q], dx[q], t);
            m[r] = t;
            s = s - t;
        }
        mu[0] = s;
        for (int r = 0; r < dim; ++r) mu[r + 1] = m[r];
    } else {
        double dx[3], m[3];
        for (int q = 0; q < dim; ++q) dx[q] = X[q] - x0[q];
        double s = 1.0;
        for (int r = 0; r < dim; ++r) {
            double t = R[r][0] * dx[0];
            for (int q = 1; q < dim; ++q) t = fma(R[r][q], dx[q], t);
            m[r] = t;
            s = s - t;
        }
        mu[0] = s;
        for (int r = 0; r < dim; ++r) mu[r + 1] = m[r];
    }
}

/* Registration test: can the cell box (centre c, half widths w, P values)
 * contain a point of element e? For each barycentric coordinate, which is an
 * affine function, its largest value over the box is its value at the
 * centre plus sum_a |gradient_a| w_a; the element is left out of the cell
 * when that largest value is below -2^-10 for some coordinate (the box lies
 * outside that face plane by a margin far above the rounding of the
 * predicate). Evaluated in P in a fixed order. */
static int cell_may_hold(const orc_grid* g, int32_t e, const double* c, const double* w)
{
    const int dim = g->dim;
    double x0[3], R[3][3];
    inverse_map(g->prec, dim, g->coords, g->conn, e, x0, R);
    if (g->prec == 1) {
        const float eps = 0x1p-10f;
        float d[3], s[3] = {0, 0, 0}, tsum = 0.0f;
        for (int a = 0; a < dim; ++a) d[a] = (float)c[a] - (float)x0[a];
        for (int m = 0; m < dim; ++m) {
            float t = (float)R[m][0] * d[0];
            float sp = fabsf((float)R[m][0]) * (float)w[0];
            for (int a = 1; a < dim; ++a) {
                t = fmaf((float)R[m][a], d[a], t);
                sp = fmaf(fabsf((float)R[m][a]), (float)w[a], sp);
            }
            if (t + sp < -eps) return 0;
            tsum = m == 0 ? t : tsum + t;
            for (int a = 0; a < dim; ++a) s[a] = m == 0 ? (float)R[m][a] : s[a] + (float)R[m][a];
        }
        float S = fabsf(s[0]) * (float)w[0];
        for (int a = 1; a < dim; ++a) S = fmaf(fabsf(s[a]), (float)w[a], S);
        return !((1.0f - tsum) + S < -eps);
    } else {
        const double eps = 0x1p-10;
        double d[3], s[3] = {0, 0, 0}, tsum = 0.0;
        for (int a = 0; a < dim; ++a) d[a] = c[a] - x0[a];
        for (int m = 0; m < dim; ++m) {
            double t = R[m][0] * d[0];
            double sp = fabs(R[m][0]) * w[0];
            for (int a = 1; a < dim; ++a) {
                t = fma(R[m][a], d[a], t);
                sp = fma(fabs(R[m][a]), w[a], sp);
            }
            if (t + sp < -eps) return 0;
            tsum = m == 0 ? t : tsum + t;
            for (int a = 0; a < dim; ++a) s[a] = m == 0 ? R[m][a] : s[a] + R[m][a];
        }
        double S = fabs(s[0]) * w[0];
        for (int a = 1; a < dim; ++a) S = fma(fabs(s[a]), w[a], S);
        return !((1.0 - tsum) + S < -eps);
    }
}

/* the candidate with the largest min(mu), ties to the lowest id; returns
 * status 0 (it accepts), 1 (none accepts: the nearest) or 2 (no candidate) */
static int scan_candidates(int prec, int dim, const double* coords, const int32_t* conn,
                           const int32_t* cand, int64_t ncand, const double* X, int32_t* elem)
{
    int32_t best = -1;
    double best_score = -INFINITY;
    for (int64_t q = 0; q < ncand; ++q) {
        const int32_t e = cand[q];
        double mu[4];
        predicate_mu(prec, dim, coords, conn, e, X, mu);
        double mn = mu[0];
        for (int m = 1; m <= dim; ++m) if (mu[m] < mn) mn = mu[m];
        if (best < 0 || mn > best_score || (mn == best_score && e < best)) { best = e; best_score = mn; }
    }
    *elem = best;
    return best < 0 ? 2 : (best_score >= 0.0 ? 0 : 1);
}

static double* rounded_coords(int prec, int dim, int64_t nv, const double* coords)
{
    double* c = (double*)malloc(sizeof(double) * (size_t)(nv * dim));
    for (int64_t i = 0; i < nv * dim; ++i) c[i] = to_prec(prec, coords[i]);
    return c;
}

/* centre of cell index i along axis a, in P */
static double cell_centre(const orc_grid* g, int a, int32_t i)
{
    if (g->prec == 1) return (double)fmaf((float)i + 0.5f, (float)g->h[a], (float)g->lo[a]);
    return fma((double)i + 0.5, g->h[a], g->lo[a]);
}

/* min barycentric coordinate of point X in element e (the predicate's value) */
static double depth(const orc_grid* g, int32_t e, const double* X)
{
    double mu[4];
    predicate_mu(g->prec, g->dim, g->coords, g->conn, e, X, mu);
    double mn = mu[0];
    for (int m = 1; m <= g->dim; ++m) if (mu[m] < mn) mn = mu[m];
    return mn;
}

/* each cell's list: decreasing depth of the cell centre, ties ascending id
 * (stable insertion sort of the ascending-id list) */
static void order_cells(orc_grid* g)
{
    int64_t cap = 0;
    double* sc = NULL;
    for (int64_t cell = 0; cell < g->ncells; ++cell) {
        const int64_t p0 = g->start[cell], n = g->start[cell + 1] - p0;
        if (n < 2) continue;
        if (n > cap) { cap = n; sc = (double*)realloc(sc, sizeof(double) * (size_t)cap); }
        const int32_t ix = (int32_t)(cell % g->n[0]);
        const int32_t iy = (int32_t)((cell / g->n[0]) % g->n[1]);
        const int32_t iz = (int32_t)(cell / ((int64_t)g->n[0] * g->n[1]));
        const int32_t idx[3] = {ix, iy, iz};
        double X[3] = {0, 0, 0};
        for (int a = 0; a < g->dim; ++a) X[a] = cell_centre(g, a, idx[a]);
        int32_t* it = g->items + p0;
        for (int64_t q = 0; q < n; ++q) sc[q] = depth(g, it[q], X);
        for (int64_t q = 1; q < n; ++q) {
            const double ks = sc[q];
            const int32_t ki = it[q];
            int64_t r = q - 1;
            while (r >= 0 && sc[r] < ks) {  /* ids ascend already: equal depths keep their order */
                sc[r + 1] = sc[r];
                it[r + 1] = it[r];
                --r;
            }
            sc[r + 1] = ks;
            it[r + 1] = ki;
        }
    }
    free(sc);
}

/* does element e2 have every vertex of element e except its local vertex m? */
static int holds_face(int k, const int32_t* conn, int64_t e, int m, int64_t e2)
{
    for (int q = 0; q < k; ++q) {
        if (q == m) continue;
        int found = 0;
        for (int r = 0; r < k; ++r) found |= conn[e2 * k + r] == conn[e * k + q];
        if (!found) return 0;
    }
    return 1;
}

/* face neighbours by their definition: for each element e and local vertex m,
 * the smallest id e2 != e among the elements incident to the face's first
 * vertex that hold every vertex of the face; -1 if there is none */
static int32_t* build_adjacency(int dim, int64_t nv, int64_t ne, const int32_t* conn)
{
    const int k = dim + 1;
    int64_t* first = (int64_t*)calloc((size_t)nv + 1, sizeof(int64_t));
    for (int64_t i = 0; i < ne * k; ++i) first[conn[i] + 1]++;
    for (int64_t v = 0; v < nv; ++v) first[v + 1] += first[v];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nv + 1));
    memcpy(fill, first, sizeof(int64_t) * (size_t)(nv + 1));
    int32_t* inc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ne * k > 0 ? ne * k : 1));
    for (int64_t e = 0; e < ne; ++e)
        for (int m = 0; m < k; ++m) inc[fill[conn[e * k + m]]++] = (int32_t)e;
    int32_t* adj = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ne * k > 0 ? ne * k : 1));
    for (int64_t e = 0; e < ne; ++e)
        for (int m = 0; m < k; ++m) {
            const int32_t v = conn[e * k + (m == 0 ? 1 : 0)];   /* a vertex of the face */
            int32_t best = -1;
            for (int64_t p = first[v]; p < first[v + 1]; ++p) {
                const int32_t e2 = inc[p];
                if (e2 == e || !holds_face(k, conn, e, m, e2)) continue;
                if (best < 0 || e2 < best) best = e2;
            }
            adj[e * k + m] = best;
        }
    free(first); free(fill); free(inc);
    return adj;
}

orc_grid* orc_grid_build(int prec, int dim, int64_t nv, const double* coords,
                         int64_t ne, const int32_t* conn, double grid_scale_L)
{
    orc_grid* g = (orc_grid*)calloc(1, sizeof(orc_grid));
    const int k = dim + 1;
    g->prec = prec; g->dim = dim; g->nv = nv; g->ne = ne; g->conn = conn;
    g->coords = rounded_coords(prec, dim, nv, coords);
    const int32_t n = cells_per_axis(dim, ne, grid_scale_L);
    g->ncells = 1;
    for (int a = 0; a < 3; ++a) g->n[a] = 1;
    for (int a = 0; a < dim; ++a) {
        double lo = INFINITY, hi = -INFINITY;
        for (int64_t i = 0; i < nv; ++i) {
            const double x = g->coords[i * dim + a];
            if (x < lo) lo = x;
            if (x > hi) hi = x;
        }
        g->n[a] = n;
        g->lo[a] = lo;
        g->inv[a] = to_prec(prec, (double)n / (hi - lo));
        g->h[a] = to_prec(prec, (hi - lo) / (double)n);
        g->ncells *= n;
    }
    /* pass 1: count registrations per cell; pass 2: fill in element order */
    int64_t* count = (int64_t*)calloc((size_t)g->ncells + 1, sizeof(int64_t));
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t e = 0; e < ne; ++e) {
            int32_t c0[3] = {0, 0, 0}, c1[3] = {0, 0, 0};
            for (int a = 0; a < dim; ++a) {
                double lo = INFINITY, hi = -INFINITY;
                for (int m = 0; m < k; ++m) {
                    const double x = g->coords[(int64_t)conn[e * k + m] * dim + a];
                    if (x < lo) lo = x;
                    if (x > hi) hi = x;
                }
                c0[a] = cell_axis(g, a, lo);
                c1[a] = cell_axis(g, a, hi);
            }
            for (int32_t iz = c0[2]; iz <= c1[2]; ++iz)
                for (int32_t iy = c0[1]; iy <= c1[1]; ++iy)
                    for (int32_t ix = c0[0]; ix <= c1[0]; ++ix) {
                        const int32_t idx[3] = {ix, iy, iz};
                        double cc[3] = {0, 0, 0}, ww[3] = {0, 0, 0};
                        for (int a = 0; a < dim; ++a) {
                            cc[a] = cell_centre(g, a, idx[a]);
                            ww[a] = 0.5 * g->h[a];
                        }
                        if (!cell_may_hold(g, (int32_t)e, cc, ww)) continue;
                        const int64_t cell = ((int64_t)iz * g->n[1] + iy) * g->n[0] + ix;
                        if (pass == 0) count[cell + 1]++;
                        else g->items[g->start[cell] + count[cell]++] = (int32_t)e;
                    }
        }
        if (pass == 0) {
            g->start = (int64_t*)malloc(sizeof(int64_t) * (size_t)(g->ncells + 1));
            g->start[0] = 0;
            for (int64_t c = 0; c < g->ncells; ++c) g->start[c + 1] = g->start[c] + count[c + 1];
            g->nitems = g->start[g->ncells];
            g->items = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->nitems > 0 ? g->nitems : 1));
            memset(count, 0, sizeof(int64_t) * (size_t)(g->ncells + 1));
        }
    }
    free(count);
    order_cells(g);
    g->adj = build_adjacency(dim, nv, ne, conn);
    return g;
}

void orc_grid_free(orc_grid* g)
{
    if (!g) return;
    free(g->start); free(g->items); free(g->coords); free(g->adj); free(g);
}

void orc_grid_shape(const orc_grid* g, int32_t n_out[3], int64_t* ncells, int64_t* nitems)
{
    for (int a = 0; a < 3; ++a) n_out[a] = g->n[a];
    *ncells = g->ncells;
    *nitems = g->nitems;
}

void orc_grid_csr(const orc_grid* g, int64_t* start, int32_t* items)
{
    memcpy(start, g->start, sizeof(int64_t) * (size_t)(g->ncells + 1));
    memcpy(items, g->items, sizeof(int32_t) * (size_t)g->nitems);
}

void orc_grid_depths(const orc_grid* g, double* out)
{
    for (int64_t cell = 0; cell < g->ncells; ++cell) {
        const int32_t idx[3] = {(int32_t)(cell % g->n[0]), (int32_t)((cell / g->n[0]) % g->n[1]),
                                (int32_t)(cell / ((int64_t)g->n[0] * g->n[1]))};
        double X[3] = {0, 0, 0};
        for (int a = 0; a < g->dim; ++a) X[a] = cell_centre(g, a, idx[a]);
        for (int64_t p = g->start[cell]; p < g->start[cell + 1]; ++p) out[p] = depth(g, g->items[p], X);
    }
}

static int locate_one(const orc_grid* g, const double* Xin, int32_t* elem)
{
    double X[3] = {0, 0, 0};
    for (int a = 0; a < g->dim; ++a) X[a] = to_prec(g->prec, Xin[a]);
    int32_t ci[3] = {0, 0, 0};
    for (int a = 0; a < g->dim; ++a) ci[a] = cell_axis(g, a, X[a]);
    const int64_t cell = ((int64_t)ci[2] * g->n[1] + ci[1]) * g->n[0] + ci[0];
    if (g->start[cell + 1] > g->start[cell]) {
        /* the walk from the element deepest at the cell centre */
        int32_t e = g->items[g->start[cell]];
        for (int s = 0; s < ORC_WALK_STEPS; ++s) {
            double mu[4];
            predicate_mu(g->prec, g->dim, g->coords, g->conn, e, X, mu);
            double mn = mu[0];
            int am = 0;
            for (int m = 1; m <= g->dim; ++m)
                if (mu[m] < mn) { mn = mu[m]; am = m; }
            if (mn >= 0.0) { *elem = e; return 0; }
            const int32_t next = g->adj[(int64_t)e * (g->dim + 1) + am];
            if (next < 0) break;
            e = next;
        }
    }
    return scan_candidates(g->prec, g->dim, g->coords, g->conn, g->items + g->start[cell],
                           g->start[cell + 1] - g->start[cell], X, elem);
}

void orc_grid_adjacency(const orc_grid* g, int32_t* out)
{
    memcpy(out, g->adj, sizeof(int32_t) * (size_t)(g->ne * (g->dim + 1)));
}

void orc_grid_locate(const orc_grid* g, int64_t npts, const double* pts,
                     int32_t* elem_out, int32_t* status_out)
{
    for (int64_t i = 0; i < npts; ++i) {
        int32_t e;
        int st = locate_one(g, pts + i * g->dim, &e);
        elem_out[i] = e;
        if (status_out) status_out[i] = st;
    }
}

void orc_brute_locate(int prec, int dim, int64_t nv, const double* coords, int64_t ne,
                      const int32_t* conn, int64_t npts, const double* pts,
                      int32_t* elem_out, int32_t* status_out)
{
    double* c = rounded_coords(prec, dim, nv, coords);
    int32_t* all = (int32_t*)malloc(sizeof(int32_t) * (size_t)(ne > 0 ? ne : 1));
    for (int64_t e = 0; e < ne; ++e) all[e] = (int32_t)e;
    for (int64_t i = 0; i < npts; ++i) {
        double X[3] = {0, 0, 0};
        for (int a = 0; a < dim; ++a) X[a] = to_prec(prec, pts[i * dim + a]);
        int32_t e;
        int st = scan_candidates(prec, dim, c, conn, all, ne, X, &e);
        elem_out[i] = e;
        if (status_out) status_out[i] = st;
    }
    free(all); free(c);
}

/* P1 evaluation in FP64: barycentric coordinates by Cramer's rule (ratios of
 * signed areas / volumes), then sum_m mu_m f_m. */
void orc_eval_p1(int dim, const double* coords, const int32_t* conn, int nf, int64_t nv,
                 const double* values, int32_t e, const double* X, double* f_out)
{
    const int k = dim + 1;
    const int32_t* v = conn + (int64_t)e * k;
    double mu[4];
    if (dim == 2) {
        const double* a = coords + (int64_t)v[0] * 2;
        const double* b = coords + (int64_t)v[1] * 2;
        const double* c = coords + (int64_t)v[2] * 2;
        const double bax = b[0] - a[0], bay = b[1] - a[1], cax = c[0] - a[0], cay = c[1] - a[1];
        const double pax = X[0] - a[0], pay = X[1] - a[1];
        const double area = bax * cay - cax * bay;
        mu[1] = (pax * cay - cax * pay) / area;
        mu[2] = (bax * pay - pax * bay) / area;
        mu[0] = 1.0 - mu[1] - mu[2];
    } else {
        const double* p[4];
        for (int m = 0; m < 4; ++m) p[m] = coords + (int64_t)v[m] * 3;
        double E[3][3], Q[3];
        for (int q = 0; q < 3; ++q) {
            E[0][q] = p[1][q] - p[0][q];
            E[1][q] = p[2][q] - p[0][q];
            E[2][q] = p[3][q] - p[0][q];
            Q[q] = X[q] - p[0][q];
        }
#define DET3(A, B, C) ((A)[0] * ((B)[1] * (C)[2] - (B)[2] * (C)[1]) \
                     - (A)[1] * ((B)[0] * (C)[2] - (B)[2] * (C)[0]) \
                     + (A)[2] * ((B)[0] * (C)[1] - (B)[1] * (C)[0]))
        const double vol = DET3(E[0], E[1], E[2]);
        mu[1] = DET3(Q, E[1], E[2]) / vol;
        mu[2] = DET3(E[0], Q, E[2]) / vol;
        mu[3] = DET3(E[0], E[1], Q) / vol;
#undef DET3
        mu[0] = 1.0 - mu[1] - mu[2] - mu[3];
    }
    for (int f = 0; f < nf; ++f) {
        double s = 0.0;
        for (int m = 0; m < k; ++m) s += mu[m] * values[(int64_t)f * nv + v[m]];
        f_out[f] = s;
    }
}
