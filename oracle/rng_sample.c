/*
 * Oracle: random numbers and the sample map (Sec. 4, step 3).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The paper only asks for independent Uniform(0,1) scalars per sample and
 * the area-uniform map of Osada et al. (2002) onto the reference triangle.
 * The reading used here (the paper names no generator):
 *   - generator: Philox4x32-10 of Salmon, Moraes, Dror and Shaw (SC'11),
 *     key = (seed low 32 bits, seed high 32 bits);
 *   - 2D: one Philox call per pair of samples q = j/2, counter
 *     (q, t, stream, 0); sample j takes words 2(j%2) and 2(j%2)+1 as (xi, eta);
 *   - 3D: one call per sample, counter (j, t, stream, 0), words 0, 1, 2;
 *   - FP32 uniform: odd multiples of 2^-24, u = ((x >> 8) | 1) * 2^-24;
 *     FP64 uniform: u = (x + 1/2) * 2^-32. Both are exact and lie in (0, 1).
 *   - 2D map (Osada): s = sqrt(xi), weights (1 - s, s (1 - eta), s eta);
 *   - 3D map (no map in the paper): sort three uniforms v1 <= v2 <= v3 and
 *     take the spacings (v1, v2 - v1, v3 - v2, 1 - v3), which are uniformly
 *     distributed on the simplex (order statistics of uniforms);
 *   - X = sum_m lambda_m x_m, added left to right, one rounding per operation.
 *
 * Stratified sampling (an instance of the general density p_t of Eq.
 * mc_element_integral_operator_general with equal-measure strata; the paper
 * names better sampling schemes as future work): with m the largest integer
 * such that m^d <= N, sample j < m^d replaces each uniform U_a by
 * u_a = (c_a + U_a) / m, where c_a is digit a of j in base m (least
 * significant first), computed in the path's precision with one rounding per
 * operation. Both maps push the uniform measure of the unit square / cube to
 * the uniform measure of the simplex, so the m^d grid cells map to regions of
 * equal measure |T| / m^d and every sample keeps the weight |T| / N: the
 * estimator stays unbiased. Samples j >= m^d keep their plain uniforms.
 *
 * Importance sampling (the general density p_t of Eq.
 * mc_element_integral_operator_general, non-uniform): a defensive mixture of
 * the uniform density and the edge-bubble densities 2-weighted on one edge,
 * p_t = (pi_u + sum_{a<b} pi_e (d+1)(d+2) lambda_a lambda_b) / |T|, with
 * pi_u = 1/4 and pi_e = 1/4 (2D: 3 edges) or 1/8 (3D: 6 edges). The P1
 * interpolation error of a smooth field, which is the control-variate
 * residual f^s - I_h f^s at alpha = 1, is a sum of such edge bubbles, so the
 * density follows it; the uniform quarter bounds the weight 1 / (|T| p_t) by
 * 4. Sample j takes two Philox blocks, counters (j, t, stream, 6) and
 * (j, t, stream, 7) = words a0..a3, b0..b3. The top bits of a0 pick the
 * component with exact probabilities: 2D, c = a0 >> 30, 0 uniform, 1..3 the
 * edges (0,1), (0,2), (1,2); 3D, c = a0 >> 29, 0..1 uniform, 2..7 the edges
 * (0,1), (0,2), (0,3), (1,2), (1,3), (2,3). The uniform component maps the
 * uniforms of a1, a2 (2D, Osada) or a1, a2, a3 (3D, sorted spacings). An edge
 * component (a, b) sorts the d + 2 uniforms of a1, a2, a3, b0 (, b1): the
 * spacings s_1..s_{d+3} of sorted uniforms are Dirichlet(1, ..., 1), so
 * lambda_a = s_1 + s_2, lambda_b = s_3 + s_4 and the remaining vertices, in
 * increasing order, s_5 (, s_6) is Dirichlet with 2 at a and b and 1
 * elsewhere, the density (d+1)(d+2) lambda_a lambda_b / |T|. The estimator
 * weights sample j by w_j = 1 / (|T| p_t(X_j)), so |T|/N sum_j w_j h(X_j) is
 * unbiased for int_T h.
 */
#include "oracle.h"
#include <math.h>

/* One Philox round: two 32x32->64 multiplications with the round constants,
 * the high halves mixed with the other two words and the key. */
static void philox_round(uint32_t c[4], const uint32_t k[2])
{
    const uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c[0];
    const uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c[2];
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {            /* Weyl key schedule between rounds */
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

float orc_u01_f32(uint32_t x)
{
    return (float)((x >> 8) | 1u) * 0x1p-24f;
}

double orc_u01_f64(uint32_t x)
{
    return ((double)x + 0.5) * 0x1p-32;
}

static void draw_words(uint64_t seed, uint32_t c0, int64_t t, uint32_t stream, uint32_t w[4])
{
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    const uint32_t ctr[4] = {c0, (uint32_t)t, stream, 0u};
    orc_philox4x32_10(ctr, key, w);
}

int orc_strata_per_axis(int dim, int32_t nsamp)
{
    int m = 1;
    for (;;) {
        int64_t p = 1;
        for (int a = 0; a < dim; ++a) p *= (int64_t)(m + 1);
        if (p > nsamp) return m;
        ++m;
    }
}

/* cell coordinate of sample j along axis a (base-m digit a of j) */
static int stratum_digit(int32_t j, int m, int a)
{
    int32_t q = j;
    for (int i = 0; i < a; ++i) q /= m;
    return (int)(q % m);
}

void orc_sample_element(int prec, int dim, uint64_t seed, uint32_t stream, int64_t t,
                        int32_t nsamp, const double* node_xyz, double* lam_out, double* X_out)
{
    orc_sample_element_s(prec, dim, seed, stream, t, nsamp, 0, node_xyz, lam_out, X_out);
}

void orc_sample_element_s(int prec, int dim, uint64_t seed, uint32_t stream, int64_t t,
                          int32_t nsamp, int sampling, const double* node_xyz, double* lam_out,
                          double* X_out)
{
    const int k = dim + 1;
    const int m = sampling == 1 ? orc_strata_per_axis(dim, nsamp) : 1;
    int32_t nstrata = 1;
    for (int a = 0; a < dim; ++a) nstrata *= m;
    for (int32_t j = 0; j < nsamp; ++j) {
        uint32_t w[4];
        double lam[4];
        const int strat = sampling == 1 && m > 1 && j < nstrata;
        if (dim == 2) {
            draw_words(seed, (uint32_t)(j >> 1), t, stream, w);
            const uint32_t wx = w[2 * (j & 1)], wy = w[2 * (j & 1) + 1];
            if (prec == 1) {
                float xi = orc_u01_f32(wx), eta = orc_u01_f32(wy);
                if (strat) {
                    xi = ((float)stratum_digit(j, m, 0) + xi) / (float)m;
                    eta = ((float)stratum_digit(j, m, 1) + eta) / (float)m;
                }
                const float s = sqrtf(xi);
                const float l0 = 1.0f - s, l1 = s * (1.0f - eta), l2 = s * eta;
                lam[0] = l0; lam[1] = l1; lam[2] = l2;
            } else {
                double xi = orc_u01_f64(wx), eta = orc_u01_f64(wy);
                if (strat) {
                    xi = ((double)stratum_digit(j, m, 0) + xi) / (double)m;
                    eta = ((double)stratum_digit(j, m, 1) + eta) / (double)m;
                }
                const double s = sqrt(xi);
                lam[0] = 1.0 - s; lam[1] = s * (1.0 - eta); lam[2] = s * eta;
            }
        } else {
            draw_words(seed, (uint32_t)j, t, stream, w);
            if (prec == 1) {
                float v[3] = {orc_u01_f32(w[0]), orc_u01_f32(w[1]), orc_u01_f32(w[2])};
                if (strat)
                    for (int a = 0; a < 3; ++a) v[a] = ((float)stratum_digit(j, m, a) + v[a]) / (float)m;
                /* three-comparator sorting network (0,1), (1,2), (0,1) */
                if (v[1] < v[0]) { float s = v[0]; v[0] = v[1]; v[1] = s; }
                if (v[2] < v[1]) { float s = v[1]; v[1] = v[2]; v[2] = s; }
                if (v[1] < v[0]) { float s = v[0]; v[0] = v[1]; v[1] = s; }
                lam[0] = v[0]; lam[1] = v[1] - v[0]; lam[2] = v[2] - v[1]; lam[3] = 1.0f - v[2];
            } else {
                double v[3] = {orc_u01_f64(w[0]), orc_u01_f64(w[1]), orc_u01_f64(w[2])};
                if (strat)
                    for (int a = 0; a < 3; ++a) v[a] = ((double)stratum_digit(j, m, a) + v[a]) / (double)m;
                if (v[1] < v[0]) { double s = v[0]; v[0] = v[1]; v[1] = s; }
                if (v[2] < v[1]) { double s = v[1]; v[1] = v[2]; v[2] = s; }
                if (v[1] < v[0]) { double s = v[0]; v[0] = v[1]; v[1] = s; }
                lam[0] = v[0]; lam[1] = v[1] - v[0]; lam[2] = v[2] - v[1]; lam[3] = 1.0 - v[2];
            }
        }
        for (int m = 0; m < k; ++m) lam_out[(int64_t)j * k + m] = lam[m];
        for (int a = 0; a < dim; ++a) {
            if (prec == 1) {
                float x = (float)lam[0] * (float)node_xyz[0 * dim + a];
                for (int m = 1; m < k; ++m) x = x + (float)lam[m] * (float)node_xyz[m * dim + a];
                X_out[(int64_t)j * dim + a] = x;
            } else {
                double x = lam[0] * node_xyz[0 * dim + a];
                for (int m = 1; m < k; ++m) x = x + lam[m] * node_xyz[m * dim + a];
                X_out[(int64_t)j * dim + a] = x;
            }
        }
    }
}

/* a few uniforms, sorted (insertion sort) */
static void sort_small(double* v, int n)
{
    for (int i = 1; i < n; ++i) {
        const double x = v[i];
        int r = i - 1;
        while (r >= 0 && v[r] > x) { v[r + 1] = v[r]; --r; }
        v[r + 1] = x;
    }
}

static const int edge_vertices[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const int edge_2d[3][2] = {{0, 1}, {0, 2}, {1, 2}};

double orc_importance_weight(int dim, const double* lam)
{
    double bub = 0.0;
    for (int a = 0; a <= dim; ++a)
        for (int b = a + 1; b <= dim; ++b) bub += lam[a] * lam[b];
    const double tp = dim == 2 ? 0.25 + 3.0 * bub : 0.25 + 2.5 * bub;   /* |T| p_t */
    return 1.0 / tp;
}

void orc_sample_element_w(int prec, int dim, uint64_t seed, uint32_t stream, int64_t t,
                          int32_t nsamp, int sampling, const double* node_xyz, double* lam_out,
                          double* X_out, double* w_out)
{
    const int k = dim + 1;
    if (sampling != 2) {
        orc_sample_element_s(prec, dim, seed, stream, t, nsamp, sampling, node_xyz, lam_out, X_out);
        for (int32_t j = 0; j < nsamp; ++j) w_out[j] = 1.0;
        return;
    }
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int32_t j = 0; j < nsamp; ++j) {
        uint32_t a[4], b[4];
        const uint32_t ca[4] = {(uint32_t)j, (uint32_t)t, stream, 6u};
        const uint32_t cb[4] = {(uint32_t)j, (uint32_t)t, stream, 7u};
        orc_philox4x32_10(ca, key, a);
        orc_philox4x32_10(cb, key, b);
        const uint32_t words[5] = {a[1], a[2], a[3], b[0], b[1]};
        double u[5];
        for (int i = 0; i < 5; ++i) u[i] = prec == 1 ? (double)orc_u01_f32(words[i]) : orc_u01_f64(words[i]);
        const int c = dim == 2 ? (int)(a[0] >> 30) : (int)(a[0] >> 29);
        const int uniform = dim == 2 ? c == 0 : c < 2;
        double lam[4];
        if (uniform) {
            if (dim == 2) {
                if (prec == 1) {
                    const float s = sqrtf((float)u[0]), eta = (float)u[1];
                    lam[0] = 1.0f - s; lam[1] = s * (1.0f - eta); lam[2] = s * eta;
                } else {
                    const double s = sqrt(u[0]);
                    lam[0] = 1.0 - s; lam[1] = s * (1.0 - u[1]); lam[2] = s * u[1];
                }
            } else {
                double v[3] = {u[0], u[1], u[2]};
                sort_small(v, 3);
                if (prec == 1) {
                    lam[0] = (float)v[0]; lam[1] = (float)v[1] - (float)v[0];
                    lam[2] = (float)v[2] - (float)v[1]; lam[3] = 1.0f - (float)v[2];
                } else {
                    lam[0] = v[0]; lam[1] = v[1] - v[0]; lam[2] = v[2] - v[1]; lam[3] = 1.0 - v[2];
                }
            }
        } else {
            /* edge (ea, eb): Dirichlet with 2 at ea and eb, 1 at the others */
            const int* e = dim == 2 ? edge_2d[c - 1] : edge_vertices[c - 2];
            const int nu = dim + 2;
            double v[5];
            for (int i = 0; i < nu; ++i) v[i] = u[i];
            sort_small(v, nu);
            double sp[6];                          /* the d + 3 spacings, in P */
            if (prec == 1) {
                sp[0] = (float)v[0];
                for (int i = 1; i < nu; ++i) sp[i] = (float)v[i] - (float)v[i - 1];
                sp[nu] = 1.0f - (float)v[nu - 1];
                lam[e[0]] = (float)sp[0] + (float)sp[1];
                lam[e[1]] = (float)sp[2] + (float)sp[3];
            } else {
                sp[0] = v[0];
                for (int i = 1; i < nu; ++i) sp[i] = v[i] - v[i - 1];
                sp[nu] = 1.0 - v[nu - 1];
                lam[e[0]] = sp[0] + sp[1];
                lam[e[1]] = sp[2] + sp[3];
            }
            int q = 4;
            for (int m = 0; m < k; ++m)
                if (m != e[0] && m != e[1]) lam[m] = sp[q++];
        }
        for (int m = 0; m < k; ++m) lam_out[(int64_t)j * k + m] = lam[m];
        w_out[j] = orc_importance_weight(dim, lam);
        for (int a_ = 0; a_ < dim; ++a_) {
            if (prec == 1) {
                float x = (float)lam[0] * (float)node_xyz[0 * dim + a_];
                for (int m = 1; m < k; ++m) x = x + (float)lam[m] * (float)node_xyz[m * dim + a_];
                X_out[(int64_t)j * dim + a_] = x;
            } else {
                double x = lam[0] * node_xyz[0 * dim + a_];
                for (int m = 1; m < k; ++m) x = x + lam[m] * node_xyz[m * dim + a_];
                X_out[(int64_t)j * dim + a_] = x;
            }
        }
    }
}

int32_t orc_adaptive_samples(int dim, const double* node_xyz, int32_t nsamp, double ref_measure)
{
    /* d! |T| as the edge determinant, evaluated left to right */
    double det;
    if (dim == 2) {
        const double* a = node_xyz; const double* b = node_xyz + 2; const double* c = node_xyz + 4;
        det = (b[0] - a[0]) * (c[1] - a[1]) - (c[0] - a[0]) * (b[1] - a[1]);
    } else {
        const double* a = node_xyz; const double* b = node_xyz + 3;
        const double* c = node_xyz + 6; const double* d = node_xyz + 9;
        const double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        const double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        const double e3[3] = {d[0] - a[0], d[1] - a[1], d[2] - a[2]};
        det = e1[0] * (e2[1] * e3[2] - e2[2] * e3[1])
            - e1[1] * (e2[0] * e3[2] - e2[2] * e3[0])
            + e1[2] * (e2[0] * e3[1] - e2[1] * e3[0]);
    }
    const double dref = ref_measure * (dim == 2 ? 2.0 : 6.0);
    const double q = ceil((double)nsamp * det / dref);
    const double cap = 8.0 * (double)nsamp;
    return (int32_t)(q < 1.0 ? 1.0 : (q > cap ? cap : q));
}
