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
