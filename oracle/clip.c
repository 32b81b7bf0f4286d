/*
 * Oracle: brute-force mesh intersection in 2D (Sec. 3, Eq. partition_ts and
 * the intersection-integration procedure), used as the exact judge of the
 * Monte Carlo load vector and of the supermesh L2 error
 * (Eq. relative_L2_error). TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Every (target, source) triangle pair with overlapping bounding boxes is
 * clipped (Sutherland-Hodgman: the source triangle against the three edge
 * half-planes of the target triangle). The convex intersection polygon is
 * split into a fan from its first vertex, and each sub-triangle is integrated
 * with the three-edge-midpoint rule, which is exact for the degree-2
 * integrands used here (a product of two functions linear on the piece).
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>

typedef struct { double x, y; } pt2;

static double cross3(pt2 o, pt2 a, pt2 b)
{
    return (a.x - o.x) * (b.y - o.y) - (a.y - o.y) * (b.x - o.x);
}

/* clip polygon in[0..n) by the half-plane left of edge (p, q); returns count */
static int clip_edge(const pt2* in, int n, pt2 p, pt2 q, pt2* out)
{
    int m = 0;
    for (int i = 0; i < n; ++i) {
        const pt2 a = in[i], b = in[(i + 1) % n];
        const double sa = cross3(p, q, a), sb = cross3(p, q, b);
        if (sa >= 0) out[m++] = a;
        if ((sa >= 0) != (sb >= 0)) {
            const double t = sa / (sa - sb);
            pt2 c = {a.x + t * (b.x - a.x), a.y + t * (b.y - a.y)};
            out[m++] = c;
        }
    }
    return m;
}

static void bary2(const pt2 v[3], pt2 x, double mu[3])
{
    const double area = cross3(v[0], v[1], v[2]);
    mu[1] = cross3(v[0], x, v[2]) / area;
    mu[2] = cross3(v[0], v[1], x) / area;
    mu[0] = 1.0 - mu[1] - mu[2];
}

static void tri_pts(const double* coords, const int32_t* conn, int64_t e, pt2 v[3])
{
    for (int m = 0; m < 3; ++m) {
        v[m].x = coords[(int64_t)conn[e * 3 + m] * 2];
        v[m].y = coords[(int64_t)conn[e * 3 + m] * 2 + 1];
    }
}

typedef struct { double lo[2], hi[2]; } box2;

static box2 tri_box(const pt2 v[3])
{
    box2 b = {{v[0].x, v[0].y}, {v[0].x, v[0].y}};
    for (int m = 1; m < 3; ++m) {
        if (v[m].x < b.lo[0]) b.lo[0] = v[m].x;
        if (v[m].y < b.lo[1]) b.lo[1] = v[m].y;
        if (v[m].x > b.hi[0]) b.hi[0] = v[m].x;
        if (v[m].y > b.hi[1]) b.hi[1] = v[m].y;
    }
    return b;
}

/* visit every sub-triangle of every nonempty intersection; mode 0 accumulates
 * the load vector, mode 1 the L2 error and norm */
static void supermesh_walk(int mode,
                           const double* sc, int64_t nes, const int32_t* sconn, const double* sv,
                           const double* tc, int64_t net, const int32_t* tconn, const double* tv,
                           double* b_out, double* err2, double* norm2)
{
    box2* sb = (box2*)malloc(sizeof(box2) * (size_t)nes);
    for (int64_t s = 0; s < nes; ++s) {
        pt2 v[3];
        tri_pts(sc, sconn, s, v);
        sb[s] = tri_box(v);
    }
    for (int64_t t = 0; t < net; ++t) {
        pt2 tvx[3];
        tri_pts(tc, tconn, t, tvx);
        const box2 tb = tri_box(tvx);
        for (int64_t s = 0; s < nes; ++s) {
            if (sb[s].lo[0] > tb.hi[0] || sb[s].hi[0] < tb.lo[0] ||
                sb[s].lo[1] > tb.hi[1] || sb[s].hi[1] < tb.lo[1]) continue;
            pt2 poly[12], tmp[12];
            tri_pts(sc, sconn, s, poly);
            int n = 3;
            for (int ed = 0; ed < 3 && n > 0; ++ed) {
                n = clip_edge(poly, n, tvx[ed], tvx[(ed + 1) % 3], tmp);
                for (int i = 0; i < n; ++i) poly[i] = tmp[i];
            }
            if (n < 3) continue;
            pt2 svx[3];
            tri_pts(sc, sconn, s, svx);
            for (int i = 1; i + 1 < n; ++i) {       /* fan from the anchor poly[0] */
                const pt2 tri[3] = {poly[0], poly[i], poly[i + 1]};
                const double area = 0.5 * cross3(tri[0], tri[1], tri[2]);
                if (!(area > 0)) continue;
                for (int e = 0; e < 3; ++e) {       /* edge midpoints, weight area/3 */
                    const pt2 mpt = {0.5 * (tri[e].x + tri[(e + 1) % 3].x),
                                     0.5 * (tri[e].y + tri[(e + 1) % 3].y)};
                    double ms[3], mt[3];
                    bary2(svx, mpt, ms);
                    bary2(tvx, mpt, mt);
                    double fs = 0.0;
                    for (int m = 0; m < 3; ++m) fs += ms[m] * sv[sconn[s * 3 + m]];
                    const double w = area / 3.0;
                    if (mode == 0) {
                        for (int m = 0; m < 3; ++m) b_out[tconn[t * 3 + m]] += w * fs * mt[m];
                    } else {
                        double ft = 0.0;
                        for (int m = 0; m < 3; ++m) ft += mt[m] * tv[tconn[t * 3 + m]];
                        *err2 += w * (fs - ft) * (fs - ft);
                        *norm2 += w * fs * fs;
                    }
                }
            }
        }
    }
    free(sb);
}

void orc_mi_load_vector_2d(int64_t nvs, const double* src_coords, int64_t nes,
                           const int32_t* src_conn, const double* src_values,
                           int64_t nvt, const double* tgt_coords, int64_t net,
                           const int32_t* tgt_conn, double* b_out)
{
    (void)nvs;
    for (int64_t i = 0; i < nvt; ++i) b_out[i] = 0.0;
    supermesh_walk(0, src_coords, nes, src_conn, src_values, tgt_coords, net, tgt_conn, NULL,
                   b_out, NULL, NULL);
}

void orc_l2_error_2d(int64_t nvs, const double* src_coords, int64_t nes,
                     const int32_t* src_conn, const double* src_values,
                     int64_t nvt, const double* tgt_coords, int64_t net,
                     const int32_t* tgt_conn, const double* tgt_values,
                     double* err_out, double* norm_out)
{
    (void)nvs; (void)nvt;
    double e2 = 0.0, n2 = 0.0;
    supermesh_walk(1, src_coords, nes, src_conn, src_values, tgt_coords, net, tgt_conn,
                   tgt_values, NULL, &e2, &n2);
    *err_out = sqrt(e2);
    *norm_out = sqrt(n2);
}
