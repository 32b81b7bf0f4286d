"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics
(closed forms, invariants, textbook special cases, brute force), not against
the oracle itself. CPU only."""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_two_tri():
    rows = {}
    with open(os.path.join(GOLDEN, "two_triangle_square.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            rows[key] = [float(v) for v in vals]
    coords = np.array(rows["nodes"]).reshape(-1, 2)
    conn = np.array(rows["tris"], dtype=np.int32).reshape(-1, 3)
    return coords, conn, rows


# --------------------------------------------------------------------------
# random numbers
# --------------------------------------------------------------------------
def _philox_block(orc, n, key=(0x1234, 0xABCD), word2=7):
    out = np.zeros((n, 4), np.uint32)
    for i in range(n):
        out[i] = orc.philox4x32_10([i, i >> 3, word2, 0], key)
    return out


def test_philox_uniform_bytes_chi2(orc):
    w = _philox_block(orc, 4096)
    byts = w.view(np.uint8).ravel()
    cnt = np.bincount(byts, minlength=256)
    exp = byts.size / 256
    chi2 = ((cnt - exp) ** 2 / exp).sum()
    # chi2 with 255 dof: mean 255, sd 22.6; 6 sd bounds
    assert 255 - 6 * 22.6 < chi2 < 255 + 6 * 22.6


def test_philox_avalanche(orc):
    """Flipping any single counter or key bit flips each output bit with
    probability 1/2 (a reduced-round or mis-wired Philox fails this)."""
    rng = np.random.default_rng(0)
    trials = 48
    worst = 0.0
    for bit in list(range(0, 128, 5)) + [127]:
        flips = np.zeros(128)
        for _ in range(trials):
            ctr = rng.integers(0, 2 ** 32, 4, dtype=np.uint64).astype(np.uint32)
            key = rng.integers(0, 2 ** 32, 2, dtype=np.uint64).astype(np.uint32)
            a = orc.philox4x32_10(ctr, key)
            c2 = ctr.copy()
            c2[bit // 32] ^= np.uint32(1 << (bit % 32))
            b = orc.philox4x32_10(c2, key)
            x = np.bitwise_xor(a, b)
            flips += np.unpackbits(x.view(np.uint8))
        frac = flips.sum() / (128 * trials)
        worst = max(worst, abs(frac - 0.5))
    assert worst < 0.03


def test_philox_distinct_counters_distinct_outputs(orc):
    w = _philox_block(orc, 20000)
    keys = set(map(bytes, w))
    assert len(keys) == w.shape[0]


def test_uniform_conversion_exact_open_interval(orc):
    for x in [0, 1, 255, 256, 2 ** 31, 2 ** 32 - 1]:
        u32 = orc.u01(x, 1)
        u64 = orc.u01(x, 0)
        assert 0.0 < u32 < 1.0 and 0.0 < u64 < 1.0
        assert u32 == ((x >> 8) | 1) / 2 ** 24
        assert u64 == (x + 0.5) / 2 ** 32


# --------------------------------------------------------------------------
# sample map (Sec. 4 step 3; Osada et al. 2002 in 2D, simplex spacings in 3D)
# --------------------------------------------------------------------------
REF = {2: np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]]),
       3: np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])}


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_sample_moments_and_uniformity(orc, dim, prec):
    """E[lambda_i] = 1/(d+1), E[lambda_i lambda_j] = (1+delta_ij)/((d+1)(d+2))
    (Dirichlet(1,...,1) moments of the uniform law on the simplex); the 2^d
    congruent sub-simplices of a midpoint split (corners: lambda_m >= 1/2)
    each receive probability 1/2^d."""
    k = dim + 1
    lam_all = []
    for t in range(200):
        lam, X = orc.sample_element(prec, dim, 11, 0, t, 512, REF[dim])
        lam_all.append(lam)
        assert np.all(lam >= 0.0)
        assert np.allclose(lam.sum(1), 1.0, atol=1e-6 if prec else 1e-15)
        assert np.allclose(X, lam @ REF[dim], atol=1e-6 if prec else 1e-15)
    lam = np.concatenate(lam_all)
    n = lam.shape[0]
    m1 = lam.mean(0)
    sd1 = math.sqrt(dim / ((dim + 1) ** 2 * (dim + 2)) / n)
    assert np.all(np.abs(m1 - 1 / k) < 6 * sd1)
    second = lam.T @ lam / n
    expect = (np.ones((k, k)) + np.eye(k)) / (k * (k + 1))
    assert np.all(np.abs(second - expect) < 6 * 0.3 / math.sqrt(n))
    corner = [(lam[:, m] >= 0.5).mean() for m in range(k)]
    p = 1.0 / 2 ** dim
    for c in corner:
        assert abs(c - p) < 6 * math.sqrt(p * (1 - p) / n)


def test_sample_map_osada_formula(orc):
    """Hand check of the 2D map for one Philox draw: (xi, eta) -> (1-s, s(1-eta), s eta)."""
    w = orc.philox4x32_10([0, 5, 3, 0], [9, 0])
    lam, X = orc.sample_element(0, 2, 9, 3, 5, 2, REF[2])
    xi0, eta0 = (w[0] + 0.5) / 2 ** 32, (w[1] + 0.5) / 2 ** 32
    xi1, eta1 = (w[2] + 0.5) / 2 ** 32, (w[3] + 0.5) / 2 ** 32
    for j, (xi, eta) in enumerate([(xi0, eta0), (xi1, eta1)]):
        s = math.sqrt(xi)
        assert np.allclose(lam[j], [1 - s, s * (1 - eta), s * eta], rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim,N", [(2, 1), (2, 16), (2, 23), (3, 8), (3, 30), (3, 64)])
@pytest.mark.parametrize("prec", [0, 1])
def test_stratified_samples_lie_in_their_strata(orc, dim, prec, N):
    """Stratified sampling: m = largest integer with m^d <= N strata per axis;
    sample j < m^d has the uniform of axis a in [c_a/m, (c_a+1)/m], c_a the
    base-m digit a of j. The uniforms are recovered from the weights by
    inverting the maps (2D: xi = (1 - lam0)^2, eta = lam2 / (1 - lam0); 3D:
    the sorted uniforms are the partial sums of the weights, and sorting
    keeps the i-th smallest uniform in the i-th smallest cell interval).
    Samples j >= m^d are the uniform scheme's, bit for bit."""
    m = orc.strata_per_axis(dim, N)
    assert m ** dim <= N < (m + 1) ** dim
    tol = 1e-6 if prec else 1e-12
    for t in range(40):
        lam, X = orc.sample_element(prec, dim, 5, 2, t, N, REF[dim], sampling=1)
        lam_u, X_u = orc.sample_element(prec, dim, 5, 2, t, N, REF[dim], sampling=0)
        assert np.all(lam >= 0.0) and np.allclose(lam.sum(1), 1.0, atol=tol)
        S = m ** dim
        assert np.array_equal(lam[S:], lam_u[S:]) and np.array_equal(X[S:], X_u[S:])
        for j in range(S):
            c = [(j // m ** a) % m for a in range(dim)]
            if dim == 2:
                sq = 1.0 - lam[j, 0]
                u = [sq * sq, lam[j, 2] / sq if sq > 0 else 0.0]
            else:
                u = sorted(np.cumsum(lam[j, :3]))
                c = sorted(c)
            for a in range(dim):
                assert c[a] / m - tol <= u[a] <= (c[a] + 1) / m + tol, (t, j, a, u[a], c[a])


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("sampling", [0, 1])
def test_sampling_unbiased_for_dirichlet_moments(orc, dim, sampling):
    """Both sampling schemes are unbiased element quadratures: the mean over
    seeds of |T|/N sum_j lam_1(X_j)^2 lam_0(X_j) approaches the closed form
    int_T lam_1^2 lam_0 = d! |T| 2! 1! / (3 + d)! (Dirichlet moments of the
    barycentric coordinates), within 5 standard errors; stratification
    lowers the spread of the estimate."""
    vol = 0.5 if dim == 2 else 1.0 / 6.0
    exact = math.factorial(dim) * vol * 2 / math.factorial(3 + dim)
    N = 16 if dim == 2 else 27
    est = []
    for t in range(400):
        lam, _ = orc.sample_element(0, dim, 7, 1, t, N, REF[dim], sampling=sampling)
        est.append(vol / N * np.sum(lam[:, 1] ** 2 * lam[:, 0]))
    est = np.array(est)
    se = est.std(ddof=1) / math.sqrt(est.size)
    assert abs(est.mean() - exact) < 5 * se
    if sampling == 1:
        unif = []
        for t in range(400):
            lam, _ = orc.sample_element(0, dim, 7, 1, t, N, REF[dim], sampling=0)
            unif.append(vol / N * np.sum(lam[:, 1] ** 2 * lam[:, 0]))
        assert est.std() < 0.7 * np.std(unif)


def test_stratified_strata_cover_each_cell_once(orc):
    """With N = m^2 every cell of the m x m grid of (xi, eta) holds exactly one
    sample of each element (a permutation check of the recovered cells)."""
    N, m = 36, 6
    for t in range(20):
        lam, _ = orc.sample_element(0, 2, 1, 0, t, N, REF[2], sampling=1)
        sq = 1.0 - lam[:, 0]
        cells = np.floor(sq * sq * m).astype(int) + m * np.floor(lam[:, 2] / sq * m).astype(int)
        assert sorted(cells.tolist()) == list(range(N))


def test_stratified_unbiased_and_faster_than_uniform(orc):
    """Stratified sampling stays unbiased (the mean over seeds approaches the
    exact mesh-intersection load vector) and its RMS error decays faster than
    the uniform N^{-1/2}: one Lipschitz integrand sample per stratum of
    diameter O(N^{-1/2}) gives variance O(N^{-2}) in 2D, slope -1."""
    s, t = _pair(2, ns=5)
    s = W.with_values(s, [W.field_sincos])
    b_mi = orc.mi_load_vector_2d(s, t)
    bs = np.stack([orc.transfer(s, t, 0, 9, seed=sd, alpha=0.0, cg_max_iter=1, sampling=1)["b"][0]
                   for sd in range(300)])
    mean, se = bs.mean(0), bs.std(0, ddof=1) / math.sqrt(bs.shape[0])
    se = np.sqrt(se ** 2 + (1e-13 * np.abs(b_mi).max()) ** 2)
    z = (mean - b_mi) / se
    assert np.abs(z).max() < 5.0
    assert abs(z.mean()) < 5.0 / math.sqrt(z.size)
    Ns = [4, 16, 64, 256]
    rms = {0: [], 1: []}
    for sampling in (0, 1):
        for N in Ns:
            errs = [np.linalg.norm(orc.transfer(s, t, 0, N, seed=sd, alpha=0.0, cg_max_iter=1,
                                                sampling=sampling)["b"][0] - b_mi) for sd in range(30)]
            rms[sampling].append(math.sqrt(np.mean(np.square(errs))))
    slope = np.polyfit(np.log(Ns), np.log(rms[1]), 1)[0]
    assert slope < -0.8, slope
    assert all(r1 < r0 for r0, r1 in zip(rms[0], rms[1]))


@pytest.mark.parametrize("dim,prec", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_importance_density_closed_forms(orc, dim, prec):
    """Importance sampling (Eq. mc_element_integral_operator_general with the
    mixture p_t = (pi_u + sum_{a<b} pi_e (d+1)(d+2) lambda_a lambda_b) / |T|):
    every sample lies in the element, the weights lie in (0, 4], and the
    weighted sample means E_p[w h] equal the plain averages int_T h / |T| of
    closed forms: h = 1 (the normalisation, which a wrong constant or
    component probability breaks), h = lambda_i lambda_j ((1 + delta_ij) /
    ((d+1)(d+2))) and h = prod lambda (d! / (2d+1)!), within 4 standard
    errors."""
    k = dim + 1
    xyz = np.vstack([np.zeros(dim), np.eye(dim)]) * 0.7 + 0.1        # a scaled reference simplex
    n = 200_000
    lam, X, w = orc.sample_element_w(prec, dim, 3, 1, 5, n, xyz, sampling=2)
    assert (lam >= 0).all()
    assert np.abs(lam.sum(1) - 1).max() <= (4e-7 if prec else 1e-15)
    assert np.allclose(X, lam @ xyz, atol=1e-6 if prec else 1e-15)
    assert np.all((w > 0) & (w <= 4.0))

    def check(vals, exact):
        m, se = vals.mean(), vals.std(ddof=1) / math.sqrt(vals.size)
        assert abs(m - exact) <= 4 * se + 1e-12, (m, exact, se)
    check(w, 1.0)
    for i in range(k):
        for j in range(i, k):
            check(w * lam[:, i] * lam[:, j], (2.0 if i == j else 1.0) / ((dim + 1) * (dim + 2)))
    check(w * np.prod(lam, axis=1), math.factorial(dim) / math.factorial(2 * dim + 1))
    assert orc.importance_weight(dim, lam[0]) == w[0]


@pytest.mark.parametrize("dim", [2, 3])
def test_importance_lowers_the_variance_of_a_bubble_residual(orc, dim):
    """The control-variate residual of a smooth field at alpha = 1 is the P1
    interpolation error, a sum of edge bubbles; for the isotropic one
    (sum_{a<b} lambda_a lambda_b) the weighted integrands w r psi_i have a
    smaller variance under p_t than r psi_i under uniform sampling, for every
    basis function: by 8 % in 2D, by 1 % only in 3D, where these integrands
    spread almost evenly over the tetrahedron (2,000,000 samples each, so the
    ratio is known to about 0.2 %)."""
    xyz = np.vstack([np.zeros(dim), np.eye(dim)])
    n = 2_000_000
    lam_u, _, _ = orc.sample_element_w(0, dim, 11, 0, 0, n, xyz, sampling=0)
    lam_p, _, w = orc.sample_element_w(0, dim, 11, 0, 0, n, xyz, sampling=2)

    def bubble(lam):
        return sum(lam[:, a] * lam[:, b] for a in range(dim + 1) for b in range(a + 1, dim + 1))
    for i in range(dim + 1):
        hu = bubble(lam_u) * lam_u[:, i]
        hp = w * bubble(lam_p) * lam_p[:, i]
        assert abs(hu.mean() - hp.mean()) <= 4 * hp.std() / math.sqrt(n)
        assert hp.var() < (0.95 if dim == 2 else 0.998) * hu.var(), (i, hp.var() / hu.var())


def test_importance_unbiased_against_mesh_intersection(orc):
    """The importance-sampled estimate stays unbiased against the exact
    mesh-intersection load vector: the mean over 300 seeds lies within 5
    standard errors, at alpha = 0 and alpha = 1."""
    s, t = _pair(2, ns=5)
    s = W.with_values(s, [W.field_sincos])
    b_mi = orc.mi_load_vector_2d(s, t)
    for alpha in (0.0, 1.0):
        bs = np.stack([orc.transfer(s, t, 0, 8, seed=sd, alpha=alpha, cg_max_iter=1, sampling=2)["b"][0]
                       for sd in range(300)])
        mean, se = bs.mean(0), bs.std(0, ddof=1) / math.sqrt(bs.shape[0])
        se = np.sqrt(se ** 2 + (1e-13 * np.abs(b_mi).max()) ** 2)
        z = (mean - b_mi) / se
        assert np.abs(z).max() < 5.0
        assert abs(z.mean()) < 5.0 / math.sqrt(z.size)


def test_adaptive_counts(orc):
    """Per-element sample counts N_t = min(8N, max(1, ceil(N |T| / A_ref))):
    equal elements with A_ref just above their measure get N each; on a
    graded mesh the counts follow the measures, so the total is N |Omega| /
    A_ref up to one sample per element; the cap and the floor hold."""
    m = W.jittered_tri_mesh(6, 0, jitter=0.0)                      # equal right triangles
    area = 0.5 / 36
    for e in range(m.nelems):
        assert orc.adaptive_samples(2, m.coords[m.conn[e]], 12, area * (1 + 1e-9)) == 12
    g = W.jittered_tri_mesh(8, 1)
    g = W.Mesh(g.coords ** 2, g.conn, None)                         # graded towards the origin
    meas = W._signed_measure(g.coords, g.conn)
    ref = meas.sum() / g.nelems
    counts = np.array([orc.adaptive_samples(2, g.coords[g.conn[e]], 10, ref) for e in range(g.nelems)])
    assert counts.min() >= 1 and counts.max() <= 80
    assert np.all(np.diff(counts[np.argsort(meas)]) >= 0)            # monotone in the measure
    assert 10 * g.nelems <= counts.sum() <= 10 * g.nelems + g.nelems
    kuhn = W.jittered_kuhn_mesh(2, 0, jitter=0.0)
    vol = 1.0 / (6 * 8)
    assert orc.adaptive_samples(3, kuhn.coords[kuhn.conn[0]], 5, vol * (1 + 1e-9)) == 5
    assert orc.adaptive_samples(3, kuhn.coords[kuhn.conn[0]], 5, vol / 100) == 40   # the cap, 8 N
    assert orc.adaptive_samples(3, kuhn.coords[kuhn.conn[0]], 5, vol * 100) == 1    # the floor


def test_adaptive_counts_unbiased_and_steadier_conservation_sum(orc):
    """With per-element counts the estimate stays unbiased against mesh
    intersection, and on a graded target (element measures spanning two
    orders of magnitude) the total sum_i b_i, an estimate of int f^s, spreads
    less over seeds than with the same total number of samples spread evenly
    (alpha = 0: the residual is f itself, whose spread over an element grows
    with its size, so the large elements need the samples)."""
    s = W.with_values(W.jittered_tri_mesh(12, 3), [W.field_sincos])
    t = W.delaunay_tri_mesh(60, 5, 4)
    t = W.Mesh(t.coords ** 2, t.conn, None)
    W._fix_orientation(t)
    meas = W._signed_measure(t.coords, t.conn)
    assert meas.max() / meas.min() > 100
    ref = meas.sum() / t.nelems
    b_mi = orc.mi_load_vector_2d(s, t)
    N = 6
    runs = [orc.transfer(s, t, 0, N, seed=sd, alpha=0.0, cg_max_iter=1, adapt_ref_measure=ref)
            for sd in range(200)]
    bs = np.stack([r["b"][0] for r in runs])
    total = runs[0]["samples"]
    assert all(r["samples"] == total for r in runs)
    mean, se = bs.mean(0), bs.std(0, ddof=1) / math.sqrt(bs.shape[0])
    se = np.sqrt(se ** 2 + (1e-13 * np.abs(b_mi).max()) ** 2)
    z = (mean - b_mi) / se
    assert np.abs(z).max() < 5.0
    # the same budget without adaptation: N' per element with N' E >= total
    Nu = -(-total // t.nelems)
    sums_u = [orc.transfer(s, t, 0, Nu, seed=sd, alpha=0.0, cg_max_iter=1)["b"][0].sum() for sd in range(200)]
    assert bs.sum(1).std() < 0.8 * np.std(sums_u)


# --------------------------------------------------------------------------
# point location
# --------------------------------------------------------------------------
def test_golden_two_triangle_locate_eval_mass(orc):
    coords, conn, rows = _golden_two_tri()
    loc = np.array(rows["locate"]).reshape(-1, 3)
    for prec in (0, 1):
        g = orc.Grid(prec, coords, conn)
        e, st = g.locate(loc[:, :2])
        assert list(e) == [int(v) for v in loc[:, 2]]
        assert np.all(st == 0)
    vals = np.array([[0.0, 1.0, 3.0, 2.0]])
    ex, ey, fexp = rows["eval"]
    assert orc.eval_p1(coords, conn, vals, 0, [ex, ey])[0] == pytest.approx(fexp, abs=1e-15)
    rp, col, val = orc.mass_csr(coords, conn)
    dense = np.zeros((4, 4))
    for i in range(4):
        dense[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    assert np.allclose(dense * 24, np.array(rows["M24"]).reshape(4, 4), atol=1e-14)


def _exact_bary(coords, conn, e, p):
    P = [[Fraction(float(c)) for c in coords[v]] for v in conn[e]]
    X = [Fraction(float(c)) for c in p]
    d = len(X)
    if d == 2:
        (ax, ay), (bx, by), (cx, cy) = P
        det = (bx - ax) * (cy - ay) - (cx - ax) * (by - ay)
        m1 = ((X[0] - ax) * (cy - ay) - (cx - ax) * (X[1] - ay)) / det
        m2 = ((bx - ax) * (X[1] - ay) - (X[0] - ax) * (by - ay)) / det
        return [1 - m1 - m2, m1, m2]
    a = P[0]
    E = [[P[i][q] - a[q] for q in range(3)] for i in (1, 2, 3)]
    Q = [X[q] - a[q] for q in range(3)]

    def det3(A, B, C):
        return (A[0] * (B[1] * C[2] - B[2] * C[1]) - A[1] * (B[0] * C[2] - B[2] * C[0])
                + A[2] * (B[0] * C[1] - B[1] * C[0]))
    v = det3(*E)
    m = [det3(Q, E[1], E[2]) / v, det3(E[0], Q, E[2]) / v, det3(E[0], E[1], Q) / v]
    return [1 - sum(m)] + m


@pytest.mark.parametrize("dim,prec", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_grid_locate_equals_brute_force_and_exact_containment(orc, dim, prec):
    """The grid answer equals a scan of every element with the same rule; the
    accepted element contains the point in exact rational arithmetic up to the
    predicate's rounding."""
    src = W.jittered_tri_mesh(7, 3) if dim == 2 else W.jittered_kuhn_mesh(3, 3)
    coords = src.coords.astype(np.float32).astype(np.float64) if prec else src.coords
    rng = np.random.default_rng(1)
    pts = rng.random((3000, dim))
    # add mesh vertices and edge midpoints: the tie cases
    pts = np.concatenate([pts, coords, coords[src.conn[:, :2]].mean(1)])
    if prec:
        pts = pts.astype(np.float32).astype(np.float64)
    g = orc.Grid(prec, coords, src.conn)
    eg, sg = g.locate(pts)
    eb, sb = orc.brute_locate(prec, coords, src.conn, pts)
    tol = 1e-5 if prec else 1e-12
    mism = 0
    for i in range(pts.shape[0]):
        assert eg[i] >= 0
        mu = _exact_bary(coords, src.conn, eg[i], pts[i])
        assert min(mu) >= -tol, (i, mu)
        if eg[i] != eb[i]:
            # both candidates must contain the point up to rounding (a tie on a
            # shared face); otherwise the grid dropped a candidate
            mism += 1
            mu_b = _exact_bary(coords, src.conn, eb[i], pts[i])
            assert min(mu_b) >= -tol
            assert abs(min(mu)) <= tol or abs(min(mu_b)) <= tol
    assert mism <= pts.shape[0] // 50


@pytest.mark.parametrize("mesh", ["tri", "delaunay", "kuhn", "star"])
def test_face_neighbours_brute_force(orc, mesh):
    """The walk's face neighbours: for every element and local vertex m, the
    other element holding all vertices of the face opposite m, found by a scan
    of every element; each interior face pairs two elements both ways, and the
    number of boundary faces is that of the domain's boundary."""
    if mesh == "tri":
        m = W.jittered_tri_mesh(6, 4)
    elif mesh == "delaunay":
        m = W.delaunay_tri_mesh(60, 5, 4)
    elif mesh == "kuhn":
        m = W.jittered_kuhn_mesh(3, 4)
    else:   # every tetrahedron shares the centre vertex 0
        c = np.array([[0.5, 0.5, 0.5]] + [[x, y, z] for z in (0, 1) for y in (0, 1) for x in (0, 1)], float)
        faces = [(1, 2, 4), (1, 4, 3), (5, 6, 8), (5, 8, 7), (1, 2, 6), (1, 6, 5), (3, 4, 8), (3, 8, 7),
                 (1, 3, 7), (1, 7, 5), (2, 4, 8), (2, 8, 6)]
        m = W.Mesh(c, np.array([[0, *f] for f in faces], np.int32), None)
        W._fix_orientation(m)
    k = m.dim + 1
    adj = orc.Grid(0, m.coords, m.conn).adjacency()
    sets = [set(r.tolist()) for r in m.conn]
    nb = 0
    for e in range(m.nelems):
        for q in range(k):
            face = sets[e] - {int(m.conn[e, q])}
            others = [e2 for e2 in range(m.nelems) if e2 != e and face <= sets[e2]]
            assert adj[e, q] == (min(others) if others else -1), (e, q)
            if others:
                e2 = adj[e, q]
                back = [r for r in range(k) if int(m.conn[e2, r]) not in face]
                assert len(back) == 1 and adj[e2, back[0]] == e
            else:
                nb += 1
    if mesh == "tri":
        assert nb == 4 * 6                       # 6 edges per side of the square
    elif mesh == "kuhn":
        assert nb == 6 * 3 * 3 * 2               # 2 triangles per cube face, 6 sides
    elif mesh == "star":
        assert nb == 12                          # the cube's surface triangles


@pytest.mark.parametrize("dim,prec", [(2, 0), (2, 1), (3, 0), (3, 1)])
def test_walk_locates_interior_points_exactly(orc, dim, prec):
    """A point inside exactly one element, by a margin above the predicate's
    rounding, is located in that element whatever the search path: the walk
    agrees with a scan of every element, including from starting cells far
    from the point's element (graded mesh)."""
    src = W.jittered_tri_mesh(9, 8) if dim == 2 else W.jittered_kuhn_mesh(4, 8)
    coords = src.coords.astype(np.float32).astype(np.float64) if prec else src.coords
    # grade the mesh towards the origin: cells then hold very different elements
    coords = coords ** 2
    if prec:
        coords = coords.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(11)
    e_true = rng.integers(0, src.nelems, 4000)
    w = rng.dirichlet(np.ones(dim + 1), 4000)
    pts = np.einsum("qk,qkd->qd", w, coords[src.conn[e_true]])
    if prec:
        pts = pts.astype(np.float32).astype(np.float64)
    g = orc.Grid(prec, coords, src.conn)
    eg, sg = g.locate(pts)
    checked = 0
    for i in range(pts.shape[0]):
        mu = _exact_bary(coords, src.conn, e_true[i], pts[i])
        if min(mu) > (1e-4 if prec else 1e-9):
            assert eg[i] == e_true[i] and sg[i] == 0, (i, eg[i], e_true[i])
            checked += 1
    assert checked > 3000


@pytest.mark.parametrize("dim", [2, 3])
def test_grid_structure(orc, dim):
    src = W.jittered_tri_mesh(9, 2) if dim == 2 else W.jittered_kuhn_mesh(3, 2)
    g = orc.Grid(0, src.coords, src.conn, 1.0)
    n, nc, ni = g.shape()
    E = src.nelems
    expect_n = int(math.isqrt(E)) if dim == 2 else max(k for k in range(1, 200) if k ** 3 <= E)
    assert n[0] == expect_n and nc == expect_n ** dim
    start, items = g.csr()
    depth = g.depths()
    assert start[0] == 0 and start[-1] == ni and np.all(np.diff(start) >= 0)
    for c in range(nc):
        seg, dep = items[start[c]:start[c + 1]], depth[start[c]:start[c + 1]]
        # decreasing centre depth, ties by ascending id; every cell centre lies
        # in the meshed unit square/cube, so the first element contains it
        assert np.all((np.diff(dep) < 0) | ((np.diff(dep) == 0) & (np.diff(seg) > 0)))
        assert len(seg) == len(set(seg.tolist()))
        assert dep[0] >= 0.0
    # registration: listed cells lie in the element's bounding-box range; a
    # bounding-box cell is left out only if a face plane separates it from
    # the element (checked exactly at the box corners); random points of the
    # element land in cells that list it
    lo = src.coords.min(0)
    hi = src.coords.max(0)
    h = (hi - lo) / expect_n
    cell_of_item = np.repeat(np.arange(nc), np.diff(start))
    listed = {}
    for c, e in zip(cell_of_item, items):
        listed.setdefault(int(e), set()).add(int(c))
    rng = np.random.default_rng(5)
    import itertools
    for e in range(E):
        bb0 = src.coords[src.conn[e]].min(0)
        bb1 = src.coords[src.conn[e]].max(0)
        c0 = np.clip(np.floor((bb0 - lo) * (expect_n / (hi - lo))), 0, expect_n - 1).astype(int)
        c1 = np.clip(np.floor((bb1 - lo) * (expect_n / (hi - lo))), 0, expect_n - 1).astype(int)
        box_cells = set()
        for idx in itertools.product(*[range(c0[a], c1[a] + 1) for a in range(dim)]):
            flat = 0
            for a in reversed(range(dim)):
                flat = flat * expect_n + idx[a]
            box_cells.add(flat)
            if flat in listed.get(e, set()):
                continue
            corners = [lo + (np.array(idx) + np.array(off)) * h for off in itertools.product((0, 1), repeat=dim)]
            mus = np.array([_exact_bary(src.coords, src.conn, e, x) for x in corners], dtype=object)
            assert any(all(mus[:, m] < 0) for m in range(dim + 1)), (e, idx)
        assert listed.get(e, set()) <= box_cells
        w = rng.dirichlet(np.ones(dim + 1), 20)
        pts = w @ src.coords[src.conn[e]]
        ci = np.clip(np.floor((pts - lo) / h), 0, expect_n - 1).astype(int)
        for row in ci:
            flat = 0
            for a in reversed(range(dim)):
                flat = flat * expect_n + row[a]
            assert flat in listed[e]


# --------------------------------------------------------------------------
# mass matrix and solve (Eqs. mass_matrix, galerkin_system)
# --------------------------------------------------------------------------
def _dense(rp, col, val, n):
    A = np.zeros((n, n))
    for i in range(n):
        A[i, col[rp[i]:rp[i + 1]]] += val[rp[i]:rp[i + 1]]
    return A


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_matrix_closed_forms(orc, dim):
    """u^T M u = int (P1 interpolant)^2; for nodal values of a linear field
    L = a + b.x on the unit square/cube this equals the closed form
    a^2 + a sum(b) + sum(b^2)/3 + sum_{i<j} b_i b_j / 2."""
    m = W.delaunay_tri_mesh(60, 5, 4) if dim == 2 else W.jittered_kuhn_mesh(3, 4)
    rp, col, val = orc.mass_csr(m.coords, m.conn)
    A = _dense(rp, col, val, m.nnodes)
    assert np.allclose(A, A.T, atol=1e-17)
    assert np.all(np.linalg.eigvalsh(A) > 0)
    assert A.sum() == pytest.approx(1.0, abs=1e-13)
    assert np.allclose(A.sum(1), orc.lumped_mass(m.coords, m.conn), atol=1e-16)
    coef = np.array([0.7, -1.3, 2.1, 0.4][: dim + 1])
    u = coef[0] + m.coords @ coef[1:]
    a, b = coef[0], coef[1:]
    cross = sum(b[i] * b[j] for i in range(dim) for j in range(i + 1, dim))
    exact = a * a + a * b.sum() + (b ** 2).sum() / 3 + cross / 2
    assert u @ A @ u == pytest.approx(exact, rel=1e-12)


def test_scaled_mass_matrix_eigenvalue_bounds(orc):
    """The mixed-precision solve relies on cond(S M S) being a small constant
    for S = diag(M)^-1/2: each P1 element mass matrix against its own diagonal
    has eigenvalues in [1/2, 2] (triangles) or [1/2, 5/2] (tetrahedra), and the
    assembled scaled matrix's Rayleigh quotients stay in the union of the
    element intervals. Checked by dense eigenvalues on quasi-uniform, Delaunay,
    strongly graded, high-valence and sliver meshes."""
    meshes = [W.jittered_tri_mesh(9, 1), W.delaunay_tri_mesh(150, 9, 2)]
    g = W.delaunay_tri_mesh(150, 9, 3)
    c = g.coords.copy()
    c[:, 0] = c[:, 0] ** 4
    g = W.Mesh(c, g.conn.copy(), None)
    W._fix_orientation(g)
    meshes.append(g)
    k = 40                                          # fan: one node with 40 triangles
    ang = 2 * np.pi * np.arange(k) / k
    meshes.append(W.Mesh(np.vstack([[0.0, 0.0], np.stack([np.cos(ang), np.sin(ang)], 1)]),
                         np.array([[0, 1 + i, 1 + (i + 1) % k] for i in range(k)], np.int32), None))
    sl = W.jittered_tri_mesh(6, 4)
    meshes.append(W.Mesh(sl.coords * np.array([1.0, 1e-3]), sl.conn, None))   # slivers
    meshes += [W.jittered_kuhn_mesh(3, 5), W.morton_reorder(W.jittered_kuhn_mesh(4, 6))]
    for m in meshes:
        d = m.coords.shape[1]
        rp, col, val = orc.mass_csr(m.coords, m.conn)
        n = len(rp) - 1
        A = np.zeros((n, n))
        for i in range(n):
            A[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
        s = 1.0 / np.sqrt(np.diag(A))
        ev = np.linalg.eigvalsh(A * s[:, None] * s[None, :])
        hi = 2.0 if d == 2 else 2.5
        assert ev.min() >= 0.5 - 1e-12 and ev.max() <= hi + 1e-12, (d, ev.min(), ev.max())


def test_chebyshev_step_count_meets_target(orc):
    """The mixed solve's inner FP32 solver is the Chebyshev iteration over the
    spectrum interval pinned above ([1/2, 2] or [1/2, 5/2], widened by 1e-3),
    run for k = ceil(acosh(1/eta) / acosh(s1)) steps with s1 = theta / delta:
    the residual polynomial's maximum on the interval is 1 / T_k(s1) <= eta
    (Saad, Iterative Methods for Sparse Linear Systems, Sec. 12.3). Replayed
    here in FP32 on scaled mass matrices from the oracle (graded and sliver
    meshes included) for several targets: ||c - A y|| <= eta ||c|| after k
    steps, the recurrence residual tracks the true one, and k - 2 steps do
    not always suffice (the count is not slack by more than a step)."""
    g = W.delaunay_tri_mesh(600, 12, 3)
    c = g.coords.copy()
    c[:, 0] = c[:, 0] ** 3
    g = W.Mesh(c, g.conn.copy(), None)
    W._fix_orientation(g)
    sl = W.jittered_tri_mesh(12, 4)
    meshes = [W.delaunay_tri_mesh(1500, 15, 2), g, W.Mesh(sl.coords * np.array([1.0, 1e-3]), sl.conn, None),
              W.morton_reorder(W.jittered_kuhn_mesh(6, 9))]
    rng = np.random.default_rng(5)
    short_ok = []
    for m in meshes:
        d = m.coords.shape[1]
        rp, col, val = orc.mass_csr(m.coords, m.conn)
        n = len(rp) - 1
        rows = np.repeat(np.arange(n), np.diff(rp))
        s = 1.0 / np.sqrt(val[col == rows])
        av = (val * s[rows] * s[col]).astype(np.float32)

        def apply(x):
            return np.bincount(rows, weights=av.astype(np.float64) * x[col], minlength=n).astype(np.float32)

        a, b = 0.5 * (1 - 1e-3), (2.0 if d == 2 else 2.5) * (1 + 1e-3)
        theta, delta = (a + b) / 2, (b - a) / 2
        s1 = theta / delta
        for eta in (1e-5, 1e-3, 0.25):
            k = max(1, int(np.ceil(np.arccosh(1 / eta) / np.arccosh(s1))))
            cvec = rng.standard_normal(n).astype(np.float32)
            cvec /= np.linalg.norm(cvec)
            res = []
            for steps in (k, max(1, k - 2)):
                y = np.zeros(n, np.float32)
                r = cvec.copy()
                dv = (cvec / np.float32(theta)).astype(np.float32)
                rho = np.float32(1 / s1)
                for _ in range(steps):
                    w = apply(dv)
                    y += dv
                    r = (r - w).astype(np.float32)
                    rn = np.float32(1 / (2 * s1 - rho))
                    dv = (rn * rho * dv + (2 * rn / delta) * r).astype(np.float32)
                    rho = rn
                true_r = float(np.linalg.norm(cvec - apply(y)))
                res.append(true_r)
                if steps == k:
                    assert true_r <= eta, (d, eta, k, true_r)
                    assert abs(float(np.linalg.norm(r)) - true_r) <= 1e-5 + 1e-3 * true_r
            short_ok.append(res[1] <= eta)
    assert not all(short_ok)


def test_pcg_matches_dense_solve(orc):
    m = W.delaunay_tri_mesh(150, 6, 5)
    rp, col, val = orc.mass_csr(m.coords, m.conn)
    A = _dense(rp, col, val, m.nnodes)
    b = np.random.default_rng(2).standard_normal(m.nnodes)
    x, it, rr = orc.pcg(rp, col, val, b, tol=1e-13, max_iter=1000)
    assert rr <= 1e-13 and 0 < it < 200
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-11


# --------------------------------------------------------------------------
# the transfer (Sec. 4)
# --------------------------------------------------------------------------
def _pair(dim, ns=6, seed=0):
    if dim == 2:
        return W.jittered_tri_mesh(ns, seed), W.delaunay_tri_mesh(40, 4, seed + 1)
    return W.jittered_kuhn_mesh(3, seed), W.morton_reorder(W.jittered_kuhn_mesh(2, seed + 1))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", [0, 1])
def test_linear_field_is_reproduced(orc, dim, prec):
    """f linear and alpha = 1: f^s - g vanishes identically (both are the same
    linear function), so the residual estimate is zero up to rounding, b equals
    M f(nodes) and u equals f(nodes) (Eq. cv_load_expanded)."""
    s, t = _pair(dim)
    if prec:
        s, t = W.as_precision(s, np.float32), W.as_precision(t, np.float32)
    f = W.linear_field([1.5, 0.3, -0.7, 0.2][: dim + 1])
    s = W.with_values(s, [f], np.float64)
    r = orc.transfer(s, t, prec, 12, seed=3, cg_tol=1e-14)
    fn = f(t.coords.astype(np.float64))
    rp, col, val = orc.mass_csr(t.coords, t.conn)
    Mf = _dense(rp, col, val, t.nnodes) @ fn
    tol = 1e-6 if prec else 1e-13
    assert np.linalg.norm(r["b"][0] - Mf) / np.linalg.norm(Mf) < tol
    assert np.linalg.norm(r["u"][0] - fn) / np.linalg.norm(fn) < (1e-6 if prec else 1e-11)
    assert np.abs(r["b_res"][0]).max() < (1e-6 if prec else 1e-14)


@pytest.mark.parametrize("alpha", [0.0, 0.3, 1.0])
def test_constant_field_sum_b(orc, alpha):
    """f = c: every estimate of int c psi_i sums to c |Omega| (partition of
    unity of the target basis)."""
    s, t = _pair(2)
    s = W.with_values(s, [lambda x: np.full(x.shape[0], 2.5)], np.float64)
    r = orc.transfer(s, t, 0, 8, seed=1, alpha=alpha)
    assert r["b"][0].sum() == pytest.approx(2.5, abs=1e-13)


def test_load_vector_sum_identity(orc):
    """sum_i b_i = alpha int g + sum_t |T|/N sum_j (f^s - alpha g)(X_j)
    (partition of unity applied to Eq. cv_load_expanded), recomputed here
    from the oracle's separate sampling / location / evaluation entry points."""
    s, t = _pair(2)
    s = W.with_values(s, [W.paper_f3])
    N, alpha, seed = 6, 0.7, 4
    r = orc.transfer(s, t, 0, N, seed=seed, alpha=alpha)
    grid = orc.Grid(0, s.coords, s.conn)
    g = r["g"][0]
    assert r["b_g"][0].sum() == pytest.approx(alpha * orc.integral_p1(t.coords, t.conn, g), rel=1e-13)
    total = 0.0
    for e in range(t.nelems):
        xyz = t.coords[t.conn[e]]
        vol = 0.5 * np.linalg.det(np.array([xyz[1] - xyz[0], xyz[2] - xyz[0]]))
        lam, X = orc.sample_element(0, 2, seed, 0, e, N, xyz)
        el, _ = grid.locate(X)
        acc = 0.0
        for j in range(N):
            fs = orc.eval_p1(s.coords, s.conn, s.values, el[j], X[j])[0]
            acc += fs - alpha * lam[j] @ g[t.conn[e]]
        total += vol / N * acc
    assert r["b_res"][0].sum() == pytest.approx(total, rel=1e-11, abs=1e-14)


def test_mesh_intersection_judge_closed_forms(orc):
    """The clipping judge: exact for a linear source (b = M f(nodes)), sums to
    int f^s for any P1 source, and equals M_s f when both meshes coincide."""
    s, t = _pair(2)
    lin = W.linear_field([1.0, 2.0, -3.0])
    sl = W.with_values(s, [lin])
    b = orc.mi_load_vector_2d(sl, t)
    rp, col, val = orc.mass_csr(t.coords, t.conn)
    Mf = _dense(rp, col, val, t.nnodes) @ lin(t.coords)
    assert np.allclose(b, Mf, rtol=0, atol=1e-13)
    sf = W.with_values(s, [W.paper_f2])
    b2 = orc.mi_load_vector_2d(sf, t)
    assert b2.sum() == pytest.approx(orc.integral_p1(s.coords, s.conn, sf.values[0]), rel=1e-13)
    b3 = orc.mi_load_vector_2d(sf, s)
    rp, col, val = orc.mass_csr(s.coords, s.conn)
    assert np.allclose(b3, _dense(rp, col, val, s.nnodes) @ sf.values[0], atol=1e-13)
    # supermesh L2 error: zero for an exactly represented field, one against 0
    e, n = orc.l2_error_2d(sf, s, sf.values[0])
    assert e / n < 1e-12
    e, n = orc.l2_error_2d(sf, t, np.zeros(t.nnodes))
    assert e / n == pytest.approx(1.0, rel=1e-12)


def test_unbiased_against_mesh_intersection(orc):
    """E[b_hat] = b (Eq. cv_load_unbiased): the mean over R seeds of the
    estimate approaches the exact mesh-intersection load vector within a few
    standard errors, for alpha = 0 and alpha = 1."""
    s, t = _pair(2, ns=5)
    s = W.with_values(s, [W.field_sincos])
    b_mi = orc.mi_load_vector_2d(s, t)
    for alpha in (0.0, 1.0):
        bs = np.stack([orc.transfer(s, t, 0, 8, seed=sd, alpha=alpha, cg_max_iter=1)["b"][0]
                       for sd in range(300)])
        mean, se = bs.mean(0), bs.std(0, ddof=1) / math.sqrt(bs.shape[0])
        # entries whose estimate has (almost) no variance are compared at the
        # FP64 rounding level instead
        se = np.sqrt(se ** 2 + (1e-13 * np.abs(b_mi).max()) ** 2)
        z = (mean - b_mi) / se
        assert np.abs(z).max() < 5.0
        assert abs(z.mean()) < 5.0 / math.sqrt(z.size)


def test_error_decays_as_inverse_sqrt_N(orc):
    """RMS load-vector error ~ N^{-1/2} (Monte Carlo variance ~ 1/N)."""
    s, t = _pair(2, ns=5)
    s = W.with_values(s, [W.field_sincos])
    b_mi = orc.mi_load_vector_2d(s, t)
    Ns = [4, 16, 64, 256]
    rms = []
    for N in Ns:
        errs = [np.linalg.norm(orc.transfer(s, t, 0, N, seed=sd, alpha=0.0, cg_max_iter=1)["b"][0]
                               - b_mi) for sd in range(40)]
        rms.append(math.sqrt(np.mean(np.square(errs))))
    slope = np.polyfit(np.log(Ns), np.log(rms), 1)[0]
    assert -0.56 < slope < -0.44


def test_roundtrip_exact_projection_conserves_and_linear_fields_survive(orc):
    """Round trips (the iterative analysis of Sec. 5): repeated exact Galerkin
    projections (mesh-intersection load vectors) conserve the integral, since
    both P1 spaces contain the constants (test function sum_i psi_i = 1), so
    E_mass stays at rounding level; a linear field is reproduced by every
    projection, exactly (MI) and by the control-variate estimate with
    alpha = 1 (the residual f - g vanishes)."""
    a = W.delaunay_tri_mesh(120, 8, 3)
    b = W.jittered_tri_mesh(5, 4)
    f = W.paper_f2(a.coords)
    errs, _ = orc.roundtrip(a, b, f, 3, 0, 8, exact=True, cg_tol=1e-14)
    assert all(em < 1e-12 for _, em in errs)
    assert 0 < errs[0][0] < errs[-1][0]          # projection errors do accumulate in l2
    lin = W.linear_field([0.3, -1.2, 2.0])(a.coords)
    for exact in (True, False):
        errs, _ = orc.roundtrip(a, b, lin, 2, 0, 8, exact=exact, cg_tol=1e-14)
        assert all(el < 1e-11 and em < 1e-11 for el, em in errs), errs


def test_roundtrip_monte_carlo_is_unbiased_for_the_exact_round_trip(orc):
    """One round trip with independent samples in its two legs is unbiased
    for the exact (mesh-intersection) round trip: each leg is linear in its
    input values and unbiased (Eq. cv_load_unbiased), and the legs draw
    independent samples, so E[A2 A1 f] = E[A2] E[A1] f. The mean over 150
    seed pairs approaches the exact round trip within a few standard errors."""
    a = W.delaunay_tri_mesh(60, 6, 5)
    b = W.jittered_tri_mesh(4, 6)
    f = W.paper_f2(a.coords)
    _, f_mi = orc.roundtrip(a, b, f, 1, 0, 8, exact=True, cg_tol=1e-14)
    runs = np.stack([orc.roundtrip(a, b, f, 1, 0, 8, seeds=(sd, 1000 + sd), cg_tol=1e-14)[1]
                     for sd in range(150)])
    mean, se = runs.mean(0), runs.std(0, ddof=1) / math.sqrt(runs.shape[0])
    se = np.sqrt(se ** 2 + (1e-12 * np.abs(f_mi).max()) ** 2)
    z = (mean - f_mi) / se
    assert np.abs(z).max() < 5.0
    assert abs(z.mean()) < 5.0 / math.sqrt(z.size)


def test_alpha_reduces_error(orc):
    """Both errors decrease as alpha goes from 0 to 1 (Sec. 5.1, alpha study)."""
    s, t = _pair(2, ns=8)
    s = W.with_values(s, [W.paper_f3])
    b_mi = orc.mi_load_vector_2d(s, t)
    Is = orc.integral_p1(s.coords, s.conn, s.values[0])
    err, cons = [], []
    for alpha in (0.0, 0.5, 1.0):
        e_b, e_c = [], []
        for sd in range(30):
            r = orc.transfer(s, t, 0, 20, seed=sd, alpha=alpha, cg_max_iter=1)
            e_b.append(np.linalg.norm(r["b"][0] - b_mi))
            e_c.append(r["b"][0].sum() - Is)
        err.append(np.sqrt(np.mean(np.square(e_b))))
        cons.append(np.sqrt(np.mean(np.square(e_c))))
    assert err[0] > err[1] > err[2]
    assert cons[0] > cons[1] > cons[2]


@pytest.mark.slow
def test_convergence_rates_in_h(orc):
    """At alpha = 1, N = 20: E_L2 ~ h^2 and the RMS conservation error
    ~ h^3 / sqrt(N) in 2D (Eqs. accuracy_bound_interpretation and
    conservation_bound_interpretation)."""
    el2, econs, hs = [], [], []
    for n in (6, 12, 24, 48):
        s = W.with_values(W.jittered_tri_mesh(n, 10), [W.paper_f3])
        side = int(round(n * 0.9))
        t = W.delaunay_tri_mesh((side - 1) ** 2, side - 1, 11)
        Is = orc.integral_p1(s.coords, s.conn, s.values[0])
        c, e = [], []
        for sd in range(12):
            r = orc.transfer(s, t, 0, 20, seed=sd, cg_tol=1e-13)
            It = orc.lumped_mass(t.coords, t.conn) @ r["u"][0]
            c.append((It - Is) / Is)
            if sd < 2:
                err, nrm = orc.l2_error_2d(s, t, r["u"][0])
                e.append(err / nrm)
        hs.append(1.0 / n)
        el2.append(np.mean(e))
        econs.append(math.sqrt(np.mean(np.square(c))))
    s_l2 = np.polyfit(np.log(hs), np.log(el2), 1)[0]
    s_c = np.polyfit(np.log(hs), np.log(econs), 1)[0]
    assert 1.6 < s_l2 < 2.4
    assert 2.4 < s_c < 3.6


def test_conservation_at_convergence(orc):
    """int f^t = sum_i u_i m_i = sum_i b_i once M u = b is solved (Sec. 2,
    Eq. conservation with 1 in V_t)."""
    s, t = _pair(2)
    s = W.with_values(s, [W.paper_f1, W.paper_f2])
    r = orc.transfer(s, t, 0, 10, seed=2, cg_tol=1e-14)
    m = orc.lumped_mass(t.coords, t.conn)
    for q in range(2):
        assert m @ r["u"][q] == pytest.approx(r["b"][q].sum(), rel=1e-12)


# --------------------------------------------------------------------------
# the surrogate network (FP64)
# --------------------------------------------------------------------------
def _mlp_params(seed, scale=1.0):
    import workloads as W_
    return W_.mlp_init(seed) * scale


def test_bf16_rounding_hand_cases(orc):
    """bfloat16 keeps 8 significant bits, ties to even (worked by hand)."""
    assert orc.bf16_round(1.0) == 1.0
    assert orc.bf16_round(1.0 + 2 ** -8) == 1.0                 # tie -> even (1.0)
    assert orc.bf16_round(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6   # tie -> even (1 + 2^-6)
    assert orc.bf16_round(1.0 + 2 ** -8 + 2 ** -12) == 1.0 + 2 ** -7
    assert orc.bf16_round(-3.0) == -3.0
    assert orc.bf16_round(0.1) == 0.10009765625


def test_mlp_zero_weights_and_silu(orc):
    p = np.zeros(orc.mlp_nparam())
    p[-1] = 0.75                        # c5
    X = np.random.default_rng(0).random((5, 3))
    assert np.allclose(orc.mlp_forward(p, X), 0.75)
    # one active path: W1[0] = e_x, w5[0] = 1 and identity-free hidden layers
    # give y = silu(x) only if later layers pass it through; use c's instead:
    q = np.zeros(orc.mlp_nparam())
    W1, c1, W2, c2, W3, c3, W4, c4, w5, c5 = orc.mlp_split(q)
    c4[0] = 2.0
    w5[0] = 1.0
    y = orc.mlp_forward(q, X)
    assert np.allclose(y, 2.0 / (1.0 + np.exp(-2.0)))   # silu(2)


def test_mlp_gradient_matches_finite_differences(orc):
    p = _mlp_params(3)
    rng = np.random.default_rng(4)
    X = rng.random((6, 3))
    t = rng.standard_normal(6)
    loss, g = orc.mlp_loss_grad(p, X, t)
    idx = rng.choice(p.size, 40, replace=False)
    idx = np.concatenate([idx, [0, 767, 768, p.size - 257, p.size - 1]])   # W1, c1, w5, c5 entries
    for i in idx:
        h = 1e-6 * max(1.0, abs(p[i]))
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (orc.mlp_loss_grad(pp, X, t)[0] - orc.mlp_loss_grad(pm, X, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(g[i])) + 1e-10, (i, fd, g[i])


def test_adam_first_step_closed_form(orc):
    """From m = v = 0 the bias-corrected first step is lr g / (|g| + eps)."""
    p = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    m, v = np.zeros(3), np.zeros(3)
    orc.adam_step(p, g, m, v, 1, lr=0.01)
    assert np.allclose(p, np.array([1.0, -2.0, 0.5]) - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


# ---------------------------------------------------------------------------
# surrogate-source transfer oracle (network as the black box, exact fallback)
# ---------------------------------------------------------------------------
def _const_net(orc, c):
    """A network whose output is the constant c (all weights zero, c5 = c)."""
    p = np.zeros(orc.mlp_nparam())
    p[-1] = c
    return p


def _sur_meshes():
    import workloads as W_
    tgt = W_.jittered_kuhn_mesh(3, seed=2)
    src = W_.with_values(W_.jittered_tri_mesh(6, seed=3), [W_.linear_field([0.3, 1.5, -0.7])])
    return src, tgt


def test_surrogate_constant_network_gives_mass_times_constant(orc):
    """alpha = 1 and a constant source c: every residual vanishes, so b is the
    control term alone, b_i = c * int psi_i (the lumped mass), and u = c."""
    from oracle import surrogate as S
    _, tgt = _sur_meshes()
    out = S.surrogate_transfer(_const_net(orc, 0.75), tgt.coords, tgt.conn, N=8, seed=4)
    m = orc.lumped_mass(tgt.coords, tgt.conn)
    assert np.allclose(out["g"], 0.75, rtol=0, atol=1e-15)
    assert np.allclose(out["b"], 0.75 * m, rtol=1e-12, atol=0)
    assert np.allclose(out["u"], 0.75, atol=1e-9)


def test_surrogate_alpha_zero_conserves_total(orc):
    """alpha = 0: b is the plain Monte Carlo load vector; the barycentric
    weights sum to one, so sum_i b_i = c * |Omega| exactly (up to rounding)."""
    from oracle import surrogate as S
    _, tgt = _sur_meshes()
    out = S.surrogate_transfer(_const_net(orc, -1.25), tgt.coords, tgt.conn, N=5, seed=9, alpha=0.0)
    assert abs(out["b"].sum() - (-1.25) * 1.0) < 1e-6   # the jittered cube keeps volume 1


def test_surrogate_exact_only_reproduces_linear_field(orc):
    """No network: every query exact. A linear field of (x, y) is reproduced
    by the 2D source, the residuals vanish (alpha = 1) and u equals the field
    at the 3D target's nodes (the source extruded along z)."""
    from oracle import surrogate as S
    src, tgt = _sur_meshes()
    out = S.surrogate_transfer(None, tgt.coords, tgt.conn, N=6, seed=1,
                               exact=(src.coords, src.conn, src.values[0]))
    ref = 0.3 + 1.5 * tgt.coords[:, 0] - 0.7 * tgt.coords[:, 1]
    assert out["fallback"].all()
    assert np.abs(out["u"] - ref).max() < 2e-6


def test_surrogate_fallback_margin_closed_form(orc):
    """Constant network c against the linear exact field l: the margin of an
    element is max_{j<s} |c - l(X_j)| over its first s sample points, and the
    element falls back exactly when that exceeds tau. Fallback elements then
    carry the exact field, the others the constant."""
    from oracle import surrogate as S
    src, tgt = _sur_meshes()
    c, N, s, seed = 0.9, 8, 3, 6
    tau = 0.35
    out = S.surrogate_transfer(_const_net(orc, c), tgt.coords, tgt.conn, N=N, seed=seed,
                               exact=(src.coords, src.conn, src.values[0]), tau=tau, s=s)
    ref_margin = np.zeros(len(tgt.conn))
    for t in range(len(tgt.conn)):
        _, X = orc.sample_element(1, 3, seed, 0, t, N, tgt.coords[tgt.conn[t]])
        lX = 0.3 + 1.5 * X[:s, 0] - 0.7 * X[:s, 1]
        ref_margin[t] = np.abs(c - lX).max()
        lall = 0.3 + 1.5 * X[:, 0] - 0.7 * X[:, 1]
        expect = lall if ref_margin[t] > tau else np.full(N, c)
        assert np.allclose(out["f"][t], expect, atol=2e-6)
    assert np.allclose(out["margin"], ref_margin, atol=2e-6)
    assert np.array_equal(out["fallback"], ref_margin > tau)
    assert 0 < out["fallback"].sum() < len(tgt.conn)


def test_surrogate_dataset_points_and_values(orc):
    """Training points lie in the box, are uniform (mean within 5 standard
    errors of the centre) and carry the exact (x, y) field, here linear, so
    it is reproduced exactly by the P1 source."""
    from oracle import surrogate as S
    src, _ = _sur_meshes()
    pts, f, e = S.surrogate_dataset(src.coords, src.conn, src.values[0], 3000, seed=11,
                                    box_lo=(0, 0, 0.25), box_hi=(1, 1, 0.75))
    assert pts.dtype == np.float32
    assert (pts[:, :2] > 0).all() and (pts[:, :2] < 1).all()
    assert (pts[:, 2] > 0.25).all() and (pts[:, 2] < 0.75).all()
    se = np.array([1, 1, 0.5]) / np.sqrt(12 * 3000)
    assert np.all(np.abs(pts.mean(axis=0) - [0.5, 0.5, 0.5]) < 5 * se)
    assert (e >= 0).all()
    ref = 0.3 + 1.5 * pts[:, 0].astype(np.float64) - 0.7 * pts[:, 1].astype(np.float64)
    assert np.abs(f - ref).max() < 1e-12
