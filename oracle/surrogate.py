"""Oracle of the surrogate-source transfer: Sec. 4, steps 1-7, with the
black-box query answered by the surrogate network (the learned source the
paper's introduction motivates) and a per-element exact fallback; plus the
surrogate's training set. Plain numpy over the oracle's C primitives (Philox,
the FP32 sampler, the FP32 grid location, the FP64 network).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Readings used (restated from the method, not from any implementation):
  * Training point j: u_a = FP32 uniform of Philox word a of counter
    (j_lo32, j_hi32, stream, 1) with key (seed_lo32, seed_hi32);
    x_a = lo_a + u_a * (hi_a - lo_a), each operation rounded to FP32.
  * An exact query of a point locates its first d_s coordinates in the exact
    source (FP32 location) and evaluates the P1 field there (0 in an empty
    cell); the network sees all three coordinates (z = 0 for a 2D target).
  * Fallback: the first s samples of an element are queried both ways; the
    element uses exact queries for all samples when max |f_net - f_exact| > tau
    (or the difference is not finite).
  * Control g = network at the target nodes (exact source when there is no
    network); deterministic term alpha * |T| / ((d+1)(d+2)) * (sum_m g_m + g_i).
"""
from __future__ import annotations

import numpy as np

from . import Grid, eval_p1, mass_csr, mlp_forward, pcg, philox4x32_10, sample_element, u01


def _exact_values(grid: Grid, coords, conn, values, X):
    """Exact P1 source at the first d_s coordinates of the points X."""
    ds = grid.dim
    e, _ = grid.locate(np.asarray(X, np.float64)[:, :ds])
    out = np.zeros(len(e))
    for k, ek in enumerate(e):
        if ek >= 0:
            out[k] = eval_p1(coords, conn, values, int(ek), X[k, :ds])[0]
    return out, e


def surrogate_dataset(coords, conn, values, n, seed=0, stream_id=0, box_lo=(0, 0, 0), box_hi=(1, 1, 1)):
    """(points [n,3] float32, exact values [n], located element [n])."""
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], np.uint32)
    lo = np.asarray(box_lo, np.float32)
    w = np.asarray(box_hi, np.float32) - lo
    pts = np.zeros((n, 3), np.float32)
    for j in range(n):
        r = philox4x32_10([j & 0xFFFFFFFF, (j >> 32) & 0xFFFFFFFF, stream_id, 1], key)
        for a in range(3):
            u = np.float32(u01(int(r[a]), 1))
            pts[j, a] = lo[a] + np.float32(u * w[a])
    grid = Grid(1, coords, conn)
    f, e = _exact_values(grid, np.asarray(coords, np.float64), conn, values, pts.astype(np.float64))
    return pts, f, e


def surrogate_transfer(params, tgt_coords, tgt_conn, N, seed=0, stream=0, alpha=1.0, exact=None, tau=0.0, s=4,
                       cg_tol=1e-12, cg_max_iter=2000, sampling=0):
    """params: the network the GPU computes with (FP64 vector) or None (every
    query exact); exact: (coords, conn, values of one field) or None;
    sampling: 0 uniform, 1 stratified (as the mesh-source transfer).
    Returns a dict: g, b, u, fallback [E] bool, margin [E], f [E, N]."""
    tc = np.asarray(tgt_coords, np.float64)
    tconn = np.asarray(tgt_conn, np.int32)
    E, K = tconn.shape
    d = K - 1
    tc32 = tc.astype(np.float32).astype(np.float64)   # the FP32 path's node coordinates
    grid = Grid(1, exact[0], exact[1]) if exact is not None else None

    def pad3(X):
        out = np.zeros((X.shape[0], 3))
        out[:, :X.shape[1]] = X
        return out

    # step 1: control values at the target nodes
    if params is not None:
        g = mlp_forward(params, pad3(tc32), act_bf16=True)
    else:
        g, _ = _exact_values(grid, exact[0], exact[1], exact[2], tc32)
    # steps 2-3: samples (FP32 sampler, the element's FP32 node coordinates)
    lam = np.zeros((E, N, K))
    X = np.zeros((E, N, d))
    for t in range(E):
        lam[t], X[t] = sample_element(1, d, seed, stream, t, N, tc[tconn[t]], sampling=sampling)
    Xf = X.reshape(-1, d)
    # step 4: the query
    fallback = np.zeros(E, bool)
    margin = np.zeros(E)
    if params is not None:
        f = mlp_forward(params, pad3(Xf), act_bf16=True).reshape(E, N)
        if grid is not None and s > 0:
            fe_sub, _ = _exact_values(grid, exact[0], exact[1], exact[2], X[:, :s].reshape(-1, d))
            diff = np.abs(f[:, :s] - fe_sub.reshape(E, s))
            margin = np.max(np.where(np.isfinite(diff), diff, np.inf), axis=1)
            fallback = ~(margin <= tau)
            if fallback.any():
                idx = np.nonzero(fallback)[0]
                fe, _ = _exact_values(grid, exact[0], exact[1], exact[2], X[idx].reshape(-1, d))
                f[idx] = fe.reshape(len(idx), N)
    else:
        fe, _ = _exact_values(grid, exact[0], exact[1], exact[2], Xf)
        f = fe.reshape(E, N)
        fallback[:] = True
    # steps 5-6: residual against the P1 control, weighted by the target basis
    gX = np.einsum("tjm,tm->tj", lam, g[tconn])
    r = f - alpha * gX
    vol = _measures(tc, tconn)
    b = np.zeros(tc.shape[0])
    mc = np.einsum("tj,tji->ti", r, lam) * (vol / N)[:, None]
    det = alpha * (vol / ((d + 1) * (d + 2)))[:, None] * (g[tconn].sum(axis=1)[:, None] + g[tconn])
    np.add.at(b, tconn.ravel(), (mc + det).ravel())
    # step 7: M u = b
    rp, col, val = mass_csr(tc, tconn)
    u, it, rr = pcg(rp, col, val, b, tol=cg_tol, max_iter=cg_max_iter)
    return {"g": g, "b": b, "u": u, "fallback": fallback, "margin": margin, "f": f, "cg_iters": it}


def _measures(coords, conn):
    d = conn.shape[1] - 1
    x = coords[conn]
    if d == 2:
        e1, e2 = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0]
        return 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    return np.linalg.det(x[:, 1:] - x[:, :1]) / 6.0
