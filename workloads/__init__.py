"""Seeded synthetic workloads: meshes, nodal fields and batched request lists.

This module is the only code shared by the CUDA path's tests/bench and the
oracle's tests. It contains input generation only -- no arithmetic of the
transfer method itself (no sampling, location, quadrature or solve).

Mesh conventions (the paper's problem statement, Sec. 2: a target P1 FE mesh
and a source P1 mesh carrying nodal values, both covering the same domain):

* ``coords``  float array ``[V, d]`` (float64, or float32 for the FP32 workloads)
* ``conn``    int32 array ``[E, d+1]``, every element positively oriented
* ``values``  float array ``[nf, V]`` nodal values of the source field(s)

Recipes (all on the unit square / unit cube, so source and target cover the
same domain exactly, which the conservation statement of Sec. 2 requires):

* jittered structured triangle mesh: (n+1)^2 nodes, interior nodes moved by a
  uniform offset in [-0.2h, 0.2h] per axis, boundary nodes only along their
  side, corners fixed; each square split SW->NE into two CCW triangles.
* Delaunay triangle mesh: uniform random interior points plus the 4 corners
  plus ``per_side`` evenly spaced points on each side, triangulated by scipy's
  Delaunay (Qhull); triangles and nodes reordered along a Morton curve.
* jittered Kuhn tetrahedral mesh: (n+1)^3 nodes, interior jitter +-0.1h,
  boundary nodes only tangentially; each cube split into the 6 tetrahedra
  around its main diagonal; negative tets are re-oriented by a vertex swap.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Mesh", "jittered_tri_mesh", "delaunay_tri_mesh", "jittered_kuhn_mesh",
    "morton_reorder", "field_sincos", "field_gauss_jump_2d", "gauss8_params",
    "field_gauss8_jump_3d", "paper_f1", "paper_f2", "paper_f3", "linear_field",
    "with_values", "as_precision", "config_meshes", "batch_requests",
]


@dataclasses.dataclass
class Mesh:
    coords: np.ndarray            # [V, d]
    conn: np.ndarray              # [E, d+1] int32
    values: np.ndarray | None = None   # [nf, V]

    @property
    def dim(self) -> int:
        return int(self.coords.shape[1])

    @property
    def nnodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def nelems(self) -> int:
        return int(self.conn.shape[0])

    @property
    def nfields(self) -> int:
        return 0 if self.values is None else int(self.values.shape[0])


# ----------------------------------------------------------------------------
# geometry helpers (input validation only)
# ----------------------------------------------------------------------------
def _signed_measure(coords: np.ndarray, conn: np.ndarray) -> np.ndarray:
    c = coords.astype(np.float64)
    if coords.shape[1] == 2:
        a, b, d = c[conn[:, 0]], c[conn[:, 1]], c[conn[:, 2]]
        return 0.5 * ((b[:, 0] - a[:, 0]) * (d[:, 1] - a[:, 1])
                      - (d[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1]))
    a = c[conn[:, 0]]
    e1, e2, e3 = c[conn[:, 1]] - a, c[conn[:, 2]] - a, c[conn[:, 3]] - a
    return np.einsum("ij,ij->i", e1, np.cross(e2, e3)) / 6.0


def _check_mesh(m: Mesh, what: str) -> None:
    vol = _signed_measure(m.coords, m.conn)
    if not np.all(vol > 0):
        raise ValueError(f"{what}: {np.count_nonzero(vol <= 0)} non-positive elements")
    tot = float(vol.sum())
    if abs(tot - 1.0) > 1e-9:
        raise ValueError(f"{what}: elements cover measure {tot}, expected 1")
    used = np.zeros(m.nnodes, bool)
    used[m.conn.ravel()] = True
    if not used.all():
        raise ValueError(f"{what}: {np.count_nonzero(~used)} unused nodes")


def _morton_codes(p: np.ndarray, bits: int) -> np.ndarray:
    """Interleaved-bit Morton code of points in [0,1]^d (d = 2 or 3)."""
    d = p.shape[1]
    q = np.clip((p * (1 << bits)).astype(np.int64), 0, (1 << bits) - 1).astype(np.uint64)
    code = np.zeros(p.shape[0], np.uint64)
    for bit in range(bits):
        for ax in range(d):
            code |= ((q[:, ax] >> np.uint64(bit)) & np.uint64(1)) << np.uint64(bit * d + ax)
    return code


def morton_reorder(m: Mesh) -> Mesh:
    """Renumber nodes and elements along a Morton curve (element order by
    centroid), so that consecutive elements and node ids are spatially close."""
    bits = 21 if m.dim == 3 else 31
    node_perm = np.argsort(_morton_codes(m.coords.astype(np.float64), bits), kind="stable")
    inv = np.empty_like(node_perm)
    inv[node_perm] = np.arange(node_perm.size)
    coords = m.coords[node_perm]
    conn = inv[m.conn].astype(np.int32)
    cen = coords.astype(np.float64)[conn].mean(axis=1)
    el_perm = np.argsort(_morton_codes(cen, bits), kind="stable")
    values = None if m.values is None else m.values[:, node_perm]
    return Mesh(np.ascontiguousarray(coords), np.ascontiguousarray(conn[el_perm]), values)


# ----------------------------------------------------------------------------
# mesh generators
# ----------------------------------------------------------------------------
def _jitter_grid(n: int, d: int, amp: float, rng: np.random.Generator) -> np.ndarray:
    h = 1.0 / n
    ax = np.linspace(0.0, 1.0, n + 1)
    grids = np.meshgrid(*([ax] * d), indexing="ij")
    pts = np.stack([g.ravel() for g in grids], axis=1)      # index = ((i*(n+1))+j)*(n+1)+k
    idx = np.stack(np.meshgrid(*([np.arange(n + 1)] * d), indexing="ij"), -1).reshape(-1, d)
    off = rng.uniform(-amp * h, amp * h, size=pts.shape)
    on_bnd = (idx == 0) | (idx == n)                        # per axis: fixed along that axis
    off[on_bnd] = 0.0
    return pts + off


def jittered_tri_mesh(n: int, seed: int, jitter: float = 0.2) -> Mesh:
    """2 n^2 triangles on the unit square (structured, jittered)."""
    rng = np.random.default_rng(seed)
    pts = _jitter_grid(n, 2, jitter, rng)
    i, j = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00 = i * (n + 1) + j
    v10 = (i + 1) * (n + 1) + j
    v01 = i * (n + 1) + j + 1
    v11 = (i + 1) * (n + 1) + j + 1
    t1 = np.stack([v00, v10, v11], 1)
    t2 = np.stack([v00, v11, v01], 1)
    conn = np.stack([t1, t2], 1).reshape(-1, 3).astype(np.int32)
    m = Mesh(pts, conn)
    _fix_orientation(m)
    _check_mesh(m, "jittered_tri_mesh")
    return m


def delaunay_tri_mesh(n_interior: int, per_side: int, seed: int) -> Mesh:
    """Delaunay triangulation of uniform random interior points, the 4 corners
    and ``per_side`` evenly spaced points per side: 2*n_interior + h - 2
    triangles with h = 4 + 4*per_side hull vertices."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    pts = rng.random((n_interior, 2))
    s = (np.arange(1, per_side + 1) / (per_side + 1)).astype(np.float64)
    z, o = np.zeros_like(s), np.ones_like(s)
    bnd = np.concatenate([np.stack([s, z], 1), np.stack([o, s], 1),
                          np.stack([s, o], 1), np.stack([z, s], 1),
                          np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])])
    allp = np.concatenate([pts, bnd])
    tri = Delaunay(allp)
    m = Mesh(allp, tri.simplices.astype(np.int32))
    _fix_orientation(m)
    expect = 2 * n_interior + (4 + 4 * per_side) - 2
    if m.nelems != expect:
        raise ValueError(f"delaunay_tri_mesh: {m.nelems} triangles, expected {expect}")
    _check_mesh(m, "delaunay_tri_mesh")
    return morton_reorder(m)


def jittered_kuhn_mesh(n: int, seed: int, jitter: float = 0.1) -> Mesh:
    """6 n^3 tetrahedra on the unit cube (Kuhn split of a jittered grid)."""
    rng = np.random.default_rng(seed)
    pts = _jitter_grid(n, 3, jitter, rng)
    i, j, k = (a.ravel() for a in np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij"))

    def v(di, dj, dk):
        return ((i + di) * (n + 1) + (j + dj)) * (n + 1) + (k + dk)

    c000, c111 = v(0, 0, 0), v(1, 1, 1)
    paths = [(v(1, 0, 0), v(1, 1, 0)), (v(1, 0, 0), v(1, 0, 1)),
             (v(0, 1, 0), v(1, 1, 0)), (v(0, 1, 0), v(0, 1, 1)),
             (v(0, 0, 1), v(1, 0, 1)), (v(0, 0, 1), v(0, 1, 1))]
    tets = [np.stack([c000, a, b, c111], 1) for a, b in paths]
    conn = np.stack(tets, 1).reshape(-1, 4).astype(np.int32)
    m = Mesh(pts, conn)
    _fix_orientation(m)
    _check_mesh(m, "jittered_kuhn_mesh")
    return m


def _fix_orientation(m: Mesh) -> None:
    vol = _signed_measure(m.coords, m.conn)
    neg = vol < 0
    if neg.any():
        m.conn[neg, 1], m.conn[neg, 2] = m.conn[neg, 2].copy(), m.conn[neg, 1].copy()


# ----------------------------------------------------------------------------
# analytic fields (evaluated at nodes: "interpolated onto the source mesh")
# ----------------------------------------------------------------------------
def field_sincos(x: np.ndarray) -> np.ndarray:
    """sin(2 pi x) cos(2 pi y) + x^2 (the small 2D workload)."""
    return np.sin(2 * np.pi * x[:, 0]) * np.cos(2 * np.pi * x[:, 1]) + x[:, 0] ** 2


def field_gauss_jump_2d(x: np.ndarray) -> np.ndarray:
    """exp(-|x-c|^2/0.01) + 0.5 sign(x-0.5), c = (0.5, 0.5), sign(0) = 0."""
    r2 = (x[:, 0] - 0.5) ** 2 + (x[:, 1] - 0.5) ** 2
    return np.exp(-r2 / 0.01) + 0.5 * np.sign(x[:, 0] - 0.5)


def gauss8_params(seed: int = 0):
    rng = np.random.default_rng(seed)
    c = rng.random((8, 3))
    sig = rng.uniform(0.03, 0.2, 8)
    amp = rng.uniform(0.5, 1.5, 8)
    return c, sig, amp


def field_gauss8_jump_3d(x: np.ndarray, seed: int = 0) -> np.ndarray:
    """Sum of 8 seeded Gaussians (sigma in [0.03, 0.2]) + 0.5 sign(z - 0.4)."""
    c, sig, amp = gauss8_params(seed)
    out = np.zeros(x.shape[0])
    for k in range(8):
        r2 = ((x - c[k]) ** 2).sum(axis=1)
        out += amp[k] * np.exp(-r2 / (2 * sig[k] ** 2))
    return out + 0.5 * np.sign(x[:, 2] - 0.4)


def paper_f1(x):  # Eq. (test_functions), f1
    return 5 * x[:, 1] ** 3 + x[:, 0] ** 2 + 2 * x[:, 1] + 3


def paper_f2(x):  # f2
    return np.sin(x[:, 0]) * np.cos(x[:, 1]) + 2


def paper_f3(x):  # f3
    return np.exp(x[:, 0] ** 2) + 2 * x[:, 1]


def linear_field(coef):
    """a0 + a1 x + a2 y (+ a3 z)."""
    coef = np.asarray(coef, np.float64)

    def f(x):
        return coef[0] + x @ coef[1:1 + x.shape[1]]
    return f


def with_values(m: Mesh, fields, dtype=None) -> Mesh:
    """Attach nodal values of the given analytic fields (evaluated in float64
    at the stored coordinates) to a copy of the mesh."""
    x = m.coords.astype(np.float64)
    vals = np.stack([np.asarray(f(x), np.float64) for f in fields])
    dt = dtype or m.coords.dtype
    return Mesh(m.coords, m.conn, np.ascontiguousarray(vals.astype(dt)))


def as_precision(m: Mesh, dtype) -> Mesh:
    vals = None if m.values is None else np.ascontiguousarray(m.values.astype(dtype))
    return Mesh(np.ascontiguousarray(m.coords.astype(dtype)), m.conn, vals)


# ----------------------------------------------------------------------------
# the named workloads
# ----------------------------------------------------------------------------
def config_meshes(name: str, scale: float = 1.0):
    """Return (source, target, params) for a named workload.

    ``scale`` < 1 shrinks the element counts (for oracle-sized parity cases)
    while keeping the generator, field and dtype of the workload.

    * ``tri2k``:   2,048-triangle source (32x32x2) with sin(2 pi x)cos(2 pi y)+x^2,
      1,500-triangle Delaunay target, N = 16, float64.
    * ``tri4m``:   3,998,792-triangle source (1414^2 x 2), Gaussian + jump field,
      float32 coords; 2,000,000-triangle Delaunay target; N = 64.
    * ``tet5m``:   4,983,504-tet source (94^3 x 6), 8 Gaussians + jump;
      2,958,234-tet target (79^3 x 6, independent jitter); N = 32; float32.
    * ``roundtrip``: (mesh 1, mesh 2, params) of the round-trip analysis: f2 on
      a 2,000,000-triangle Delaunay mesh, a 199,712-triangle jittered mesh,
      N = 20, float64 values.
    * ``sur3d``:   the tri4m source field extruded along z, F(x,y,z) = f(x,y),
      learned by the surrogate network from 2,000,000 seeded points, onto the
      tet5m target with N = 64; exact fallback subsample s = 4,
      tau = 1e-2 max |f| over the training set.
    """
    if name == "tri2k":
        n = max(2, int(round(32 * math.sqrt(scale))))
        src = with_values(jittered_tri_mesh(n, seed=0), [field_sincos])
        ni = max(4, int(round(721 * scale)))
        ps = max(1, int(round(14 * math.sqrt(scale))))
        tgt = delaunay_tri_mesh(ni, ps, seed=1)
        return src, tgt, dict(samples_per_elem=16, dtype="float64", cg_tol=1e-12)
    if name == "tri4m":
        n = max(2, int(round(1414 * math.sqrt(scale))))
        src = as_precision(with_values(jittered_tri_mesh(n, seed=0), [field_gauss_jump_2d]), np.float32)
        side = max(2, int(round(1000 * math.sqrt(scale))))
        tgt = as_precision(delaunay_tri_mesh((side - 1) ** 2, side - 1, seed=1), np.float32)
        return src, tgt, dict(samples_per_elem=64, dtype="float32", cg_tol=1e-10)
    if name == "tet5m":
        ns = max(2, int(round(94 * scale ** (1 / 3))))
        nt = max(2, int(round(79 * scale ** (1 / 3))))
        src = as_precision(with_values(jittered_kuhn_mesh(ns, seed=0),
                                       [lambda x: field_gauss8_jump_3d(x, 0)]), np.float32)
        tgt = as_precision(morton_reorder(jittered_kuhn_mesh(nt, seed=1)), np.float32)
        return src, tgt, dict(samples_per_elem=32, dtype="float32", cg_tol=1e-10)
    if name == "sur3d":
        # the 2D source of tri4m, extruded along z, learned by the surrogate
        # network and transferred onto the 3D target of tet5m with N = 64
        n = max(2, int(round(1414 * math.sqrt(scale))))
        src = as_precision(with_values(jittered_tri_mesh(n, seed=0), [field_gauss_jump_2d]), np.float32)
        nt = max(2, int(round(79 * scale ** (1 / 3))))
        tgt = as_precision(morton_reorder(jittered_kuhn_mesh(nt, seed=1)), np.float32)
        return src, tgt, dict(samples_per_elem=64, dtype="float32", cg_tol=1e-10,
                              train_points=max(4096, int(round(2_000_000 * scale))), subsample=4, tau_rel=1e-2)
    if name == "roundtrip":
        # the iterative analysis (Sec. 5) at scale: the reference field f2 on a
        # fine 2,000,000-triangle Delaunay mesh (mesh 1) carried through a
        # 10x coarser 199,712-triangle jittered mesh (mesh 2) and back,
        # N = 20 samples per element as in the paper; FP64 values (each leg's
        # FP64 solution is the next leg's source)
        side = max(2, int(round(1000 * math.sqrt(scale))))
        m1 = with_values(delaunay_tri_mesh((side - 1) ** 2, side - 1, seed=1), [paper_f2], np.float64)
        n2 = max(2, int(round(316 * math.sqrt(scale))))
        m2 = with_values(jittered_tri_mesh(n2, seed=2), [lambda x: 0.0 * x[:, 0]], np.float64)
        return m1, m2, dict(samples_per_elem=20, dtype="float64", cg_tol=1e-10)
    raise KeyError(name)


BATCH_FIELDS_2D = [paper_f1, paper_f2, paper_f3, field_sincos, field_gauss_jump_2d,
                   linear_field([1.0, 2.0, -1.0]), lambda x: np.cos(3 * x[:, 0]) + x[:, 1],
                   lambda x: x[:, 0] * x[:, 1]]


def batch_workload(nreq: int = 256, seed: int = 5, scale: float = 1.0):
    """The batched workload: three sources carrying 8 fields each (the small
    and the large 2D source meshes, the 3D source mesh) and ``nreq`` requests
    from ``batch_requests``. 2D requests alternate between the two 2D
    sources, 3D requests use the 3D source. Targets are jittered structured
    meshes of the requested size (2 n^2 triangles or 6 n^3 tetrahedra; a
    Delaunay build for 32 M elements would dominate the run)."""
    f3 = [lambda x, f=f: f(x[:, :2]) + 0.5 * np.sign(x[:, 2] - 0.4) for f in BATCH_FIELDS_2D]
    n_small = max(2, int(round(32 * math.sqrt(scale))))
    n_big = max(2, int(round(1414 * math.sqrt(scale))))
    n_3d = max(2, int(round(94 * scale ** (1 / 3))))
    sources = [
        as_precision(with_values(jittered_tri_mesh(n_small, seed=0), BATCH_FIELDS_2D, np.float64), np.float32),
        as_precision(with_values(jittered_tri_mesh(n_big, seed=0), BATCH_FIELDS_2D, np.float64), np.float32),
        as_precision(with_values(jittered_kuhn_mesh(n_3d, seed=0), f3, np.float64), np.float32),
    ]
    reqs = batch_requests(nreq, seed, emin=1e4 * scale, emax=5e5 * scale)
    out = []
    k2 = 0
    for r, q in enumerate(reqs):
        if q["dim"] == 2:
            n = max(2, int(round(math.sqrt(q["elems"] / 2))))
            tgt = as_precision(jittered_tri_mesh(n, seed=1000 + r), np.float32)
            src = k2 % 2
            k2 += 1
        else:
            n = max(2, int(round((q["elems"] / 6) ** (1 / 3))))
            tgt = as_precision(jittered_kuhn_mesh(n, seed=1000 + r), np.float32)
            src = 2
        out.append(dict(q, source=src, target=tgt, elems=tgt.nelems))
    return sources, out


MLP_HIDDEN = 256
MLP_NPARAM = MLP_HIDDEN * 3 + MLP_HIDDEN + 3 * (MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN) + MLP_HIDDEN + 1


def mlp_init(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters of the surrogate network 3->256->256->256->256->1
    (layout: W1 [256][3], c1, W2 [256][256], c2, W3, c3, W4, c4, w5 [256], c5):
    uniform weights with He-uniform bounds sqrt(6/fan_in) (the first layer
    scaled up for the unit-box inputs), uniform first-layer biases, zero
    other biases."""
    rng = np.random.default_rng(seed)
    H = MLP_HIDDEN
    parts = [rng.uniform(-1, 1, (H, 3)) * 6.0,
             rng.uniform(-1, 1, H) * 3.0]
    for _ in range(3):
        parts += [rng.uniform(-1, 1, (H, H)) * math.sqrt(6.0 / H), np.zeros(H)]
    parts += [rng.uniform(-1, 1, H) * math.sqrt(3.0 / H), np.zeros(1)]
    out = np.concatenate([x.ravel() for x in parts])
    assert out.size == MLP_NPARAM
    return out


def batch_requests(nreq: int = 256, seed: int = 5, emin: float = 1e4, emax: float = 5e5):
    """The batched-transfer request list: per request the target dimension
    (50/50), the element count (log-uniform in [emin, emax]), the number of
    fields (1..8) and the samples per element (one of 8, 16, 32, 64, 128)."""
    rng = np.random.default_rng(seed)
    dims = rng.integers(2, 4, nreq)
    elems = np.exp(rng.uniform(math.log(emin), math.log(emax), nreq)).astype(np.int64)
    nf = rng.integers(1, 9, nreq)
    nsamp = rng.choice(np.array([8, 16, 32, 64, 128]), nreq)
    return [dict(dim=int(d), elems=int(e), nfields=int(f), samples_per_elem=int(s))
            for d, e, f, s in zip(dims, elems, nf, nsamp)]
