"""Python access to the FP64 CPU oracle (plain C, see ``oracle.h``).

TEST INFRASTRUCTURE ONLY: the oracle is the independent, slow, obviously
correct restatement of the paper's method that the CUDA library is checked
against. Only the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline / reference leg may import this package. It shares no code with
the CUDA library.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["rng_sample.c", "locate.c", "transfer.c", "clip.c", "mlp.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# plain ISO C, one rounding per operation: no contraction into FMA, no fast-math
CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
          "-fno-unsafe-math-optimizations", "-Wall"]


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (seconds)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES if os.path.exists(os.path.join(_HERE, s))]
    newest = max(os.path.getmtime(s) for s in srcs + [os.path.join(_HERE, "oracle.h")])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *CFLAGS, *srcs, "-o", tmp, "-lm"], check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = ctypes.CDLL(_LIB_PATH)
            _declare(_lib)
        return _lib


_i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int


class _Params(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("samples_per_elem", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("stream", ctypes.c_uint32),
                ("alpha", ctypes.c_double), ("grid_scale_L", ctypes.c_double),
                ("cg_tol", ctypes.c_double), ("cg_max_iter", ctypes.c_int), ("sampling", ctypes.c_int),
                ("adapt_ref_measure", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("cg_iters", ctypes.c_int), ("cg_rel_resid", ctypes.c_double),
                ("fallback_queries", ctypes.c_int64), ("empty_queries", ctypes.c_int64),
                ("samples", ctypes.c_int64)]


def _declare(L):
    L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.orc_u01_f32.argtypes = [ctypes.c_uint32]
    L.orc_u01_f32.restype = ctypes.c_float
    L.orc_u01_f64.argtypes = [ctypes.c_uint32]
    L.orc_u01_f64.restype = ctypes.c_double
    L.orc_sample_element.argtypes = [_int, _int, ctypes.c_uint64, ctypes.c_uint32, _i64,
                                     ctypes.c_int32, _f64p, _f64p, _f64p]
    L.orc_sample_element_w.argtypes = [_int, _int, ctypes.c_uint64, ctypes.c_uint32, _i64,
                                       ctypes.c_int32, _int, _f64p, _f64p, _f64p, _f64p]
    L.orc_adaptive_samples.argtypes = [_int, _f64p, ctypes.c_int32, ctypes.c_double]
    L.orc_adaptive_samples.restype = ctypes.c_int32
    L.orc_importance_weight.argtypes = [_int, _f64p]
    L.orc_importance_weight.restype = ctypes.c_double
    L.orc_sample_element_s.argtypes = [_int, _int, ctypes.c_uint64, ctypes.c_uint32, _i64,
                                       ctypes.c_int32, _int, _f64p, _f64p, _f64p]
    L.orc_strata_per_axis.argtypes = [_int, ctypes.c_int32]
    L.orc_strata_per_axis.restype = _int
    L.orc_grid_build.argtypes = [_int, _int, _i64, _f64p, _i64, _i32p, ctypes.c_double]
    L.orc_grid_build.restype = _vp
    L.orc_grid_free.argtypes = [_vp]
    L.orc_grid_shape.argtypes = [_vp, _i32p, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
    L.orc_grid_csr.argtypes = [_vp, _i64p, _i32p]
    L.orc_grid_locate.argtypes = [_vp, _i64, _f64p, _i32p, _i32p]
    L.orc_grid_depths.argtypes = [_vp, _f64p]
    L.orc_grid_adjacency.argtypes = [_vp, _i32p]
    L.orc_brute_locate.argtypes = [_int, _int, _i64, _f64p, _i64, _i32p, _i64, _f64p,
                                   _i32p, _i32p]
    L.orc_eval_p1.argtypes = [_int, _f64p, _i32p, _int, _i64, _f64p, ctypes.c_int32,
                              _f64p, _f64p]
    L.orc_mass_nnz.argtypes = [_int, _i64, _i64, _i32p]
    L.orc_mass_nnz.restype = _i64
    L.orc_mass_csr.argtypes = [_int, _i64, _f64p, _i64, _i32p, _i64p, _i32p, _f64p]
    L.orc_lumped_mass.argtypes = [_int, _i64, _f64p, _i64, _i32p, _f64p]
    L.orc_pcg.argtypes = [_i64, _i64p, _i32p, _f64p, _f64p, _f64p, ctypes.c_double, _int,
                          ctypes.POINTER(ctypes.c_double)]
    L.orc_pcg.restype = _int
    L.orc_transfer.argtypes = [_int, ctypes.POINTER(_Params),
                               _i64, _f64p, _i64, _i32p, _int, _f64p,
                               _i64, _f64p, _i64, _i32p,
                               _f64p, _f64p, _f64p, _f64p, _f64p, _vp,
                               ctypes.POINTER(_Stats)]
    L.orc_integral_p1.argtypes = [_int, _i64, _f64p, _i64, _i32p, _f64p]
    L.orc_integral_p1.restype = ctypes.c_double
    L.orc_mi_load_vector_2d.argtypes = [_i64, _f64p, _i64, _i32p, _f64p, _i64, _f64p, _i64,
                                        _i32p, _f64p]
    L.orc_l2_error_2d.argtypes = [_i64, _f64p, _i64, _i32p, _f64p, _i64, _f64p, _i64, _i32p,
                                  _f64p, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]
    if hasattr(L, "orc_mlp_forward"):
        _declare_mlp(L)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------------------
def philox4x32_10(ctr, key) -> np.ndarray:
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.ascontiguousarray(ctr, np.uint32),
                            np.ascontiguousarray(key, np.uint32), out)
    return out


def u01(x: int, prec: int) -> float:
    return float(lib().orc_u01_f32(x) if prec == 1 else lib().orc_u01_f64(x))


def sample_element_w(prec, dim, seed, stream, t, nsamp, node_xyz, sampling=0):
    """(lam [N][d+1], X [N][d], w [N]) of one element under any sampling scheme."""
    k = dim + 1
    lam = np.zeros((nsamp, k))
    X = np.zeros((nsamp, dim))
    w = np.zeros(nsamp)
    lib().orc_sample_element_w(prec, dim, seed, stream, t, nsamp, sampling, _f64(node_xyz).ravel(), lam, X, w)
    return lam, X, w


def adaptive_samples(dim, node_xyz, nsamp, ref_measure) -> int:
    return int(lib().orc_adaptive_samples(dim, _f64(node_xyz).ravel(), nsamp, float(ref_measure)))


def importance_weight(dim, lam) -> float:
    return float(lib().orc_importance_weight(dim, _f64(lam)))


def sample_element(prec, dim, seed, stream, t, nsamp, node_xyz, sampling=0):
    """Barycentric weights [nsamp, dim+1] and points [nsamp, dim] of the samples
    of target element t (sampling 0 uniform, 1 stratified)."""
    lam = np.zeros((nsamp, dim + 1))
    X = np.zeros((nsamp, dim))
    lib().orc_sample_element_s(prec, dim, seed, stream, t, nsamp, sampling, _f64(node_xyz), lam, X)
    return lam, X


def strata_per_axis(dim, nsamp) -> int:
    return int(lib().orc_strata_per_axis(dim, nsamp))


class Grid:
    """The oracle's uniform grid over a source mesh (build + locate)."""

    def __init__(self, prec, coords, conn, grid_scale_L=1.0):
        self.coords = _f64(coords)
        self.conn = _i32(conn)
        self.dim = self.coords.shape[1]
        self.prec = prec
        self._h = lib().orc_grid_build(prec, self.dim, self.coords.shape[0], self.coords,
                                       self.conn.shape[0], self.conn, grid_scale_L)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_grid_free(self._h)
            self._h = None

    def shape(self):
        n = np.zeros(3, np.int32)
        nc, ni = _i64(), _i64()
        lib().orc_grid_shape(self._h, n, ctypes.byref(nc), ctypes.byref(ni))
        return n, nc.value, ni.value

    def csr(self):
        _, nc, ni = self.shape()
        start = np.zeros(nc + 1, np.int64)
        items = np.zeros(max(ni, 1), np.int32)
        lib().orc_grid_csr(self._h, start, items)
        return start, items[:ni]

    def depths(self):
        _, _, ni = self.shape()
        out = np.zeros(max(ni, 1))
        lib().orc_grid_depths(self._h, out)
        return out[:ni]

    def adjacency(self):
        """[ne][dim+1] face neighbours: across the face opposite local vertex m, or -1"""
        out = np.zeros((self.conn.shape[0], self.dim + 1), np.int32)
        lib().orc_grid_adjacency(self._h, out)
        return out

    def locate(self, pts):
        pts = _f64(pts).reshape(-1, self.dim)
        e = np.zeros(pts.shape[0], np.int32)
        st = np.zeros(pts.shape[0], np.int32)
        lib().orc_grid_locate(self._h, pts.shape[0], pts, e, st)
        return e, st


def brute_locate(prec, coords, conn, pts):
    coords, conn = _f64(coords), _i32(conn)
    dim = coords.shape[1]
    pts = _f64(pts).reshape(-1, dim)
    e = np.zeros(pts.shape[0], np.int32)
    st = np.zeros(pts.shape[0], np.int32)
    lib().orc_brute_locate(prec, dim, coords.shape[0], coords, conn.shape[0], conn,
                           pts.shape[0], pts, e, st)
    return e, st


def eval_p1(coords, conn, values, e, X):
    coords, conn, values = _f64(coords), _i32(conn), _f64(np.atleast_2d(values))
    out = np.zeros(values.shape[0])
    lib().orc_eval_p1(coords.shape[1], coords, conn, values.shape[0], coords.shape[0], values,
                      int(e), _f64(X), out)
    return out


def mass_csr(coords, conn):
    coords, conn = _f64(coords), _i32(conn)
    dim, nv = coords.shape[1], coords.shape[0]
    nnz = lib().orc_mass_nnz(dim, nv, conn.shape[0], conn)
    rp = np.zeros(nv + 1, np.int64)
    col = np.zeros(nnz, np.int32)
    val = np.zeros(nnz)
    lib().orc_mass_csr(dim, nv, coords, conn.shape[0], conn, rp, col, val)
    return rp, col, val


def lumped_mass(coords, conn):
    coords, conn = _f64(coords), _i32(conn)
    m = np.zeros(coords.shape[0])
    lib().orc_lumped_mass(coords.shape[1], coords.shape[0], coords, conn.shape[0], conn, m)
    return m


def pcg(rp, col, val, b, tol=1e-12, max_iter=1000):
    b = _f64(b)
    x = np.zeros_like(b)
    rr = ctypes.c_double()
    it = lib().orc_pcg(b.shape[0], np.ascontiguousarray(rp, np.int64), _i32(col), _f64(val),
                       b, x, tol, max_iter, ctypes.byref(rr))
    return x, it, rr.value


def transfer(src, tgt, prec, samples_per_elem, seed=0, stream=0, alpha=1.0, grid_scale_L=1.0,
             cg_tol=1e-12, cg_max_iter=1000, want_sample_elem=False, sampling=0, adapt_ref_measure=0.0):
    """Steps 1-7 of Sec. 4 on the CPU; returns a dict of FP64 arrays.
    sampling: 0 uniform, 1 stratified, 2 importance; adapt_ref_measure > 0:
    per-element sample counts (sample_elem is then [E][8 N], -1 padded)."""
    sc, sconn, sv = _f64(src.coords), _i32(src.conn), _f64(src.values)
    tc, tconn = _f64(tgt.coords), _i32(tgt.conn)
    dim, nf = sc.shape[1], sv.shape[0]
    nvt, net = tc.shape[0], tconn.shape[0]
    p = _Params(prec, samples_per_elem, seed, stream, alpha, grid_scale_L, cg_tol, cg_max_iter, sampling,
                adapt_ref_measure)
    st = _Stats()
    out = {k: np.zeros((nf, nvt)) for k in ("g", "b_g", "b_res", "b", "u")}
    nmax = samples_per_elem * (8 if adapt_ref_measure > 0 else 1)
    se = np.zeros((net, nmax), np.int32) if want_sample_elem else None
    lib().orc_transfer(dim, ctypes.byref(p), sc.shape[0], sc, sconn.shape[0], sconn, nf, sv,
                       nvt, tc, net, tconn, out["g"], out["b_g"], out["b_res"], out["b"],
                       out["u"], None if se is None else se.ctypes.data_as(_vp),
                       ctypes.byref(st))
    out.update(cg_iters=st.cg_iters, cg_rel_resid=st.cg_rel_resid,
               fallback_queries=st.fallback_queries, empty_queries=st.empty_queries, samples=st.samples)
    if se is not None:
        out["sample_elem"] = se
    return out


def integral_p1(coords, conn, values):
    coords, conn = _f64(coords), _i32(conn)
    return lib().orc_integral_p1(coords.shape[1], coords.shape[0], coords, conn.shape[0],
                                 conn, _f64(values))


def mi_load_vector_2d(src, tgt, field=0):
    sc, tc = _f64(src.coords), _f64(tgt.coords)
    b = np.zeros(tc.shape[0])
    lib().orc_mi_load_vector_2d(sc.shape[0], sc, src.conn.shape[0], _i32(src.conn),
                                _f64(src.values[field]), tc.shape[0], tc, tgt.conn.shape[0],
                                _i32(tgt.conn), b)
    return b


def l2_error_2d(src, tgt, tgt_values, field=0):
    sc, tc = _f64(src.coords), _f64(tgt.coords)
    e, n = ctypes.c_double(), ctypes.c_double()
    lib().orc_l2_error_2d(sc.shape[0], sc, src.conn.shape[0], _i32(src.conn),
                          _f64(src.values[field]), tc.shape[0], tc, tgt.conn.shape[0],
                          _i32(tgt.conn), _f64(tgt_values), ctypes.byref(e), ctypes.byref(n))
    return e.value, n.value


def roundtrip(mesh1, mesh2, f_ref, iters, prec, samples_per_elem, seeds=(0, 1), alpha=1.0, cg_tol=1e-12,
              cg_max_iter=1000, sampling=0, exact=False):
    """Repeated round trips mesh1 -> mesh2 -> mesh1 of a nodal field (the
    iterative analysis of Sec. 5): transfer i of the first leg uses
    seeds[0], of the second leg seeds[1], so every round trip draws the same
    samples (the fixed-sample online mode). exact=True replaces the Monte
    Carlo load vector by the mesh-intersection one (2D only), i.e. repeated
    exact Galerkin projections. Returns (errors, field): errors[k] =
    (E_l2, E_mass) after round trip k + 1, E_l2 the discrete l2 error of the
    nodal values and E_mass the conservation error of the P1 integral on
    mesh 1 (exact quadrature: sum_i m_i f_i with the lumped masses), both
    relative to f_ref."""
    f_ref = _f64(f_ref)
    m1 = lumped_mass(mesh1.coords, mesh1.conn)
    i_ref = float(m1 @ f_ref)
    if exact:
        csr1, csr2 = mass_csr(mesh2.coords, mesh2.conn), mass_csr(mesh1.coords, mesh1.conn)

    def leg(src_mesh, tgt_mesh, vals, seed, csr):
        src = _Mesh(src_mesh.coords, src_mesh.conn, vals[None, :])
        if exact:
            b = mi_load_vector_2d(src, tgt_mesh)
            u, _, _ = pcg(*csr, b, tol=cg_tol, max_iter=cg_max_iter)
            return u
        return transfer(src, tgt_mesh, prec, samples_per_elem, seed=seed, stream=0, alpha=alpha, cg_tol=cg_tol,
                        cg_max_iter=cg_max_iter, sampling=sampling)["u"][0]

    f = f_ref.copy()
    errors = []
    for _ in range(iters):
        g = leg(mesh1, mesh2, f, seeds[0], csr1 if exact else None)
        f = leg(mesh2, mesh1, g, seeds[1], csr2 if exact else None)
        e_l2 = float(np.linalg.norm(f - f_ref) / np.linalg.norm(f_ref))
        e_mass = abs(float(m1 @ f) - i_ref) / abs(i_ref)
        errors.append((e_l2, e_mass))
    return errors, f


class _Mesh:
    """coords, conn, values: the attributes transfer() reads from a mesh."""

    def __init__(self, coords, conn, values):
        self.coords, self.conn, self.values = coords, conn, values


def _declare_mlp(L):
    L.orc_mlp_nparam.restype = _i64
    L.orc_bf16_round.argtypes = [ctypes.c_double]
    L.orc_bf16_round.restype = ctypes.c_double
    L.orc_mlp_forward.argtypes = [_f64p, _i64, _f64p, _int, _f64p]
    L.orc_mlp_loss_grad.argtypes = [_f64p, _i64, _f64p, _f64p, _int, _f64p]
    L.orc_mlp_loss_grad.restype = ctypes.c_double
    L.orc_adam_step.argtypes = [_i64, _f64p, _f64p, _f64p, _f64p, _i64, ctypes.c_double, ctypes.c_double,
                                ctypes.c_double, ctypes.c_double]


MLP_H = 256


def mlp_nparam() -> int:
    return int(lib().orc_mlp_nparam())


def mlp_split(params):
    """Views of the parameter vector: W1 [256,3], c1, W2, c2, W3, c3, W4, c4, w5 [256], c5 [1]."""
    H = MLP_H
    sizes = [H * 3, H, H * H, H, H * H, H, H * H, H, H, 1]
    shapes = [(H, 3), (H,), (H, H), (H,), (H, H), (H,), (H, H), (H,), (H,), (1,)]
    out, o = [], 0
    for n, sh in zip(sizes, shapes):
        out.append(params[o:o + n].reshape(sh))
        o += n
    return out


def bf16_round(x: float) -> float:
    return float(lib().orc_bf16_round(float(x)))


def mlp_forward(params, X, act_bf16=False):
    X = _f64(X).reshape(-1, 3)
    y = np.zeros(X.shape[0])
    lib().orc_mlp_forward(_f64(params), X.shape[0], X, int(act_bf16), y)
    return y


def mlp_loss_grad(params, X, t, act_bf16=False):
    X = _f64(X).reshape(-1, 3)
    g = np.zeros(mlp_nparam())
    loss = lib().orc_mlp_loss_grad(_f64(params), X.shape[0], X, _f64(t), int(act_bf16), g)
    return loss, g


def adam_step(params, grad, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """In place on params, m, v (float64 arrays)."""
    lib().orc_adam_step(params.size, params, _f64(grad), m, v, int(t), lr, beta1, beta2, eps)
