"""Python binding of libsft (include/sft.h): argument marshalling only.

Every step of the transfer runs in the CUDA library. The functions carry the
names of the C entry points. Arrays may be numpy arrays (host memory) or torch
tensors (host or CUDA); CUDA tensors are passed to the library as device
pointers on the current torch stream.

The library is required: importing works without it (so the build step can
run), but every call raises ``SftUnavailable`` when ``libsft.so`` is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsft.so")

(SFT_OK, SFT_ERR_ARG, SFT_ERR_MESH, SFT_ERR_CUDA, SFT_ERR_OOM, SFT_ERR_NOT_CONVERGED, SFT_ERR_OUTSIDE,
 SFT_ERR_DEVICE_STATUS, SFT_ERR_UNSUPPORTED) = range(9)
SFT_PREC_FP64, SFT_PREC_FP32 = 0, 1
SFT_CG_MIXED, SFT_CG_FP64 = 0, 1
SFT_SAMPLING_UNIFORM, SFT_SAMPLING_STRATIFIED, SFT_SAMPLING_IMPORTANCE = 0, 1, 2
SFT_F32, SFT_F64 = 0, 1


class SftUnavailable(RuntimeError):
    pass


class SftError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({msg})")
        self.status = status


class sft_mesh_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("nfields", ctypes.c_int32), ("nnodes", ctypes.c_int64),
                ("nelems", ctypes.c_int64), ("coords", ctypes.c_void_p), ("conn", ctypes.c_void_p),
                ("values", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("device_ptrs", ctypes.c_int32),
                ("grid_scale_L", ctypes.c_double), ("cuda_stream", ctypes.c_void_p)]


class sft_options(ctypes.Structure):
    _fields_ = [("samples_per_elem", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("stream_id", ctypes.c_uint32), ("cg_max_iter", ctypes.c_int32),
                ("alpha", ctypes.c_double), ("cg_tol", ctypes.c_double), ("strict_inside", ctypes.c_int32),
                ("out_device", ctypes.c_int32), ("cuda_stream", ctypes.c_void_p),
                ("sample_elem_out", ctypes.c_void_p), ("field_count", ctypes.c_int32),
                ("cg_mode", ctypes.c_int32), ("sampling", ctypes.c_int32), ("cg_warm_start", ctypes.c_int32),
                ("adapt_ref_measure", ctypes.c_double)]


class sft_stats(ctypes.Structure):
    _fields_ = [("cg_iters", ctypes.c_int32), ("reserved", ctypes.c_int32), ("cg_rel_resid", ctypes.c_double),
                ("queries", ctypes.c_int64), ("fallback_queries", ctypes.c_int64),
                ("empty_queries", ctypes.c_int64), ("ms_setup", ctypes.c_float), ("ms_control", ctypes.c_float),
                ("ms_assembly", ctypes.c_float), ("ms_solve", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("reserved2", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


class sft_batch_stats(ctypes.Structure):
    _fields_ = [("nreq", ctypes.c_int32), ("graph", ctypes.c_int32), ("max_cg_iters", ctypes.c_int32),
                ("nonconverged", ctypes.c_int32), ("max_rel_resid", ctypes.c_double),
                ("queries", ctypes.c_int64), ("fallback_queries", ctypes.c_int64),
                ("empty_queries", ctypes.c_int64), ("ms_control", ctypes.c_float),
                ("ms_assembly", ctypes.c_float), ("ms_solve", ctypes.c_float), ("ms_total", ctypes.c_float),
                ("tile", ctypes.c_int32 * 6)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "tile"}
        d["tile"] = list(self.tile)
        return d


class sft_surrogate_opts(ctypes.Structure):
    _fields_ = [("exact_field", ctypes.c_int32), ("subsample", ctypes.c_int32), ("tau", ctypes.c_float),
                ("exact_cost", ctypes.c_int32), ("fallback_out", ctypes.c_void_p), ("sample_f_out", ctypes.c_void_p)]


class sft_surrogate_stats(ctypes.Structure):
    _fields_ = [("cg_iters", ctypes.c_int32), ("reserved", ctypes.c_int32), ("cg_rel_resid", ctypes.c_double),
                ("net_queries", ctypes.c_int64), ("exact_queries", ctypes.c_int64),
                ("fallback_elems", ctypes.c_int64), ("empty_queries", ctypes.c_int64),
                ("ms_control", ctypes.c_float), ("ms_assembly", ctypes.c_float), ("ms_solve", ctypes.c_float),
                ("ms_total", ctypes.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if not k.startswith("reserved")}


_vp, _i32, _i64, _d = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGS = {
    "sft_source_create": ([ctypes.POINTER(sft_mesh_desc), ctypes.POINTER(_vp)], _i32),
    "sft_target_create": ([ctypes.POINTER(sft_mesh_desc), ctypes.POINTER(_vp)], _i32),
    "sft_source_destroy": ([_vp], None),
    "sft_source_set_values": ([_vp, _vp, _i32, _vp], _i32),
    "sft_target_destroy": ([_vp], None),
    "sft_transfer": ([_vp, _vp, ctypes.POINTER(sft_options), _vp, _vp, _vp, ctypes.POINTER(sft_stats)], _i32),
    "sft_conservation_error": ([_vp, _vp, _vp, _i32, _i32, _vp, _vp], _i32),
    "sft_locate": ([_vp, _i32, _i64, _vp, _i32, _vp, _vp, _vp], _i32),
    "sft_mass_solve": ([_vp, _i32, _vp, _vp, _i32, _d, _i32, _i32, _vp, _vp, _vp], _i32),
    "sft_source_grid": ([_vp, _i32, _vp, _vp, _vp, _vp, _vp], _i32),
    "sft_source_adjacency": ([_vp, _i32, _vp], _i32),
    "sft_source_cell_first": ([_vp, _i32, _vp], _i32),
    "sft_target_set_wait_limit": ([_vp, ctypes.c_double], _i32),
    "sft_trim_memory": ([], _i32),
    "sft_batch_groups": ([_vp, _vp], _i32),
    "sft_mi_load_vector": ([_vp, _vp, _i32, _vp, _i32, _vp], _i32),
    "sft_mi_l2_error": ([_vp, _vp, _i32, _vp, _i32, _vp, _vp], _i32),
    "sft_target_mass": ([_vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "sft_status_str": ([_i32], ctypes.c_char_p),
    "sft_last_error": ([], ctypes.c_char_p),
    "sft_kernel_launches": ([], _i64),
    "sft_batch_create": ([_i32, _vp, _vp, _vp, _i32, _vp, _vp], _i32),
    "sft_batch_run": ([_vp, _vp, ctypes.POINTER(sft_batch_stats)], _i32),
    "sft_batch_result": ([_vp, _i32, _vp, _vp, _i32, _vp], _i32),
    "sft_batch_destroy": ([_vp], None),
    "sft_mlp_nparam": ([], _i64),
    "sft_mlp_create": ([_vp, _i32, _vp, _vp], _i32),
    "sft_mlp_params": ([_vp, _vp, _i32, _vp], _i32),
    "sft_mlp_forward": ([_vp, _i64, _vp, _vp, _i32, _vp], _i32),
    "sft_mlp_destroy": ([_vp], None),
    "sft_mlp_loss_grad": ([_vp, _i64, _vp, _vp, _vp, _vp, _i32, _vp], _i32),
    "sft_mlp_train": ([_vp, _i64, _vp, _vp, _i32, _i32, ctypes.c_float, ctypes.c_float, _vp, _i32, _vp], _i32),
    "sft_transfer_surrogate": ([_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp], _i32),
    "sft_plan_create": ([_vp, _vp, _vp, _vp], _i32),
    "sft_plan_transfer": ([_vp, _vp, _vp, _vp, _vp], _i32),
    "sft_plan_bytes": ([_vp], _i64),
    "sft_plan_destroy": ([_vp], None),
    "sft_surrogate_dataset": ([_vp, _i32, _i64, ctypes.c_uint64, ctypes.c_uint32, _vp, _vp, _vp, _vp, _vp, _vp],
                              _i32),
    "sft_mass_solve_static": ([_i64, _vp, _vp, _vp, _i32, _vp, _vp, _d, _i32, _vp, _vp, _vp], _i32),
}
EXPORTS = tuple(_SIGS)
_lib = None


def lib() -> ctypes.CDLL:
    """Load libsft.so (raises SftUnavailable if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise SftUnavailable(f"libsft.so not built (expected at {LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(status: int, where: str, allow=(SFT_OK,)):
    if status not in allow:
        raise SftError(status, where, lib().sft_last_error().decode())
    return status


# --------------------------------------------------------------------------
# array marshalling (no arithmetic)
# --------------------------------------------------------------------------
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, on_device, keepalive) of a numpy array or torch tensor."""
    if x is None:
        return None, False, None
    if _is_torch(x):
        x = x.contiguous()
        return x.data_ptr(), bool(x.is_cuda), x
    x = np.ascontiguousarray(x)
    return x.ctypes.data, False, x


def _dtype_code(x):
    name = str(x.dtype)
    if name.endswith("float64"):
        return SFT_F64
    if name.endswith("float32"):
        return SFT_F32
    raise TypeError(f"coordinates must be float32 or float64, got {x.dtype}")


def _current_stream():
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def _int32(x):
    if _is_torch(x):
        import torch
        return x.to(torch.int32).contiguous()
    return np.ascontiguousarray(x, dtype=np.int32)


class _Handle:
    def __init__(self, h, destroy, keep):
        self.h = h
        self._destroy = destroy
        self._keep = keep

    def close(self):
        if self.h:
            self._destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Source(_Handle):
    pass


class Target(_Handle):
    pass


def _desc(coords, conn, values, grid_scale_L, stream):
    conn = _int32(conn)
    cp, cdev, ck = _ptr(coords)
    kp, kdev, kk = _ptr(conn)
    vp, vdev, vk = _ptr(values)
    if values is not None and _dtype_code(values) != _dtype_code(coords):
        raise TypeError("values must have the coordinates' dtype")
    if len({cdev, kdev} | ({vdev} if values is not None else set())) != 1:
        raise ValueError("coords, conn and values must all be host or all device arrays")
    d = sft_mesh_desc()
    d.dim = int(coords.shape[1])
    d.nfields = 0 if values is None else int(values.shape[0])
    d.nnodes = int(coords.shape[0])
    d.nelems = int(conn.shape[0])
    d.coords, d.conn, d.values = cp, kp, vp
    d.dtype = _dtype_code(coords)
    d.device_ptrs = int(cdev)
    d.grid_scale_L = float(grid_scale_L)
    d.cuda_stream = stream if stream is not None else (_current_stream() if cdev else None)
    return d, (ck, kk, vk)


def sft_source_create(coords, conn, values, grid_scale_L=1.0, stream=None) -> Source:
    """Source mesh + nodal fields -> handle with its point-location grid."""
    d, keep = _desc(coords, conn, values, grid_scale_L, stream)
    h = _vp()
    _check(lib().sft_source_create(ctypes.byref(d), ctypes.byref(h)), "sft_source_create")
    return Source(h.value, lib().sft_source_destroy, keep)


def sft_target_create(coords, conn, stream=None) -> Target:
    """Target mesh -> handle with its FP64 CSR mass matrix."""
    d, keep = _desc(coords, conn, None, 1.0, stream)
    h = _vp()
    _check(lib().sft_target_create(ctypes.byref(d), ctypes.byref(h)), "sft_target_create")
    return Target(h.value, lib().sft_target_destroy, keep)


def sft_source_set_values(src: Source, values, stream=None):
    """Replace the source's nodal values [nfields, nnodes] (same dtype)."""
    vp, dev, keep = _ptr(values)
    _check(lib().sft_source_set_values(src.h, vp, int(dev), stream if stream is not None else _current_stream()),
           "sft_source_set_values")


def sft_source_destroy(src: Source):
    src.close()


def sft_target_destroy(tgt: Target):
    tgt.close()


def sft_transfer(src: Source, tgt: Target, samples_per_elem: int, precision: int = SFT_PREC_FP32,
                 seed: int = 0, stream_id: int = 0, alpha: float = 1.0, cg_tol: float = 1e-10,
                 cg_max_iter: int = 1000, strict_inside: bool = False, u_out=None, b_out=None, g_out=None,
                 sample_elem_out=None, stream=None, allow_not_converged: bool = False, field_count: int = 0,
                 cg_mode: int = SFT_CG_MIXED, sampling: int = SFT_SAMPLING_UNIFORM, cg_warm_start: bool = False,
                 adapt_ref_measure: float = 0.0):
    """Run one transfer. Outputs are caller-provided arrays (numpy for host,
    torch CUDA tensors for device); when u_out is None a host array
    [nfields, nnodes] is allocated. sample_elem_out is [nelems, N], or
    [nelems, 8 N] with adapt_ref_measure > 0. Returns (status, stats dict, u_out)."""
    nf = int(field_count) if field_count > 0 else _nf(src)
    if u_out is None:
        u_out = np.zeros((nf, _nv(tgt)), np.float64)
    up, udev, _ = _ptr(u_out)
    bp, bdev, _ = _ptr(b_out)
    gp, gdev, _ = _ptr(g_out)
    sp, sdev, _ = _ptr(sample_elem_out)
    for p, dv in ((bp, bdev), (gp, gdev), (sp, sdev)):
        if p is not None and dv != udev:
            raise ValueError("all outputs must be host arrays or all device tensors")
    o = sft_options()
    o.samples_per_elem = int(samples_per_elem)
    o.precision = int(precision)
    o.seed = int(seed)
    o.stream_id = int(stream_id)
    o.cg_max_iter = int(cg_max_iter)
    o.alpha = float(alpha)
    o.cg_tol = float(cg_tol)
    o.strict_inside = int(bool(strict_inside))
    o.out_device = int(udev)
    o.cuda_stream = stream if stream is not None else _current_stream()
    o.sample_elem_out = sp
    o.field_count = int(field_count)
    o.cg_mode = int(cg_mode)
    o.sampling = int(sampling)
    o.cg_warm_start = int(bool(cg_warm_start))
    o.adapt_ref_measure = float(adapt_ref_measure)
    st = sft_stats()
    allow = (SFT_OK, SFT_ERR_NOT_CONVERGED) if allow_not_converged else (SFT_OK,)
    status = _check(lib().sft_transfer(src.h, tgt.h, ctypes.byref(o), up, bp, gp, ctypes.byref(st)),
                    "sft_transfer", allow)
    return status, st.as_dict(), u_out


class Plan(_Handle):
    pass


def sft_plan_create(src: Source, tgt: Target, samples_per_elem: int, precision: int = SFT_PREC_FP32, seed: int = 0,
                    stream_id: int = 0, alpha: float = 1.0, cg_tol: float = 1e-10, cg_max_iter: int = 1000,
                    field_count: int = 0, out_device: bool = False, strict_inside: bool = False,
                    stream=None, cg_mode: int = SFT_CG_MIXED, sampling: int = SFT_SAMPLING_UNIFORM,
                    cg_warm_start: bool = False) -> Plan:
    """Initialization of a transfer between fixed meshes (node and sample
    locations recorded); outputs of later transfers go to host arrays, or to
    CUDA tensors with out_device=True."""
    o = _options(samples_per_elem, seed, stream_id, alpha, cg_tol, cg_max_iter, field_count, precision, cg_mode,
                 sampling, cg_warm_start)
    o.out_device = int(bool(out_device))
    o.strict_inside = int(bool(strict_inside))
    o.cuda_stream = stream if stream is not None else _current_stream()
    h = _vp()
    _check(lib().sft_plan_create(src.h, tgt.h, ctypes.byref(o), ctypes.byref(h)), "sft_plan_create")
    pl = Plan(h.value, lib().sft_plan_destroy, (src, tgt))
    pl.nfields = int(field_count) if field_count > 0 else _nf(src)
    pl.nnodes = _nv(tgt)
    return pl


def sft_plan_transfer(pl: Plan, u_out=None, b_out=None, g_out=None, allow_not_converged: bool = False):
    """Online transfer with the source's current values. Returns (status, stats dict, u_out)."""
    if u_out is None:
        u_out = np.zeros((pl.nfields, pl.nnodes), np.float64)
    st = sft_stats()
    allow = (SFT_OK, SFT_ERR_NOT_CONVERGED) if allow_not_converged else (SFT_OK,)
    status = _check(lib().sft_plan_transfer(pl.h, _ptr(u_out)[0], _ptr(b_out)[0], _ptr(g_out)[0], ctypes.byref(st)),
                    "sft_plan_transfer", allow)
    return status, st.as_dict(), u_out


def sft_plan_bytes(pl: Plan) -> int:
    return int(lib().sft_plan_bytes(pl.h))


def sft_conservation_error(src: Source, tgt: Target, u, field: int = 0, stream=None):
    """(E_mass, int f^s, int f^t) for one target field u [nnodes]."""
    p, dev, _ = _ptr(u)
    out = (ctypes.c_double * 3)()
    _check(lib().sft_conservation_error(src.h, tgt.h, p, int(dev), int(field),
                                        stream if stream is not None else _current_stream(), out),
           "sft_conservation_error")
    return out[0], out[1], out[2]


def sft_mi_load_vector(src: Source, tgt: Target, field: int = 0, b_out=None, stream=None):
    """Exact load vector int psi_i f^s by 2D mesh intersection (FP64 [nnodes])."""
    if b_out is None:
        b_out = np.zeros(_nv(tgt), np.float64)
    p, dev, _ = _ptr(b_out)
    _check(lib().sft_mi_load_vector(src.h, tgt.h, int(field), p, int(dev),
                                    stream if stream is not None else _current_stream()), "sft_mi_load_vector")
    return b_out


def sft_mi_l2_error(src: Source, tgt: Target, u, field: int = 0, stream=None):
    """(||f^s - f^t||_L2, ||f^s||_L2) on the supermesh (2D) for a target field u [nnodes]."""
    p, dev, _ = _ptr(u)
    out = (ctypes.c_double * 2)()
    _check(lib().sft_mi_l2_error(src.h, tgt.h, int(field), p, int(dev),
                                 stream if stream is not None else _current_stream(), out), "sft_mi_l2_error")
    return out[0], out[1]


def sft_locate(src: Source, pts, precision: int = SFT_PREC_FP32, elem_out=None, val_out=None, stream=None):
    """Locate FP64 points [n, dim]; returns (elem [n], values [nfields, n])."""
    n = int(pts.shape[0])
    pp, dev, _ = _ptr(pts)
    if elem_out is None:
        elem_out = np.zeros(n, np.int32)
    if val_out is None:
        val_out = np.zeros((_nf(src), n), np.float64)
    ep, _, _ = _ptr(elem_out)
    vp, _, _ = _ptr(val_out)
    _check(lib().sft_locate(src.h, int(precision), n, pp, int(dev), ep, vp,
                            stream if stream is not None else _current_stream()), "sft_locate")
    return elem_out, val_out


def sft_mass_solve(tgt: Target, b, tol=1e-12, max_iter=1000, u_out=None, stream=None, cg_mode=SFT_CG_MIXED):
    """Solve M u = b for b [nrhs, nnodes]; returns (u, iters, rel_resid)."""
    b2 = b if _is_torch(b) else np.ascontiguousarray(np.atleast_2d(b), np.float64)
    nrhs = int(b2.shape[0]) if b2.ndim == 2 else 1
    bp, dev, keep = _ptr(b2)
    if u_out is None:
        u_out = np.zeros((nrhs, _nv(tgt)), np.float64)
    up, _, _ = _ptr(u_out)
    it = ctypes.c_int32()
    rr = ctypes.c_double()
    _check(lib().sft_mass_solve(tgt.h, nrhs, bp, up, int(dev), float(tol), int(max_iter), int(cg_mode),
                                stream if stream is not None else _current_stream(),
                                ctypes.byref(it), ctypes.byref(rr)), "sft_mass_solve")
    return u_out, it.value, rr.value


def sft_mass_solve_static(row_ptr, col, val, b, u_out, tol=1e-12, max_iter=1000, stream=None):
    """Allocation-free solve of M u = b (all arguments CUDA tensors: row_ptr
    int32 [n+1], col int32, val float64, b and u_out float64 [nrhs, n]).
    Returns (iters, rel_resid).

    The arguments are checked here before any pointer reaches the library,
    which trusts them: dtypes (an int64 row_ptr read as int32 would give a
    wrong answer), shapes (a b or u_out shorter than nrhs x n would be read
    or written past its end), one device, a contiguous u_out (a copy would
    receive the solution and drop it) and col / val holding row_ptr[n]
    entries. ValueError / TypeError otherwise."""
    import torch
    args = dict(row_ptr=row_ptr, col=col, val=val, b=b, u_out=u_out)
    for name, x in args.items():
        if not (_is_torch(x) and x.is_cuda):
            raise ValueError(f"sft_mass_solve_static: {name} must be a CUDA tensor")
    want = dict(row_ptr=torch.int32, col=torch.int32, val=torch.float64, b=torch.float64, u_out=torch.float64)
    for name, dt in want.items():
        if args[name].dtype != dt:
            raise TypeError(f"sft_mass_solve_static: {name} must be {dt}, got {args[name].dtype}")
    if len({x.device for x in args.values()}) != 1:
        raise ValueError("sft_mass_solve_static: all tensors must be on one device")
    if row_ptr.dim() != 1 or row_ptr.shape[0] < 2 or col.dim() != 1 or val.dim() != 1:
        raise ValueError("sft_mass_solve_static: row_ptr [n+1] (n >= 1), col and val must be 1-D")
    n = int(row_ptr.shape[0]) - 1
    if b.shape != u_out.shape or b.dim() not in (1, 2) or b.shape[-1] != n:
        raise ValueError(f"sft_mass_solve_static: b and u_out must both be [nrhs, {n}] or [{n}], "
                         f"got {tuple(b.shape)} and {tuple(u_out.shape)}")
    if not u_out.is_contiguous():
        raise ValueError("sft_mass_solve_static: u_out must be contiguous (the solution is written in place)")
    nnz = int(row_ptr[-1])
    if int(row_ptr[0]) != 0 or nnz < 0 or col.numel() < nnz or val.numel() < nnz:
        raise ValueError(f"sft_mass_solve_static: row_ptr[0] must be 0 and col / val hold row_ptr[n] = {nnz} "
                         f"entries, got {col.numel()} / {val.numel()}")
    nrhs = int(b.shape[0]) if b.dim() == 2 else 1
    ptrs = [_ptr(x) for x in (row_ptr, col, val, b, u_out)]
    it = ctypes.c_int32()
    rr = ctypes.c_double()
    _check(lib().sft_mass_solve_static(n, ptrs[0][0], ptrs[1][0], ptrs[2][0], nrhs, ptrs[3][0], ptrs[4][0],
                                       float(tol), int(max_iter),
                                       stream if stream is not None else _current_stream(),
                                       ctypes.byref(it), ctypes.byref(rr)), "sft_mass_solve_static")
    return it.value, rr.value


class Batch(_Handle):
    pass


def _options(samples_per_elem, seed=0, stream_id=0, alpha=1.0, cg_tol=1e-10, cg_max_iter=1000,
             field_count=0, precision=SFT_PREC_FP32, cg_mode=SFT_CG_MIXED, sampling=SFT_SAMPLING_UNIFORM,
             cg_warm_start=False, adapt_ref_measure=0.0):
    o = sft_options()
    o.samples_per_elem = int(samples_per_elem)
    o.precision = int(precision)
    o.seed = int(seed)
    o.stream_id = int(stream_id)
    o.cg_max_iter = int(cg_max_iter)
    o.alpha = float(alpha)
    o.cg_tol = float(cg_tol)
    o.field_count = int(field_count)
    o.cg_mode = int(cg_mode)
    o.sampling = int(sampling)
    o.cg_warm_start = int(bool(cg_warm_start))
    o.adapt_ref_measure = float(adapt_ref_measure)
    return o


def sft_batch_create(sources, targets, options, autotune=True, stream=None) -> Batch:
    """Plan of len(sources) transfers; options: list of dicts for _options()."""
    n = len(sources)
    srcs = (ctypes.c_void_p * n)(*[s.h for s in sources])
    tgts = (ctypes.c_void_p * n)(*[t.h for t in targets])
    opts = (sft_options * n)(*[_options(**o) for o in options])
    h = _vp()
    _check(lib().sft_batch_create(n, srcs, tgts, opts, int(bool(autotune)),
                                  stream if stream is not None else _current_stream(), ctypes.byref(h)),
           "sft_batch_create")
    b = Batch(h.value, lib().sft_batch_destroy, (list(sources), list(targets)))
    b.nfields = [int(o.get("field_count", 0)) or _nf(s) for o, s in zip(options, sources)]
    b.nnodes = [_nv(t) for t in targets]
    return b


def sft_batch_run(batch: Batch, stream=None, allow_not_converged=False):
    st = sft_batch_stats()
    allow = (SFT_OK, SFT_ERR_NOT_CONVERGED) if allow_not_converged else (SFT_OK,)
    status = _check(lib().sft_batch_run(batch.h, stream if stream is not None else _current_stream(),
                                        ctypes.byref(st)), "sft_batch_run", allow)
    return status, st.as_dict()


def sft_batch_result(batch: Batch, req: int, u_out=None, b_out=None, stream=None):
    if u_out is None:
        u_out = np.zeros((batch.nfields[req], batch.nnodes[req]))
    up, dev, _ = _ptr(u_out)
    bp, _, _ = _ptr(b_out)
    _check(lib().sft_batch_result(batch.h, int(req), up, bp, int(dev),
                                  stream if stream is not None else _current_stream()), "sft_batch_result")
    return u_out, b_out


def sft_batch_destroy(batch: Batch):
    batch.close()


class RoundTrip:
    """Repeated round trips mesh 1 -> mesh 2 -> mesh 1 of one nodal field (the
    iterative analysis of Sec. 5) through two transfer plans (initialization
    once; every round trip reuses the recorded samples). src1/tgt1 and
    src2/tgt2 are the same meshes as sources (one FP64 field) and targets.
    run(f, iters) maps the CUDA tensor f [1, nnodes1] (float64) in place.
    warm_start: each leg's solve starts from that leg's previous result (the
    field it is about to overwrite) instead of 0."""

    def __init__(self, src1: Source, tgt1: Target, src2: Source, tgt2: Target, samples_per_elem: int,
                 precision: int = SFT_PREC_FP32, seeds=(0, 1), alpha: float = 1.0, cg_tol: float = 1e-10,
                 cg_max_iter: int = 1000, sampling: int = SFT_SAMPLING_UNIFORM, cg_mode: int = SFT_CG_MIXED,
                 warm_start: bool = False):
        import torch
        if _nf(src1) != 1 or _nf(src2) != 1:
            raise ValueError("round-trip sources carry exactly one field")
        kw = dict(alpha=alpha, cg_tol=cg_tol, cg_max_iter=cg_max_iter, out_device=True, sampling=sampling,
                  cg_mode=cg_mode, cg_warm_start=warm_start)
        self.src1, self.src2 = src1, src2
        self.p12 = sft_plan_create(src1, tgt2, samples_per_elem, precision, seed=seeds[0], **kw)
        self.p21 = sft_plan_create(src2, tgt1, samples_per_elem, precision, seed=seeds[1], **kw)
        self.g = torch.zeros((1, _nv(tgt2)), dtype=torch.float64, device=torch.device("cuda",
                                                                                       torch.cuda.current_device()))
        self.queries = 0

    def run(self, f, iters: int = 1):
        for _ in range(iters):
            sft_source_set_values(self.src1, f)
            _, st, _ = sft_plan_transfer(self.p12, u_out=self.g)
            q = st["queries"]
            sft_source_set_values(self.src2, self.g)
            _, st, _ = sft_plan_transfer(self.p21, u_out=f)
            self.queries = q + st["queries"]
        return f

    def close(self):
        self.p12.close()
        self.p21.close()


class Mlp(_Handle):
    pass


def sft_mlp_nparam() -> int:
    return int(lib().sft_mlp_nparam())


def sft_mlp_create(params, stream=None) -> Mlp:
    """Network handle from an FP32 parameter vector (numpy or torch)."""
    p = params if _is_torch(params) else np.ascontiguousarray(params, np.float32)
    pp, dev, keep = _ptr(p)
    h = _vp()
    _check(lib().sft_mlp_create(pp, int(dev), stream if stream is not None else _current_stream(),
                                ctypes.byref(h)), "sft_mlp_create")
    return Mlp(h.value, lib().sft_mlp_destroy, None)


def sft_mlp_params(m: Mlp, out=None, stream=None):
    if out is None:
        out = np.zeros(sft_mlp_nparam(), np.float32)
    op, dev, _ = _ptr(out)
    _check(lib().sft_mlp_params(m.h, op, int(dev), stream if stream is not None else _current_stream()),
           "sft_mlp_params")
    return out


def sft_mlp_forward(m: Mlp, pts, out=None, stream=None):
    """Network values at pts [n, 3] (float32, numpy or CUDA tensor)."""
    n = int(pts.shape[0])
    if out is None:
        out = np.zeros(n, np.float32)
    pp, dev, _ = _ptr(pts if _is_torch(pts) else np.ascontiguousarray(pts, np.float32))
    op, _, _ = _ptr(out)
    _check(lib().sft_mlp_forward(m.h, n, pp, op, int(dev), stream if stream is not None else _current_stream()),
           "sft_mlp_forward")
    return out


def _cuda_f32(x, name):
    if not (_is_torch(x) and x.is_cuda and str(x.dtype).endswith("float32") and x.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    return x.data_ptr()


def sft_mlp_loss_grad(m: Mlp, pts, targets, grad_out, stream=None):
    """Mean squared error of the network on (pts [n,3], targets [n]) and its
    gradient, written into grad_out [nparam]; all contiguous float32 CUDA
    tensors. Returns the loss."""
    n = int(pts.shape[0])
    loss = ctypes.c_double()
    _check(lib().sft_mlp_loss_grad(m.h, n, _cuda_f32(pts, "pts"), _cuda_f32(targets, "targets"),
                                   _cuda_f32(grad_out, "grad_out"), ctypes.byref(loss), 1,
                                   stream if stream is not None else _current_stream()), "sft_mlp_loss_grad")
    return loss.value


def sft_mlp_train(m: Mlp, pts, targets, epochs=10, batch=16384, lr=2e-3, lr_final=1e-4, stream=None):
    """Adam training on (pts [n,3], targets [n]) contiguous float32 CUDA
    tensors; returns the per-epoch mean losses."""
    n = int(pts.shape[0])
    hist = np.zeros(int(epochs))
    _check(lib().sft_mlp_train(m.h, n, _cuda_f32(pts, "pts"), _cuda_f32(targets, "targets"), int(epochs),
                               int(batch), float(lr), float(lr_final), hist.ctypes.data, 1,
                               stream if stream is not None else _current_stream()), "sft_mlp_train")
    return hist


def sft_surrogate_dataset(src: Source, n: int, seed: int = 0, stream_id: int = 0, box_lo=(0.0, 0.0, 0.0),
                          box_hi=(1.0, 1.0, 1.0), field: int = 0, pts_out=None, f_out=None, stream=None):
    """Training set of the surrogate on the device: (pts [n,3], f [n] float32
    CUDA tensors, max |f|)."""
    import torch
    n = int(n)
    if pts_out is None:
        pts_out = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    if f_out is None:
        f_out = torch.empty(n, dtype=torch.float32, device="cuda")
    lo = (ctypes.c_float * 3)(*[float(x) for x in box_lo])
    hi = (ctypes.c_float * 3)(*[float(x) for x in box_hi])
    mx = ctypes.c_float()
    _check(lib().sft_surrogate_dataset(src.h, int(field), n, int(seed), int(stream_id), lo, hi,
                                       _cuda_f32(pts_out, "pts_out"), _cuda_f32(f_out, "f_out"), ctypes.byref(mx),
                                       stream if stream is not None else _current_stream()), "sft_surrogate_dataset")
    return pts_out, f_out, mx.value


def sft_transfer_surrogate(net, exact, tgt: Target, samples_per_elem: int, seed: int = 0, stream_id: int = 0,
                           alpha: float = 1.0, cg_tol: float = 1e-10, cg_max_iter: int = 1000, subsample: int = 4,
                           tau: float = 0.0, exact_field: int = 0, u_out=None, b_out=None, g_out=None,
                           fallback_out=None, sample_f_out=None, strict_inside: bool = False, stream=None,
                           allow_not_converged: bool = False, cg_mode: int = SFT_CG_MIXED,
                           sampling: int = SFT_SAMPLING_UNIFORM, cg_warm_start: bool = False,
                           exact_cost: int = 0):
    """Transfer with the surrogate network `net` (Mlp or None) backed by the
    exact source `exact` (Source or None). Outputs as sft_transfer (numpy for
    host, CUDA tensors for device). exact_cost: dependent FMAs added to every
    exact query (a stand-in for a costly black-box source). Returns (status,
    stats dict, u_out)."""
    if u_out is None:
        u_out = np.zeros(_nv(tgt), np.float64)
    up, udev, _ = _ptr(u_out)
    ptrs = [_ptr(x) for x in (b_out, g_out, fallback_out, sample_f_out)]
    for p, dv, _ in ptrs:
        if p is not None and dv != udev:
            raise ValueError("all outputs must be host arrays or all device tensors")
    o = _options(samples_per_elem, seed, stream_id, alpha, cg_tol, cg_max_iter, cg_mode=cg_mode, sampling=sampling,
                 cg_warm_start=cg_warm_start)
    o.strict_inside = int(bool(strict_inside))
    o.out_device = int(udev)
    o.cuda_stream = stream if stream is not None else _current_stream()
    so = sft_surrogate_opts()
    so.exact_field = int(exact_field)
    so.subsample = int(subsample)
    so.tau = float(tau)
    so.exact_cost = int(exact_cost)
    so.fallback_out = ptrs[2][0]
    so.sample_f_out = ptrs[3][0]
    st = sft_surrogate_stats()
    allow = (SFT_OK, SFT_ERR_NOT_CONVERGED) if allow_not_converged else (SFT_OK,)
    status = _check(lib().sft_transfer_surrogate(net.h if net is not None else None,
                                                 exact.h if exact is not None else None, tgt.h, ctypes.byref(o),
                                                 ctypes.byref(so), up, ptrs[0][0], ptrs[1][0], ctypes.byref(st)),
                    "sft_transfer_surrogate", allow)
    return status, st.as_dict(), u_out


def sft_source_grid(src: Source, precision: int):
    """(n[3], cell start [ncells+1] int64, cell items [nitems] int32)."""
    n = (ctypes.c_int32 * 3)()
    nc, ni = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().sft_source_grid(src.h, int(precision), n, ctypes.byref(nc), ctypes.byref(ni), None, None),
           "sft_source_grid")
    start = np.zeros(nc.value + 1, np.int64)
    items = np.zeros(max(ni.value, 1), np.int32)
    _check(lib().sft_source_grid(src.h, int(precision), None, None, None, start.ctypes.data, items.ctypes.data),
           "sft_source_grid")
    return np.array(list(n)), start, items[:ni.value]


def sft_batch_groups(plan) -> list:
    """Per non-empty request group: dict(requests, dim, max_fields, tile, lanes_per_element)."""
    out = np.zeros((6, 5), np.int32)
    _check(lib().sft_batch_groups(plan.h, out.ctypes.data), "sft_batch_groups")
    keys = ("requests", "dim", "max_fields", "tile", "lanes_per_element")
    return [dict(zip(keys, (int(v) for v in row))) for row in out if row[0] > 0]


def sft_trim_memory() -> None:
    """Return the unused blocks of the library's device memory pools to the driver."""
    _check(lib().sft_trim_memory(), "sft_trim_memory")


def sft_target_set_wait_limit(tgt: Target, seconds: float) -> None:
    """Limit of the device waits of the solves on this target (default 2 s)."""
    _check(lib().sft_target_set_wait_limit(tgt.h, float(seconds)), "sft_target_set_wait_limit")


def sft_source_cell_first(src: Source, precision: int) -> np.ndarray:
    """[ncells] int32 start element of the location walk per grid cell (-1: empty)."""
    n, _, _ = sft_source_grid(src, precision)
    out = np.zeros(int(np.prod(n)), np.int32)
    _check(lib().sft_source_cell_first(src.h, int(precision), out.ctypes.data), "sft_source_cell_first")
    return out


def sft_source_adjacency(src: Source, precision: int) -> np.ndarray:
    """[nelems][dim+1] int32 face neighbours of the source mesh (-1 on the boundary)."""
    conn = src._keep[1]
    out = np.zeros((int(conn.shape[0]), int(conn.shape[1])), np.int32)
    _check(lib().sft_source_adjacency(src.h, int(precision), out.ctypes.data), "sft_source_adjacency")
    return out


def sft_target_mass(tgt: Target):
    """(row_ptr int64, col int32, val float64, lumped float64) of the mass matrix."""
    nnz = ctypes.c_int64()
    _check(lib().sft_target_mass(tgt.h, ctypes.byref(nnz), None, None, None, None), "sft_target_mass")
    nv = _nv(tgt)
    rp = np.zeros(nv + 1, np.int64)
    col = np.zeros(nnz.value, np.int32)
    val = np.zeros(nnz.value, np.float64)
    lump = np.zeros(nv, np.float64)
    _check(lib().sft_target_mass(tgt.h, None, rp.ctypes.data, col.ctypes.data, val.ctypes.data,
                                 lump.ctypes.data), "sft_target_mass")
    return rp, col, val, lump


def sft_kernel_launches() -> int:
    """Kernels launched by libsft in this process so far."""
    return int(lib().sft_kernel_launches())


def _nf(src: Source) -> int:
    return int(src._keep[2].shape[0])


def _nv(tgt: Target) -> int:
    return int(tgt._keep[0].shape[0])


def mesh_source(mesh, grid_scale_L=1.0, device=None):
    """Convenience: a ``workloads.Mesh``-like object (coords, conn, values)."""
    c, k, v = mesh.coords, mesh.conn, mesh.values
    if device is not None:
        import torch
        c, k, v = (torch.as_tensor(np.ascontiguousarray(a)).to(device) for a in (c, k, v))
    return sft_source_create(c, k, v, grid_scale_L)


def mesh_target(mesh, device=None):
    c, k = mesh.coords, mesh.conn
    if device is not None:
        import torch
        c, k = (torch.as_tensor(np.ascontiguousarray(a)).to(device) for a in (c, k))
    return sft_target_create(c, k)
