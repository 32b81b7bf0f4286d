"""Parity of the CUDA library (through the C ABI) with the FP64 oracle.

Bar: integer results (grid cells, located elements, per-sample source
elements, CSR pattern) bit-exact; FP64 paths within rounding; FP32 paths:
b within 1e-5 relative, the rest within the bounds derived in the design
notes (FP32 evaluation error ~1e-7 relative, amplified at most by the mass
matrix condition number). Floating-point vectors are held to each bound both
as a 2-norm ratio and entry by entry (max_i |a_i - b_i| against max_i |b_i|),
so a few wrong entries cannot hide under the norm of a long vector."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_00538_gb300 as sft  # noqa: E402

DEV = torch.device("cuda:0")
FP64, FP32 = sft.SFT_PREC_FP64, sft.SFT_PREC_FP32


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _rel_max(a, b):
    """largest entry-wise difference relative to the largest entry of b"""
    a, b = np.asarray(a), np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def _close(a, b, lim):
    return _rel(a, b) < lim and _rel_max(a, b) < lim


def _run(src, tgt, prec, N, seed=0, alpha=1.0, tol=1e-13, device=True, stream_id=0, L=1.0, maxit=2000):
    s = sft.mesh_source(src, grid_scale_L=L, device=DEV if device else None)
    t = sft.mesh_target(tgt, device=DEV if device else None)
    nf = src.nfields
    if device:
        u = torch.zeros((nf, tgt.nnodes), dtype=torch.float64, device=DEV)
        b, g = torch.zeros_like(u), torch.zeros_like(u)
        se = torch.zeros((tgt.nelems, N), dtype=torch.int32, device=DEV)
    else:
        u = np.zeros((nf, tgt.nnodes))
        b, g = np.zeros_like(u), np.zeros_like(u)
        se = np.zeros((tgt.nelems, N), np.int32)
    _, stats, _ = sft.sft_transfer(s, t, N, prec, seed=seed, stream_id=stream_id, alpha=alpha, cg_tol=tol,
                                   cg_max_iter=maxit, u_out=u, b_out=b, g_out=g, sample_elem_out=se)
    cv = lambda x: x.cpu().numpy() if device else x  # noqa: E731
    return dict(u=cv(u), b=cv(b), g=cv(g), sample_elem=cv(se), stats=stats, s=s, t=t)


# --------------------------------------------------------------------------
# location and grid
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim,prec", [(2, FP64), (2, FP32), (3, FP64), (3, FP32)])
def test_grid_bit_exact(orc, dim, prec):
    m = W.jittered_tri_mesh(23, 5) if dim == 2 else W.jittered_kuhn_mesh(7, 5)
    m = W.with_values(m, [W.paper_f2], np.float32 if prec == FP32 else np.float64)
    if prec == FP32:
        m = W.as_precision(m, np.float32)
    s = sft.mesh_source(m, device=DEV)
    n, start, items = sft.sft_source_grid(s, prec)
    g = orc.Grid(1 if prec == FP32 else 0, m.coords, m.conn)
    n_o, nc_o, _ = g.shape()
    start_o, items_o = g.csr()
    assert list(n) == list(n_o)
    assert np.array_equal(start, start_o)
    # the same elements in every cell (a cell's order is not part of the
    # structure), and the same start element of the walk: the oracle lists a
    # cell deepest-first, so its first item is the deepest at the centre
    cell = np.repeat(np.arange(len(start) - 1), np.diff(start))
    assert np.array_equal(items[np.lexsort((items, cell))], items_o[np.lexsort((items_o, cell))])
    first = sft.sft_source_cell_first(s, prec)
    nonempty = np.diff(start_o) > 0
    assert np.array_equal(first[nonempty], items_o[start_o[:-1][nonempty]])
    assert np.all(first[~nonempty] == -1)


@pytest.mark.parametrize("dim,prec", [(2, FP64), (2, FP32), (3, FP64), (3, FP32)])
def test_locate_bit_exact(orc, dim, prec):
    m = W.jittered_tri_mesh(31, 6) if dim == 2 else W.jittered_kuhn_mesh(9, 6)
    dt = np.float32 if prec == FP32 else np.float64
    m = W.as_precision(W.with_values(m, [W.paper_f1, W.paper_f3], np.float64), dt)
    rng = np.random.default_rng(3)
    pts = np.concatenate([rng.random((20000, dim)), m.coords.astype(np.float64),
                          m.coords[m.conn[:, :2]].astype(np.float64).mean(1),
                          rng.random((500, dim)) * 1.2 - 0.1])  # some points outside the box
    s = sft.mesh_source(m, device=DEV)
    e_gpu, v_gpu = sft.sft_locate(s, pts, prec)
    p_o = 1 if prec == FP32 else 0
    e_o, st_o = orc.Grid(p_o, m.coords, m.conn).locate(pts)
    assert np.array_equal(e_gpu, e_o)
    # values: FP64 path to rounding; FP32 path to single-precision evaluation error
    x = pts.astype(np.float32).astype(np.float64) if prec == FP32 else pts
    ref = np.stack([orc.eval_p1(m.coords, m.conn, m.values, e, xi) for e, xi in zip(e_o[:3000], x[:3000])], 1)
    tol = 2e-6 if prec == FP32 else 1e-13
    assert np.max(np.abs(v_gpu[:, :3000] - ref)) <= tol * np.max(np.abs(ref))


@pytest.mark.parametrize("dim,prec", [(2, FP64), (2, FP32), (3, FP64), (3, FP32)])
def test_adjacency_bit_exact(orc, dim, prec):
    """Face neighbours of the location walk, built on the GPU through the
    grid, equal the oracle's (built from their definition) entry for entry,
    on a jittered mesh and on a Delaunay / graded one."""
    meshes = ([W.jittered_tri_mesh(29, 5), W.delaunay_tri_mesh(700, 9, 5)] if dim == 2 else
              [W.jittered_kuhn_mesh(7, 5), W.morton_reorder(W.jittered_kuhn_mesh(5, 6))])
    for m in meshes:
        if dim == 3 and m is meshes[1]:
            m = W.Mesh(m.coords ** 2, m.conn, None)    # graded towards the origin
        m = W.with_values(m, [W.paper_f2] if dim == 2 else [lambda x: x[:, 0]])
        if prec == FP32:
            m = W.as_precision(m, np.float32)
        s = sft.mesh_source(m, device=DEV)
        adj = sft.sft_source_adjacency(s, prec)
        ref = orc.Grid(1 if prec == FP32 else 0, m.coords, m.conn).adjacency()
        assert np.array_equal(adj, ref)


def test_locate_host_pointers_match_device(orc):
    m = W.with_values(W.jittered_tri_mesh(12, 1), [W.paper_f3])
    pts = np.random.default_rng(0).random((777, 2))
    s_h = sft.mesh_source(m)                 # host inputs
    s_d = sft.mesh_source(m, device=DEV)     # device inputs
    e1, v1 = sft.sft_locate(s_h, pts, FP64)
    e2, v2 = sft.sft_locate(s_d, pts, FP64)
    assert np.array_equal(e1, e2) and np.array_equal(v1, v2)


# --------------------------------------------------------------------------
# mass matrix and solve
# --------------------------------------------------------------------------
@pytest.mark.parametrize("dim", [2, 3])
def test_mass_matrix_parity(orc, dim):
    m = W.delaunay_tri_mesh(900, 12, 8) if dim == 2 else W.morton_reorder(W.jittered_kuhn_mesh(6, 8))
    t = sft.mesh_target(m, device=DEV)
    rp, col, val, lump = sft.sft_target_mass(t)
    rp_o, col_o, val_o = orc.mass_csr(m.coords, m.conn)
    assert np.array_equal(rp, rp_o) and np.array_equal(col, col_o)
    assert np.max(np.abs(val - val_o)) <= 1e-15 * np.max(np.abs(val_o))
    assert np.max(np.abs(lump - orc.lumped_mass(m.coords, m.conn))) <= 1e-15


def _fan_2d(k=24):
    ang = 2 * np.pi * np.arange(k) / k
    coords = np.vstack([[0.0, 0.0], np.stack([np.cos(ang), np.sin(ang)], 1)])
    conn = np.array([[0, 1 + i, 1 + (i + 1) % k] for i in range(k)], np.int32)
    return W.Mesh(coords, conn, None)


def _star_3d():
    """Tetrahedra joining the centre to the faces of a once-subdivided
    icosahedron (80 faces, 42 surface nodes): the centre's row has 43 entries."""
    t = (1 + 5 ** 0.5) / 2
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
         (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    v = [np.array(p, float) / np.linalg.norm(p) for p in v]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6),
         (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10),
         (8, 6, 7), (9, 8, 1)]
    mid = {}

    def m(a, b):
        key = (min(a, b), max(a, b))
        if key not in mid:
            p = v[a] + v[b]
            v.append(p / np.linalg.norm(p))
            mid[key] = len(v) - 1
        return mid[key]
    faces = []
    for a, b, c in f:
        ab, bc, ca = m(a, b), m(b, c), m(c, a)
        faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
    coords = np.vstack([[0.0, 0.0, 0.0], np.array(v)])
    conn = np.array([[0, 1 + a, 1 + b, 1 + c] for a, b, c in faces], np.int32)
    mesh = W.Mesh(coords, conn, None)
    W._fix_orientation(mesh)
    return mesh


@pytest.mark.parametrize("dim", [2, 3])
def test_mass_matrix_high_valence(orc, dim):
    """Rows longer than the small per-thread buffers of the first counting
    pass (16 entries in 2D, 32 in 3D) are built again with the full ones."""
    m = _fan_2d() if dim == 2 else _star_3d()
    rp_o, col_o, val_o = orc.mass_csr(m.coords, m.conn)
    assert np.diff(rp_o).max() > (16 if dim == 2 else 32)
    t = sft.mesh_target(m, device=DEV)
    rp, col, val, lump = sft.sft_target_mass(t)
    assert np.array_equal(rp, rp_o) and np.array_equal(col, col_o)
    assert np.max(np.abs(val - val_o)) <= 1e-15 * np.max(np.abs(val_o))
    assert np.max(np.abs(lump - orc.lumped_mass(m.coords, m.conn))) <= 1e-15


@pytest.mark.parametrize("dim,nrhs", [(2, 1), (2, 3), (3, 2)])
def test_mass_solve_parity(orc, dim, nrhs):
    """Given the same b, the FP64 CG solutions agree to 1e-10 (tol 1e-13)."""
    m = W.delaunay_tri_mesh(3000, 20, 9) if dim == 2 else W.morton_reorder(W.jittered_kuhn_mesh(8, 9))
    t = sft.mesh_target(m, device=DEV)
    b = np.random.default_rng(4).standard_normal((nrhs, m.nnodes))
    u, it, rr = sft.sft_mass_solve(t, b, tol=1e-13, max_iter=2000)
    assert rr <= 1e-13
    rp, col, val = orc.mass_csr(m.coords, m.conn)
    for f in range(nrhs):
        uo, _, _ = orc.pcg(rp, col, val, b[f], tol=1e-13, max_iter=2000)
        assert _rel(u[f], uo) < 1e-10


def test_mass_solve_not_converged_is_reported():
    m = W.delaunay_tri_mesh(400, 8, 2)
    t = sft.mesh_target(m, device=DEV)
    b = np.random.default_rng(1).standard_normal((1, m.nnodes))
    with pytest.raises(sft.SftError) as ei:
        sft.sft_mass_solve(t, b, tol=1e-15, max_iter=2)
    assert ei.value.status == 5


# --------------------------------------------------------------------------
# the transfer
# --------------------------------------------------------------------------
CASES = [
    # name, scale, precision, N
    ("tri2k", 1.0, FP64, 16),
    ("tri2k", 1.0, FP32, 16),
    ("tri4m", 3e-3, FP32, 64),
    ("tri4m", 3e-3, FP64, 64),
    ("tet5m", 2e-3, FP32, 32),
    ("tet5m", 2e-3, FP64, 32),
]


@pytest.mark.parametrize("name,scale,prec,N", CASES)
def test_transfer_parity(orc, name, scale, prec, N):
    src, tgt, _ = W.config_meshes(name, scale)
    r = _run(src, tgt, prec, N)
    o = orc.transfer(src, tgt, 1 if prec == FP32 else 0, N, cg_tol=1e-13, cg_max_iter=2000,
                     want_sample_elem=True)
    assert np.array_equal(r["sample_elem"], o["sample_elem"])
    assert r["stats"]["fallback_queries"] == o["fallback_queries"]
    assert r["stats"]["empty_queries"] == o["empty_queries"] == 0
    lim = dict(g=1e-13, b=1e-13, u=1e-10) if prec == FP64 else dict(g=2e-6, b=1e-5, u=1e-4)
    for f in range(src.nfields):
        for k in ("g", "b", "u"):
            assert _close(r[k][f], o[k][f], lim[k]), (k, f, _rel(r[k][f], o[k][f]), _rel_max(r[k][f], o[k][f]))


@pytest.mark.parametrize("dim,N,nf,alpha", [
    (2, 1, 1, 1.0), (2, 7, 1, 1.0), (2, 20, 1, 0.5), (2, 33, 1, 1.0), (2, 128, 2, 1.0),
    (3, 1, 1, 1.0), (3, 5, 3, 0.0), (3, 40, 1, 1.0), (2, 16, 8, 1.0), (3, 8, 5, 0.7),
])
def test_transfer_edge_shapes(orc, dim, N, nf, alpha):
    """Ragged unit counts, packed and long warp modes, odd N in 2D, several
    fields (masked template widths), alpha = 0."""
    fields = [W.paper_f1, W.paper_f2, W.paper_f3, W.field_sincos, W.linear_field([1, 2, 3, 4])][:nf]
    fields = (fields * 2)[:nf]
    if dim == 2:
        src = W.with_values(W.jittered_tri_mesh(9, 11), fields)
        tgt = W.delaunay_tri_mesh(53, 5, 12)
    else:
        src = W.with_values(W.jittered_kuhn_mesh(4, 11), [lambda x, f=f: f(x[:, :2]) + x[:, 2] for f in fields])
        tgt = W.morton_reorder(W.jittered_kuhn_mesh(3, 12))
    for prec in (FP64, FP32):
        r = _run(src, tgt, prec, N, seed=5, alpha=alpha, stream_id=3)
        o = orc.transfer(src, tgt, 1 if prec == FP32 else 0, N, seed=5, stream=3, alpha=alpha,
                         cg_tol=1e-13, cg_max_iter=2000, want_sample_elem=True)
        assert np.array_equal(r["sample_elem"], o["sample_elem"])
        lim_b = 1e-13 if prec == FP64 else 1e-5
        for f in range(nf):
            assert _close(r["b"][f], o["b"][f], lim_b), (prec, f, _rel_max(r["b"][f], o["b"][f]))
            assert _close(r["u"][f], o["u"][f], 1e-10 if prec == FP64 else 1e-4), (prec, f)


@pytest.mark.parametrize("dim", [2, 3])
def test_transfer_field_subset(orc, dim):
    """The first k fields of a 5-field source (the per-element value copies
    hold all five per element; k = 1 runs a multi-field kernel width)."""
    fields = [W.paper_f1, W.paper_f2, W.paper_f3, W.field_sincos, W.linear_field([1, 2, 3, 4])]
    if dim == 2:
        src = W.with_values(W.jittered_tri_mesh(9, 11), fields)
        tgt = W.delaunay_tri_mesh(53, 5, 12)
    else:
        src = W.with_values(W.jittered_kuhn_mesh(4, 11), [lambda x, f=f: f(x[:, :2]) + x[:, 2] for f in fields])
        tgt = W.morton_reorder(W.jittered_kuhn_mesh(3, 12))
    N = 12
    for prec in (FP64, FP32):
        o = orc.transfer(src, tgt, 1 if prec == FP32 else 0, N, seed=4, cg_tol=1e-13, cg_max_iter=2000,
                         want_sample_elem=True)
        s = sft.mesh_source(src, device=DEV)
        t = sft.mesh_target(tgt, device=DEV)
        for k in (1, 2, 3, 5):
            u = torch.zeros((k, tgt.nnodes), dtype=torch.float64, device=DEV)
            b = torch.zeros_like(u)
            se = torch.zeros((tgt.nelems, N), dtype=torch.int32, device=DEV)
            sft.sft_transfer(s, t, N, prec, seed=4, cg_tol=1e-13, cg_max_iter=2000, field_count=k,
                             u_out=u, b_out=b, sample_elem_out=se)
            assert np.array_equal(se.cpu().numpy(), o["sample_elem"])
            bb, uu = b.cpu().numpy(), u.cpu().numpy()
            for f in range(k):
                assert _close(bb[f], o["b"][f], 1e-13 if prec == FP64 else 1e-5), (prec, k, f)
                assert _close(uu[f], o["u"][f], 1e-10 if prec == FP64 else 1e-4), (prec, k, f)


def test_host_buffers_equal_device_buffers():
    src, tgt, _ = W.config_meshes("tri2k")
    a = _run(src, tgt, FP64, 16, device=True)
    b = _run(src, tgt, FP64, 16, device=False)
    assert np.array_equal(a["sample_elem"], b["sample_elem"])
    assert _rel(a["u"], b["u"]) < 1e-13


def test_seeds_and_streams_change_samples():
    src, tgt, _ = W.config_meshes("tri2k")
    a = _run(src, tgt, FP64, 16, seed=1)
    b = _run(src, tgt, FP64, 16, seed=2)
    c = _run(src, tgt, FP64, 16, seed=1, stream_id=9)
    assert not np.array_equal(a["sample_elem"], b["sample_elem"])
    assert not np.array_equal(a["sample_elem"], c["sample_elem"])


def test_conservation_api(orc):
    src, tgt, _ = W.config_meshes("tri2k")
    r = _run(src, tgt, FP64, 16)
    e, i_s, i_t = sft.sft_conservation_error(r["s"], r["t"], r["u"][0])
    assert i_s == pytest.approx(orc.integral_p1(src.coords, src.conn, src.values[0]), rel=1e-13)
    assert i_t == pytest.approx(orc.lumped_mass(tgt.coords, tgt.conn) @ r["u"][0], rel=1e-13)
    assert i_t == pytest.approx(r["b"][0].sum(), rel=1e-11)
    assert e == pytest.approx(abs(i_s - i_t) / abs(i_s), rel=1e-9)


def test_empty_cells_and_strict_mode():
    """An L-shaped source leaves grid cells empty; queries there return -1
    and value 0, and strict mode reports SFT_ERR_OUTSIDE."""
    m = W.jittered_tri_mesh(8, 0)
    cen = m.coords[m.conn].mean(1)
    keep = ~((cen[:, 0] > 0.5) & (cen[:, 1] > 0.5))
    used = np.unique(m.conn[keep])
    remap = -np.ones(m.nnodes, np.int64)
    remap[used] = np.arange(used.size)
    src = W.with_values(W.Mesh(m.coords[used], remap[m.conn[keep]].astype(np.int32)), [W.paper_f2])
    s = sft.mesh_source(src, device=DEV)
    e, v = sft.sft_locate(s, np.array([[0.9, 0.9], [0.1, 0.1]]), FP64)
    assert e[0] == -1 and v[0, 0] == 0.0 and e[1] >= 0
    tgt = W.delaunay_tri_mesh(50, 4, 3)
    t = sft.mesh_target(tgt, device=DEV)
    with pytest.raises(sft.SftError) as ei:
        sft.sft_transfer(s, t, 8, FP64, strict_inside=True)
    assert ei.value.status == 6


def test_memory_pool_reuse_and_trim():
    """Meshes created and destroyed in a loop reuse the library pool's blocks
    (the device's free memory does not move on the second round), and
    sft_trim_memory returns them to the driver."""
    src, tgt, _ = W.config_meshes("tri4m", 0.05)
    free = lambda: (torch.cuda.synchronize(), torch.cuda.mem_get_info(DEV)[0])[1]  # noqa: E731
    sft.sft_trim_memory()
    f0 = free()
    after = []
    for _ in range(2):
        s = sft.mesh_source(src)           # host inputs: only the library allocates
        t = sft.mesh_target(tgt)
        sft.sft_transfer(s, t, 8, FP32, cg_tol=1e-10)
        s.close()
        t.close()
        after.append(free())
    assert after[0] < f0                   # the pool kept the freed blocks
    assert after[1] == after[0]            # and the second round reused them
    sft.sft_trim_memory()
    assert free() > after[1]


def test_invalid_meshes_rejected():
    m = W.with_values(W.jittered_tri_mesh(4, 0), [W.paper_f1])
    bad = m.conn.copy()
    bad[3, 1] = m.nnodes + 5
    with pytest.raises(sft.SftError) as ei:
        sft.sft_source_create(m.coords, bad, m.values)
    assert ei.value.status == 2
    flip = m.conn.copy()
    flip[0, [1, 2]] = flip[0, [2, 1]]
    with pytest.raises(sft.SftError) as ei:
        sft.sft_target_create(m.coords, flip)
    assert ei.value.status == 2
    nanc = m.coords.copy()
    nanc[2, 0] = np.nan
    with pytest.raises(sft.SftError) as ei:
        sft.sft_source_create(nanc, m.conn, m.values)
    assert ei.value.status == 2
    assert "non-finite" in str(ei.value)
    # non-finite coordinates are found on the device: device inputs too, and
    # in a node no element uses
    for bad_val in (np.inf, -np.inf, np.nan):
        c2 = np.concatenate([m.coords, [[bad_val, 0.5]]])
        for dev in (False, True):
            cc = torch.as_tensor(c2).to(DEV) if dev else c2
            kk = torch.as_tensor(m.conn).to(DEV) if dev else m.conn
            with pytest.raises(sft.SftError) as ei:
                sft.sft_target_create(cc, kk)
            assert ei.value.status == 2 and "non-finite" in str(ei.value)
            vv = np.concatenate([m.values, np.zeros((m.values.shape[0], 1))], axis=1)
            vv = torch.as_tensor(vv).to(DEV) if dev else vv
            with pytest.raises(sft.SftError) as ei:
                sft.sft_source_create(cc, kk, vv)
            assert ei.value.status == 2 and "non-finite" in str(ei.value)
    # the library stays usable after the rejections
    s = sft.sft_source_create(m.coords, m.conn, m.values)
    t = sft.sft_target_create(m.coords, m.conn)
    s.close()
    t.close()
    # a target index out of range: the setup skips the element in every pass
    # and reports the error once the row counts are read back
    for v in (m.nnodes, m.nnodes + 1000, -1):
        badt = m.conn.copy()
        badt[5, 2] = v
        with pytest.raises(sft.SftError) as ei:
            sft.sft_target_create(m.coords, badt)
        assert ei.value.status == 2
    # a valid target afterwards on the same stream
    t = sft.sft_target_create(m.coords, m.conn)
    t.close()


# --------------------------------------------------------------------------
# full size, in the benchmark's launch configuration: every output
# --------------------------------------------------------------------------
@pytest.mark.parametrize("name", ["tri4m", "tet5m"])
def test_full_size_elementwise(orc, name):
    """The benchmark's workloads at full size (4.0 M -> 2.0 M triangles x 64
    samples; 5.0 M -> 3.0 M tetrahedra x 32 samples), FP32 path, against the
    oracle run on the whole workload: the source element of every one of the
    128 M / 95 M samples bit for bit, g, b and u entry by entry within the
    FP32 bounds, plus properties that hold at any size."""
    src, tgt, p = W.config_meshes(name)
    N = p["samples_per_elem"]
    r = _run(src, tgt, FP32, N, tol=p["cg_tol"])
    # every sample lands in an element (the meshes cover the same domain)
    assert r["stats"]["empty_queries"] == 0
    assert (r["sample_elem"] >= 0).all()
    # properties: partition of unity of the control term and convergence of M u = b
    e_mass, i_s, i_t = sft.sft_conservation_error(r["s"], r["t"], r["u"][0])
    assert i_t == pytest.approx(r["b"][0].sum(), rel=1e-8)
    assert r["stats"]["cg_rel_resid"] <= p["cg_tol"]
    assert e_mass < 1e-3
    gpu_se = r.pop("sample_elem")
    r["s"].close()
    r["t"].close()
    o = orc.transfer(src, tgt, 1, N, cg_tol=p["cg_tol"], want_sample_elem=True)
    assert o["empty_queries"] == 0 and o["cg_rel_resid"] <= p["cg_tol"]
    assert r["stats"]["fallback_queries"] == o["fallback_queries"]
    bad = np.count_nonzero(gpu_se != o["sample_elem"])
    assert bad == 0, f"{bad} of {gpu_se.size} samples located in another element"
    del gpu_se, o["sample_elem"]
    lim = dict(g=2e-6, b=1e-5, u=1e-4)
    for k in ("g", "b", "u"):
        assert _close(r[k][0], o[k][0], lim[k]), (k, _rel(r[k][0], o[k][0]), _rel_max(r[k][0], o[k][0]))


def test_set_values_equals_recreate(orc):
    """Updating a source's values in place gives the transfer of a source
    created with those values (same mesh, same grid)."""
    src, tgt, _ = W.config_meshes("tri4m", 2e-3)
    s = sft.mesh_source(src, device=DEV)
    t = sft.mesh_target(tgt, device=DEV)
    new = W.as_precision(W.with_values(src, [W.paper_f3], np.float64), np.float32)
    # the source integral of the old values is computed (and cached) first
    _, i_old, _ = sft.sft_conservation_error(s, t, np.ones(tgt.nnodes))
    assert i_old == pytest.approx(orc.integral_p1(src.coords, src.conn, src.values[0]), rel=1e-6)
    sft.sft_source_set_values(s, torch.as_tensor(new.values).to(DEV))
    _, _, u1 = sft.sft_transfer(s, t, 16, FP32, cg_tol=1e-12)
    s2 = sft.mesh_source(new, device=DEV)
    _, _, u2 = sft.sft_transfer(s2, t, 16, FP32, cg_tol=1e-12)
    # same samples, locations and values: the load vectors differ only by the
    # order of the FP64 atomic sums
    assert _rel(u1, u2) < 1e-12
    e1 = sft.sft_conservation_error(s, t, u1[0])
    e2 = sft.sft_conservation_error(s2, t, u2[0])
    assert e1[1] == e2[1]                      # the same source integral
    assert e1[2] == pytest.approx(e2[2], rel=1e-12)
    assert e1[1] == pytest.approx(orc.integral_p1(new.coords, new.conn, new.values[0]), rel=1e-6)
