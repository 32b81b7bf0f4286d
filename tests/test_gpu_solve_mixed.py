"""The step-7 solve in both CG modes against the oracle's FP64 Jacobi-PCG.

MIXED mode (FP64 refinement around FP32 CG on the Jacobi-scaled matrix)
stops on the true FP64 residual, so the residual it reports is checked
against ||b - M u|| recomputed on the host from the oracle's CSR matrix.
Both modes must give the oracle's solution to the accuracy the tolerance
fixes: two solutions whose residuals are below tol ||b|| differ by at most
2 cond(M) tol relative, and cond(M) <= 5 max diag / min diag (the scaled
matrix diag(M)^-1/2 M diag(M)^-1/2 has cond <= 5), which for the
quasi-uniform and tiny meshes is below 100: 1e-10 at tol = 1e-13.
Meshes cover quasi-uniform, strongly graded (diag(M) spanning 3.3 (3D) to
6.5 (2D) orders of magnitude) and tiny-scale ones (mass entries below the FP32 range)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_00538_gb300 as sft  # noqa: E402

DEV = torch.device("cuda:0")
MODES = [sft.SFT_CG_MIXED, sft.SFT_CG_FP64]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _spmv(rp, col, val, x):
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return np.bincount(rows, weights=val * x[col], minlength=len(rp) - 1)


def _graded(dim):
    m = W.delaunay_tri_mesh(2500, 18, 3) if dim == 2 else W.morton_reorder(W.jittered_kuhn_mesh(7, 3))
    c = m.coords.copy()
    c[:, 0] = c[:, 0] ** 3          # element sizes shrink ~ x^2 towards x = 0
    g = W.Mesh(c, m.conn.copy(), None)
    W._fix_orientation(g)           # the nonlinear map can flip a sliver
    return g


def _mesh(kind, dim):
    if kind == "uniform":
        return W.delaunay_tri_mesh(3000, 20, 9) if dim == 2 else W.morton_reorder(W.jittered_kuhn_mesh(8, 9))
    if kind == "graded":
        return _graded(dim)
    m = W.delaunay_tri_mesh(800, 12, 5) if dim == 2 else W.jittered_kuhn_mesh(5, 5)
    return W.Mesh(m.coords * 1e-15, m.conn, None)   # |T| ~ 1e-33 (2D) / 1e-48 (3D)


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("kind,dim,nrhs", [("uniform", 2, 1), ("uniform", 3, 2), ("graded", 2, 1),
                                           ("graded", 3, 3), ("tiny", 2, 1), ("tiny", 3, 5)])
def test_solve_modes_match_oracle(orc, mode, kind, dim, nrhs):
    m = _mesh(kind, dim)
    t = sft.mesh_target(m, device=DEV)
    rp, col, val = orc.mass_csr(m.coords, m.conn)
    rng = np.random.default_rng(11)
    # right-hand sides of load-vector size: b = M f for random nodal f
    b = np.stack([_spmv(rp, col, val, rng.standard_normal(m.nnodes)) for _ in range(nrhs)])
    tol = 1e-13
    u, it, rr = sft.sft_mass_solve(t, b, tol=tol, max_iter=2000, cg_mode=mode)
    assert rr <= tol and it > 0
    diag = val[col == np.repeat(np.arange(m.nnodes), np.diff(rp))]
    bound = 1e-10 if kind != "graded" else 2 * 5 * diag.max() / diag.min() * tol
    for f in range(nrhs):
        uo, _, _ = orc.pcg(rp, col, val, b[f], tol=tol, max_iter=2000)
        assert _rel(u[f], uo) < bound, (f, _rel(u[f], uo))
        true_rel = np.linalg.norm(b[f] - _spmv(rp, col, val, u[f])) / np.linalg.norm(b[f])
        if mode == sft.SFT_CG_MIXED:
            # the reported residual is the true one (same quantity, FP64 rounding apart)
            assert true_rel <= 2 * tol
        else:
            assert true_rel <= 1e-11


def test_mixed_zero_rhs_and_iteration_budget(orc):
    m = W.delaunay_tri_mesh(3000, 20, 9)
    t = sft.mesh_target(m, device=DEV)
    rp, col, val = orc.mass_csr(m.coords, m.conn)
    rng = np.random.default_rng(2)
    b = np.stack([_spmv(rp, col, val, rng.standard_normal(m.nnodes)), np.zeros(m.nnodes),
                  _spmv(rp, col, val, rng.standard_normal(m.nnodes))])
    u, it, rr = sft.sft_mass_solve(t, b, tol=1e-12, max_iter=2000)
    assert rr <= 1e-12
    assert np.all(u[1] == 0.0)
    # the budget counts inner iterations: a tolerance the FP32 inner solves
    # reach in a few cycles uses about as many iterations as the FP64 CG
    _, it64, _ = sft.sft_mass_solve(t, b, tol=1e-12, max_iter=2000, cg_mode=sft.SFT_CG_FP64)
    assert it <= 2 * it64 + 4
    with pytest.raises(sft.SftError) as e:
        sft.sft_mass_solve(t, b, tol=1e-12, max_iter=3)
    assert e.value.status == sft.SFT_ERR_NOT_CONVERGED
    with pytest.raises(sft.SftError) as e:
        sft.sft_mass_solve(t, b, tol=1e-12, max_iter=100, cg_mode=7)
    assert e.value.status == sft.SFT_ERR_ARG


def test_transfer_modes_agree(orc):
    """The transfer's u in either mode is the oracle's to the solve tolerance."""
    src, tgt, _ = W.config_meshes("tri2k", 1.0)
    s, t = sft.mesh_source(src), sft.mesh_target(tgt)
    o = orc.transfer(src, tgt, 0, 16, seed=4, cg_tol=1e-13, cg_max_iter=2000)
    for mode in MODES:
        _, st, u = sft.sft_transfer(s, t, 16, sft.SFT_PREC_FP64, seed=4, cg_tol=1e-13, cg_max_iter=2000,
                                    cg_mode=mode)
        assert st["cg_rel_resid"] <= 1e-13
        for f in range(u.shape[0]):
            assert _rel(u[f], o["u"][f]) < 1e-10


def test_warm_start(orc):
    """cg_warm_start: the solve starts from the values in u_out. From the
    converged solution it stops after the first residual check (0 inner
    iterations, u unchanged to the tolerance); from a poor start it reaches
    the cold-start solution within the solve tolerance; FP64 mode and batched
    plans reject it."""
    src, tgt, _ = W.config_meshes("tri2k", 1.0)
    s, t = sft.mesh_source(src, device=DEV), sft.mesh_target(tgt, device=DEV)
    u = torch.zeros((1, tgt.nnodes), dtype=torch.float64, device=DEV)
    _, st0, _ = sft.sft_transfer(s, t, 16, sft.SFT_PREC_FP64, seed=2, cg_tol=1e-12, u_out=u)
    u0 = u.cpu().numpy().copy()
    _, st1, _ = sft.sft_transfer(s, t, 16, sft.SFT_PREC_FP64, seed=2, cg_tol=1e-12, u_out=u, cg_warm_start=True)
    assert st1["cg_iters"] == 0 and st1["cg_rel_resid"] <= 1e-12
    assert _rel(u.cpu().numpy(), u0) < 1e-12
    # poor start (host buffers: the start is copied in)
    rng = np.random.default_rng(3)
    uh = rng.standard_normal((1, tgt.nnodes))
    _, st2, _ = sft.sft_transfer(s, t, 16, sft.SFT_PREC_FP64, seed=2, cg_tol=1e-12, u_out=uh, cg_warm_start=True)
    assert st2["cg_rel_resid"] <= 1e-12 and st2["cg_iters"] > 0
    assert _rel(uh, u0) < 1e-10
    # a second transfer with other samples starts close: fewer iterations than cold
    u2 = u.clone()
    _, st3, _ = sft.sft_transfer(s, t, 16, sft.SFT_PREC_FP64, seed=9, cg_tol=1e-12, u_out=u2, cg_warm_start=True)
    u3 = torch.zeros_like(u)
    _, st4, _ = sft.sft_transfer(s, t, 16, sft.SFT_PREC_FP64, seed=9, cg_tol=1e-12, u_out=u3)
    assert st3["cg_iters"] <= st4["cg_iters"]
    assert _rel(u2.cpu().numpy(), u3.cpu().numpy()) < 1e-10
    with pytest.raises(sft.SftError) as e:
        sft.sft_transfer(s, t, 16, sft.SFT_PREC_FP64, u_out=u, cg_warm_start=True, cg_mode=sft.SFT_CG_FP64)
    assert e.value.status == sft.SFT_ERR_UNSUPPORTED
    with pytest.raises(sft.SftError) as e:
        sft.sft_batch_create([s], [t], [dict(samples_per_elem=8, cg_warm_start=True)])
    assert e.value.status == sft.SFT_ERR_UNSUPPORTED
