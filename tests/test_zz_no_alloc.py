"""The allocation-free solve entry point (sft_mass_solve_static), for callers
that cannot allocate device memory at solve time (a coupled code whose memory
pool owns the device, a time-stepping loop that must not call cudaMalloc or
cudaFree). It must give the oracle's FP64 Jacobi-PCG solution and the same
iterations as sft_mass_solve's FP64 CG on the same matrix, on consecutive
calls that reuse its fixed work array, leave the device's free memory
unchanged, refuse problems larger than that array (checked at the limit) and
matrices without a positive diagonal. Kept in its own file, collected after
every other test."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_00538_gb300 as sft  # noqa: E402

DEV = torch.device("cuda:0")


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dev_csr(rp, col, val):
    return (torch.as_tensor(np.ascontiguousarray(rp, np.int32)).to(DEV),
            torch.as_tensor(np.ascontiguousarray(col, np.int32)).to(DEV),
            torch.as_tensor(np.ascontiguousarray(val, np.float64)).to(DEV))


@pytest.mark.parametrize("dim,nrhs", [(2, 1), (3, 3)])
def test_static_solve_matches_oracle_and_mass_solve_twice(orc, dim, nrhs):
    m = W.delaunay_tri_mesh(3000, 20, 9) if dim == 2 else W.morton_reorder(W.jittered_kuhn_mesh(8, 9))
    t = sft.mesh_target(m, device=DEV)
    rp, col, val, _ = sft.sft_target_mass(t)
    rp_d, col_d, val_d = _dev_csr(rp, col, val)
    rp_o, col_o, val_o = orc.mass_csr(m.coords, m.conn)
    rng = np.random.default_rng(7)
    for call in range(2):                      # the second call reuses the array's old contents
        b = rng.standard_normal((nrhs, m.nnodes))
        u_ref, it_ref, _ = sft.sft_mass_solve(t, b, tol=1e-13, max_iter=2000, cg_mode=sft.SFT_CG_FP64)
        u = torch.full((nrhs, m.nnodes), float("nan"), dtype=torch.float64, device=DEV)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(DEV)[0]
        it, rr = sft.sft_mass_solve_static(rp_d, col_d, val_d, torch.as_tensor(b).to(DEV), u,
                                           tol=1e-13, max_iter=2000)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info(DEV)[0] == free0   # nothing allocated on the device
        assert rr <= 1e-13
        assert it == it_ref                    # the same FP64 Jacobi-PCG, the same reductions
        uh = u.cpu().numpy()
        for f in range(nrhs):
            assert _rel(uh[f], u_ref[f]) < 1e-10
            uo, _, _ = orc.pcg(rp_o, col_o, val_o, b[f], tol=1e-13, max_iter=2000)
            assert _rel(uh[f], uo) < 1e-10


def _tridiag(n):
    """SPD tridiagonal [1, 4, 1] in CSR (int32 row_ptr / col, FP64 values)."""
    cnt = np.full(n, 3, np.int64)
    cnt[0] = cnt[-1] = 2
    rp = np.zeros(n + 1, np.int64)
    rp[1:] = np.cumsum(cnt)
    col = np.zeros(rp[-1], np.int32)
    val = np.zeros(rp[-1])
    i = np.arange(n)
    pos = rp[:-1].copy()
    for off, v in ((-1, 1.0), (0, 4.0), (1, 1.0)):
        j = i + off
        ok = (j >= 0) & (j < n)
        col[pos[ok]] = j[ok]
        val[pos[ok]] = v
        pos[ok] += 1
    return rp, col, val


def test_static_solve_eight_rhs_at_the_limit(orc):
    """With 8 right-hand sides the work space holds 8 n (1 + 4 * 8) bytes plus
    per-block partials: n = 127,000 fits in 32 MiB (15 KB to spare), n =
    127,100 does not and is refused before any device work."""
    nrhs = 8
    for n, fits in ((127_000, True), (127_100, False)):
        rp, col, val = _tridiag(n)
        rp_d, col_d, val_d = _dev_csr(rp, col, val)
        b = np.random.default_rng(n).standard_normal((nrhs, n))
        u = torch.zeros((nrhs, n), dtype=torch.float64, device=DEV)
        if not fits:
            with pytest.raises(sft.SftError) as ei:
                sft.sft_mass_solve_static(rp_d, col_d, val_d, torch.as_tensor(b).to(DEV), u)
            assert ei.value.status == 1
            continue
        it, rr = sft.sft_mass_solve_static(rp_d, col_d, val_d, torch.as_tensor(b).to(DEV), u, tol=1e-12)
        assert rr <= 1e-12
        uh = u.cpu().numpy()
        for f in (0, 7):
            uo, _, _ = orc.pcg(rp, col, val, b[f], tol=1e-12, max_iter=1000)
            assert _rel(uh[f], uo) < 1e-10


def test_static_solve_rejects_oversize_problem():
    n = 5_000_000                               # 8 n (1 + 4) bytes > 32 MiB
    rp = torch.zeros(n + 1, dtype=torch.int32, device=DEV)
    col = torch.zeros(1, dtype=torch.int32, device=DEV)
    val = torch.ones(1, dtype=torch.float64, device=DEV)
    b = torch.zeros((1, n), dtype=torch.float64, device=DEV)
    u = torch.zeros_like(b)
    with pytest.raises(sft.SftError) as ei:
        sft.sft_mass_solve_static(rp, col, val, b, u)
    assert ei.value.status == 1


def test_static_solve_rejects_missing_diagonal_and_recovers(orc):
    """A row without a positive diagonal entry is reported as SFT_ERR_ARG
    (the matrix cannot be SPD); the next call on the same work array works."""
    n = 1000
    rp, col, val = _tridiag(n)
    bad = val.copy()
    bad[rp[500] + 1] = 0.0                     # row 500's diagonal
    b = np.random.default_rng(3).standard_normal((1, n))
    u = torch.zeros((1, n), dtype=torch.float64, device=DEV)
    with pytest.raises(sft.SftError) as ei:
        sft.sft_mass_solve_static(*_dev_csr(rp, col, bad), torch.as_tensor(b).to(DEV), u)
    assert ei.value.status == 1
    it, rr = sft.sft_mass_solve_static(*_dev_csr(rp, col, val), torch.as_tensor(b).to(DEV), u, tol=1e-12)
    uo, _, _ = orc.pcg(rp, col, val, b[0], tol=1e-12, max_iter=1000)
    assert _rel(u.cpu().numpy()[0], uo) < 1e-10


def test_static_solve_wrapper_checks_arguments():
    rp, col, val = _tridiag(100)
    rp_d, col_d, val_d = _dev_csr(rp, col, val)
    b = torch.zeros((1, 100), dtype=torch.float64, device=DEV)
    u = torch.zeros((1, 100), dtype=torch.float64, device=DEV)
    with pytest.raises(TypeError):
        sft.sft_mass_solve_static(rp_d.to(torch.int64), col_d, val_d, b, u)
    with pytest.raises(TypeError):
        sft.sft_mass_solve_static(rp_d, col_d, val_d, b.float(), u)
    with pytest.raises(ValueError):
        sft.sft_mass_solve_static(rp_d, col_d, val_d, b, torch.zeros((1, 99), dtype=torch.float64, device=DEV))
    with pytest.raises(ValueError):
        sft.sft_mass_solve_static(rp_d, col_d, val_d, b, torch.zeros((1, 200), dtype=torch.float64, device=DEV)[:, ::2])
    with pytest.raises(ValueError):
        sft.sft_mass_solve_static(rp_d, col_d[:10], val_d, b, u)
    with pytest.raises(ValueError):
        sft.sft_mass_solve_static(rp_d.cpu(), col_d, val_d, b, u)
