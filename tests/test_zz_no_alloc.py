"""The allocation-free solve entry point (sft_mass_solve_static), for callers
that cannot allocate device memory at solve time. It must give the same
solution as sft_mass_solve on the same matrix, on consecutive calls that
reuse its fixed work array, and refuse problems larger than that array.
Kept in its own file, collected after every other test."""
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


@pytest.mark.parametrize("dim,nrhs", [(2, 1), (3, 3)])
def test_static_solve_matches_mass_solve_twice(dim, nrhs):
    m = W.delaunay_tri_mesh(3000, 20, 9) if dim == 2 else W.morton_reorder(W.jittered_kuhn_mesh(8, 9))
    t = sft.mesh_target(m, device=DEV)
    rp, col, val, _ = sft.sft_target_mass(t)
    rp_d = torch.as_tensor(rp.astype(np.int32)).to(DEV)
    col_d = torch.as_tensor(col).to(DEV)
    val_d = torch.as_tensor(val).to(DEV)
    rng = np.random.default_rng(7)
    for call in range(2):                      # the second call reuses the array's old contents
        b = rng.standard_normal((nrhs, m.nnodes))
        u_ref, it_ref, _ = sft.sft_mass_solve(t, b, tol=1e-13, max_iter=2000)
        u = torch.full((nrhs, m.nnodes), float("nan"), dtype=torch.float64, device=DEV)
        it, rr = sft.sft_mass_solve_static(rp_d, col_d, val_d, torch.as_tensor(b).to(DEV), u,
                                           tol=1e-13, max_iter=2000)
        torch.cuda.synchronize()
        assert rr <= 1e-13
        uh = u.cpu().numpy()
        for f in range(nrhs):
            assert _rel(uh[f], u_ref[f]) < 1e-10


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
