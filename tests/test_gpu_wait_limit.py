"""Failure detection on the device path without a GPU fault: every grid
barrier wait of the cooperative CG kernels is bounded. With the limit set far
below a barrier's latency the waits run out; the kernel records the expiry in
its error word, every block returns, and the call reports
SFT_ERR_DEVICE_STATUS. The stream and the context stay usable: the same
target solves and transfers correctly once the limit is restored."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_00538_gb300 as sft  # noqa: E402

DEV = torch.device("cuda:0")
SFT_ERR_ARG, SFT_ERR_DEVICE_STATUS = 1, 7


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("cg_mode", [sft.SFT_CG_FP64, sft.SFT_CG_MIXED])
def test_expired_barrier_wait_is_reported_and_the_stream_recovers(orc, cg_mode):
    m = W.jittered_tri_mesh(200, 3)          # 80,000 triangles: tens of cooperative blocks
    t = sft.mesh_target(m, device=DEV)
    b = np.random.default_rng(5).standard_normal((1, m.nnodes))
    sft.sft_target_set_wait_limit(t, 1e-9)
    with pytest.raises(sft.SftError) as ei:
        sft.sft_mass_solve(t, b, tol=1e-12, max_iter=1000, cg_mode=cg_mode)
    assert ei.value.status == SFT_ERR_DEVICE_STATUS
    sft.sft_target_set_wait_limit(t, 2.0)
    u, it, rr = sft.sft_mass_solve(t, b, tol=1e-12, max_iter=1000, cg_mode=cg_mode)
    assert rr <= 1e-12
    rp, col, val = orc.mass_csr(m.coords, m.conn)
    uo, _, _ = orc.pcg(rp, col, val, b[0], tol=1e-12, max_iter=1000)
    assert _rel(u[0], uo) < 1e-9


def test_transfer_reports_expired_wait_then_succeeds(orc):
    src, tgt, _ = W.config_meshes("tri4m", 1e-2)
    s = sft.mesh_source(src, device=DEV)
    t = sft.mesh_target(tgt, device=DEV)
    sft.sft_target_set_wait_limit(t, 1e-9)
    with pytest.raises(sft.SftError) as ei:
        sft.sft_transfer(s, t, 16, sft.SFT_PREC_FP32, cg_tol=1e-12)
    assert ei.value.status == SFT_ERR_DEVICE_STATUS
    sft.sft_target_set_wait_limit(t, 2.0)
    b = np.zeros((1, tgt.nnodes))
    _, st, u = sft.sft_transfer(s, t, 16, sft.SFT_PREC_FP32, cg_tol=1e-12, b_out=b)
    o = orc.transfer(src, tgt, 1, 16, cg_tol=1e-12)
    assert _rel(b[0], o["b"][0]) < 1e-5
    assert _rel(u[0], o["u"][0]) < 1e-4


def test_wait_limit_arguments():
    m = W.jittered_tri_mesh(4, 0)
    t = sft.mesh_target(m, device=DEV)
    for bad in (0.0, -1.0, float("nan"), float("inf"), 1e9):
        with pytest.raises(sft.SftError) as ei:
            sft.sft_target_set_wait_limit(t, bad)
        assert ei.value.status == SFT_ERR_ARG
