"""Transfer plans (the initialization / online split of Sec. 5.3): an online
transfer from recorded locations equals sft_transfer with the same options
and values (same samples, same elements and barycentric coordinates; only
the order of the FP64 atomic sums differs), and equals the oracle's transfer
of the new values after sft_source_set_values (FP32 bound 1e-5, FP64 1e-13)."""
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
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _case(dim, prec):
    if dim == 2:
        src, tgt, _ = W.config_meshes("tri2k", 1.0)
        fields = [W.field_sincos, W.paper_f2]
        new_fields = [W.paper_f3, W.linear_field([0.5, -1.0, 2.0])]
    else:
        src = W.jittered_kuhn_mesh(6, seed=4)
        tgt = W.morton_reorder(W.jittered_kuhn_mesh(4, seed=5))
        fields = [lambda x: np.sin(3 * x[:, 0]) * x[:, 1] + x[:, 2] ** 2, lambda x: x[:, 0] + 2 * x[:, 2]]
        new_fields = [lambda x: np.cos(2 * x[:, 1]) + x[:, 0] * x[:, 2], lambda x: 1.0 + 0 * x[:, 0]]
    dt = np.float64 if prec == sft.SFT_PREC_FP64 else np.float32
    src = W.as_precision(W.with_values(src, fields, np.float64), dt)
    tgt = W.as_precision(tgt, dt)
    src_new = W.as_precision(W.with_values(src, new_fields, np.float64), dt)
    return src, tgt, src_new


@pytest.mark.parametrize("dim,prec,N", [(2, sft.SFT_PREC_FP32, 16), (2, sft.SFT_PREC_FP64, 9),
                                        (3, sft.SFT_PREC_FP32, 33), (3, sft.SFT_PREC_FP64, 8)])
def test_plan_equals_transfer_and_oracle(orc, dim, prec, N):
    src, tgt, src_new = _case(dim, prec)
    s, t = sft.mesh_source(src), sft.mesh_target(tgt)
    tol = 1e-12 if prec == sft.SFT_PREC_FP64 else 1e-10
    pl = sft.sft_plan_create(s, t, N, precision=prec, seed=3, stream_id=1, cg_tol=tol, cg_max_iter=2000)
    nf, nv = 2, tgt.nnodes
    assert sft.sft_plan_bytes(pl) == (4 + dim * (8 if prec == sft.SFT_PREC_FP64 else 4)) * (nv + tgt.nelems * N)
    # online with the same values == sft_transfer
    bp, gp = np.zeros((nf, nv)), np.zeros((nf, nv))
    _, stp, up = sft.sft_plan_transfer(pl, b_out=bp, g_out=gp)
    bs, gs = np.zeros((nf, nv)), np.zeros((nf, nv))
    _, sts, us = sft.sft_transfer(s, t, N, prec, seed=3, stream_id=1, cg_tol=tol, cg_max_iter=2000, b_out=bs,
                                  g_out=gs)
    assert np.array_equal(gp, gs)
    for f in range(nf):
        assert _rel(bp[f], bs[f]) < 1e-14
        assert _rel(up[f], us[f]) < 1e-9
    assert stp["queries"] == sts["queries"]
    assert stp["fallback_queries"] == sts["fallback_queries"]
    # new source values: online == oracle transfer of the new values
    sft.sft_source_set_values(s, src_new.values)
    bp2 = np.zeros((nf, nv))
    _, _, up2 = sft.sft_plan_transfer(pl, b_out=bp2)
    o = orc.transfer(src_new, tgt, 1 if prec == sft.SFT_PREC_FP32 else 0, N, seed=3, stream=1, cg_tol=tol,
                     cg_max_iter=2000)
    bound = 1e-13 if prec == sft.SFT_PREC_FP64 else 1e-5
    for f in range(nf):
        assert _rel(bp2[f], o["b"][f]) < bound
        assert _rel(up2[f], o["u"][f]) < (1e-10 if prec == sft.SFT_PREC_FP64 else 1e-4)
    pl.close()


def test_plan_device_outputs_and_field_count():
    src, tgt, src_new = _case(2, sft.SFT_PREC_FP32)
    s, t = sft.mesh_source(src, device=DEV), sft.mesh_target(tgt, device=DEV)
    pl = sft.sft_plan_create(s, t, 64, seed=9, field_count=1, out_device=True)
    u = torch.zeros((1, tgt.nnodes), dtype=torch.float64, device=DEV)
    b = torch.zeros_like(u)
    sft.sft_plan_transfer(pl, u_out=u, b_out=b)
    torch.cuda.synchronize()
    bs = np.zeros((1, tgt.nnodes))
    sft.sft_transfer(s, t, 64, sft.SFT_PREC_FP32, seed=9, field_count=1, b_out=bs)
    assert _rel(b.cpu().numpy()[0], bs[0]) < 1e-14
    # repeated online transfers with changing values stay consistent
    for k in range(3):
        vals = torch.as_tensor(src_new.values * (1.0 + k)).to(DEV)
        sft.sft_source_set_values(s, vals)
        sft.sft_plan_transfer(pl, u_out=u, b_out=b)
        torch.cuda.synchronize()
        bs = np.zeros((1, tgt.nnodes))
        sft.sft_transfer(s, t, 64, sft.SFT_PREC_FP32, seed=9, field_count=1, b_out=bs)
        assert _rel(b.cpu().numpy()[0], bs[0]) < 1e-14
    pl.close()


def test_plan_rejects_bad_arguments():
    src, tgt, _ = _case(2, sft.SFT_PREC_FP32)
    s, t = sft.mesh_source(src), sft.mesh_target(tgt)
    with pytest.raises(sft.SftError):
        sft.sft_plan_create(s, t, 0)
    with pytest.raises(sft.SftError):
        sft.sft_plan_create(s, t, 8, field_count=9)
