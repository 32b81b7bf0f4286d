"""Round trips mesh 1 -> mesh 2 -> mesh 1 (the iterative analysis of Sec. 5)
through two transfer plans, against the oracle's round trip with the same
seeds (every round trip reuses each leg's samples). Each leg is a stable
projection that matches the oracle's leg within the transfer bound (FP64
path: u within 1e-10; FP32 path: 1e-4), so after L legs the fields agree
within L times that bound."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_00538_gb300 as sft  # noqa: E402

DEV = torch.device("cuda:0")


def _meshes():
    a = W.with_values(W.delaunay_tri_mesh(300, 14, 3), [W.paper_f2], np.float64)
    b = W.with_values(W.jittered_tri_mesh(7, 4), [lambda x: 0.0 * x[:, 0]], np.float64)
    return a, b


@pytest.mark.parametrize("prec,N,iters", [(sft.SFT_PREC_FP64, 8, 3), (sft.SFT_PREC_FP32, 20, 4)])
def test_roundtrip_matches_oracle(orc, prec, N, iters):
    a, b = _meshes()
    s1, t1 = sft.mesh_source(a, device=DEV), sft.mesh_target(a, device=DEV)
    s2, t2 = sft.mesh_source(b, device=DEV), sft.mesh_target(b, device=DEV)
    tol = 1e-13 if prec == sft.SFT_PREC_FP64 else 1e-12
    rt = sft.RoundTrip(s1, t1, s2, t2, N, precision=prec, seeds=(5, 6), cg_tol=tol, cg_max_iter=2000)
    f = torch.as_tensor(a.values.copy()).to(DEV)
    rt.run(f, iters)
    torch.cuda.synchronize()
    assert rt.queries == (b.nnodes + b.nelems * N) + (a.nnodes + a.nelems * N)
    errs, f_orc = orc.roundtrip(a, b, a.values[0], iters, 1 if prec == sft.SFT_PREC_FP32 else 0, N, seeds=(5, 6),
                                cg_tol=tol, cg_max_iter=2000)
    fg = f.cpu().numpy()[0]
    legs = 2 * iters
    bound = legs * (1e-10 if prec == sft.SFT_PREC_FP64 else 1e-4)
    assert np.linalg.norm(fg - f_orc) <= bound * np.linalg.norm(f_orc)
    # the two errors of the analysis, computed from the GPU field, agree with the oracle's
    m1 = orc.lumped_mass(a.coords, a.conn)
    ref = a.values[0]
    e_l2 = np.linalg.norm(fg - ref) / np.linalg.norm(ref)
    e_mass = abs(m1 @ fg - m1 @ ref) / abs(m1 @ ref)
    assert abs(e_l2 - errs[-1][0]) <= bound * 10 * max(e_l2, 1e-3)
    assert abs(e_mass - errs[-1][1]) <= bound * 10
    rt.close()


def test_roundtrip_linear_field_is_preserved():
    """alpha = 1 and a linear field: every leg reproduces it (the residual
    vanishes), so any number of round trips leaves it unchanged."""
    a, b = _meshes()
    lin = W.linear_field([0.5, 2.0, -1.0])
    a = W.with_values(a, [lin], np.float64)
    s1, t1 = sft.mesh_source(a, device=DEV), sft.mesh_target(a, device=DEV)
    s2, t2 = sft.mesh_source(b, device=DEV), sft.mesh_target(b, device=DEV)
    rt = sft.RoundTrip(s1, t1, s2, t2, 16, precision=sft.SFT_PREC_FP64, cg_tol=1e-14, cg_max_iter=2000)
    f = torch.as_tensor(a.values.copy()).to(DEV)
    rt.run(f, 5)
    torch.cuda.synchronize()
    assert np.abs(f.cpu().numpy()[0] - a.values[0]).max() <= 1e-10 * np.abs(a.values[0]).max()
    rt.close()


def test_roundtrip_warm_start_matches_cold():
    """Warm-started legs (each solve from that leg's previous result) give the
    cold-started round trips' fields to the solve tolerance: two solutions of
    one leg differ by at most 2 cond(M) tol, cond(M) <= 5 max/min diagonal
    (< 600 on these meshes), and 8 stable legs add at most 8 such terms."""
    a, b = _meshes()
    s1, t1 = sft.mesh_source(a, device=DEV), sft.mesh_target(a, device=DEV)
    s2, t2 = sft.mesh_source(b, device=DEV), sft.mesh_target(b, device=DEV)
    out = []
    for warm in (False, True):
        rt = sft.RoundTrip(s1, t1, s2, t2, 12, seeds=(3, 4), cg_tol=1e-12, cg_max_iter=2000, warm_start=warm)
        f = torch.as_tensor(a.values.copy()).to(DEV)
        rt.run(f, 4)
        torch.cuda.synchronize()
        out.append(f.cpu().numpy()[0])
        rt.close()
    assert np.linalg.norm(out[1] - out[0]) <= 1e-8 * np.linalg.norm(out[0])
