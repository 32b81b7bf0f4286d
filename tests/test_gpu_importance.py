"""Importance sampling (SFT_SAMPLING_IMPORTANCE) and per-element adaptive
sample counts (adapt_ref_measure) on the GPU against the oracle. The sample
maps, the component choice (integer bits of a Philox word) and the adaptive
counts (FP64 operations in the same order on both sides) are reproduced
exactly, so every sample's source element is bit-exact (padding -1 past each
element's count); b and u meet the uniform scheme's bounds (FP64 1e-13 /
1e-10; FP32 1e-5 / 1e-4: the FP32 path forms the weight 1 / (|T| p_t) in
FP32, the oracle in FP64, a 1e-7 relative difference per sample). The
entry points that do not take the schemes refuse them."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_00538_gb300 as sft  # noqa: E402

DEV = torch.device("cuda:0")
FP64, FP32, IMP = sft.SFT_PREC_FP64, sft.SFT_PREC_FP32, sft.SFT_SAMPLING_IMPORTANCE


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _rel_max(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(b)), 1e-300))


def _graded(mesh):
    m = W.Mesh(mesh.coords ** 2, mesh.conn, None)
    W._fix_orientation(m)
    return m


CASES = [
    # name, scale, precision, N, sampling, adaptive
    ("tri2k", 1.0, FP64, 16, IMP, False),
    ("tri2k", 1.0, FP32, 7, IMP, False),
    ("tri4m", 3e-3, FP32, 64, IMP, False),
    ("tet5m", 2e-3, FP32, 20, IMP, False),
    ("tet5m", 2e-3, FP64, 9, IMP, False),
    ("tri2k", 1.0, FP64, 12, 0, True),
    ("tri4m", 3e-3, FP32, 16, 0, True),
    ("tri4m", 3e-3, FP32, 16, IMP, True),
    ("tet5m", 2e-3, FP32, 8, IMP, True),
    ("graded2d", 1.0, FP32, 10, 0, True),
]


@pytest.mark.parametrize("name,scale,prec,N,sampling,adapt", CASES)
def test_importance_and_adaptive_parity(orc, name, scale, prec, N, sampling, adapt):
    if name == "graded2d":
        src = W.with_values(W.jittered_tri_mesh(30, 3), [W.paper_f2])
        tgt = _graded(W.delaunay_tri_mesh(500, 8, 4))
    else:
        src, tgt, _ = W.config_meshes(name, scale)
    meas = W._signed_measure(tgt.coords.astype(np.float64), tgt.conn)
    ref = float(meas.sum() / tgt.nelems) if adapt else 0.0
    s, t = sft.mesh_source(src, device=DEV), sft.mesh_target(tgt, device=DEV)
    nf = src.nfields
    nmax = N * (8 if adapt else 1)
    u = torch.zeros((nf, tgt.nnodes), dtype=torch.float64, device=DEV)
    b = torch.zeros_like(u)
    se = torch.zeros((tgt.nelems, nmax), dtype=torch.int32, device=DEV)
    _, st, _ = sft.sft_transfer(s, t, N, prec, seed=3, stream_id=1, cg_tol=1e-13, cg_max_iter=2000, u_out=u,
                                b_out=b, sample_elem_out=se, sampling=sampling, adapt_ref_measure=ref)
    o = orc.transfer(src, tgt, 1 if prec == FP32 else 0, N, seed=3, stream=1, cg_tol=1e-13, cg_max_iter=2000,
                     want_sample_elem=True, sampling=sampling, adapt_ref_measure=ref)
    assert np.array_equal(se.cpu().numpy(), o["sample_elem"])
    assert st["fallback_queries"] == o["fallback_queries"]
    assert st["queries"] == tgt.nnodes + o["samples"]
    if adapt:
        assert o["samples"] != N * tgt.nelems            # the counts do vary
    bh, uh = b.cpu().numpy(), u.cpu().numpy()
    lim_b, lim_u = (1e-13, 1e-10) if prec == FP64 else (1e-5, 1e-4)
    for f in range(nf):
        assert _rel(bh[f], o["b"][f]) < lim_b and _rel_max(bh[f], o["b"][f]) < lim_b, (f, _rel(bh[f], o["b"][f]))
        assert _rel(uh[f], o["u"][f]) < lim_u and _rel_max(uh[f], o["u"][f]) < lim_u


def test_importance_changes_the_samples_and_keeps_the_load_sum():
    """The scheme draws other points than uniform sampling, and sum_i b_i,
    an estimate of int f^s (partition of unity), stays near the exact
    integral for both schemes: within 1e-3 absolute on a field of scale 1
    whose integral is small (0.031; its +-0.5 jump cancels), the Monte Carlo
    error of 6,000 elements x 16 samples."""
    src, tgt, _ = W.config_meshes("tri4m", 3e-3)
    s, t = sft.mesh_source(src, device=DEV), sft.mesh_target(tgt, device=DEV)
    N = 16
    se_u = torch.zeros((tgt.nelems, N), dtype=torch.int32, device=DEV)
    se_i = torch.zeros_like(se_u)
    bu = np.zeros((1, tgt.nnodes))
    bi = np.zeros((1, tgt.nnodes))
    sft.sft_transfer(s, t, N, FP32, b_out=bu)
    sft.sft_transfer(s, t, N, FP32, b_out=bi, sampling=IMP)
    _, i_s, _ = sft.sft_conservation_error(s, t, np.zeros(tgt.nnodes))
    assert abs(bi.sum() - i_s) < 1e-3 and abs(bu.sum() - i_s) < 1e-3
    uu = torch.zeros((1, tgt.nnodes), dtype=torch.float64, device=DEV)
    sft.sft_transfer(s, t, N, FP32, u_out=uu, sample_elem_out=se_u)
    sft.sft_transfer(s, t, N, FP32, u_out=uu, sample_elem_out=se_i, sampling=IMP)
    assert not np.array_equal(se_u.cpu().numpy(), se_i.cpu().numpy())


def test_schemes_refused_where_not_supported():
    src, tgt, _ = W.config_meshes("tri2k", 1.0)
    s, t = sft.mesh_source(src), sft.mesh_target(tgt)
    with pytest.raises(sft.SftError) as e:
        sft.sft_plan_create(s, t, 8, sampling=IMP)
    assert e.value.status == sft.SFT_ERR_UNSUPPORTED
    with pytest.raises(sft.SftError) as e:
        sft.sft_transfer(s, t, 8, FP32, sampling=sft.SFT_SAMPLING_STRATIFIED, adapt_ref_measure=1e-3)
    assert e.value.status == sft.SFT_ERR_UNSUPPORTED
    with pytest.raises(sft.SftError) as e:
        sft.sft_transfer(s, t, 8, FP32, adapt_ref_measure=-1.0)
    assert e.value.status == sft.SFT_ERR_ARG
    with pytest.raises(sft.SftError) as e:
        sft.sft_transfer_surrogate(None, s, t, 8, sampling=IMP)
    assert e.value.status == sft.SFT_ERR_UNSUPPORTED
