"""Stratified sampling (SFT_SAMPLING_STRATIFIED) on the GPU against the oracle:
the strata are formed with correctly rounded operations in the path's
precision on both sides, so every sample's source element is bit-exact and
b, u meet the same bounds as the uniform scheme (FP64: 1e-13 / 1e-10; FP32:
1e-5 / 1e-4). The plan, batched and surrogate paths draw the same samples."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_00538_gb300 as sft  # noqa: E402

DEV = torch.device("cuda:0")
FP64, FP32, STRAT = sft.SFT_PREC_FP64, sft.SFT_PREC_FP32, sft.SFT_SAMPLING_STRATIFIED


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("name,scale,prec,N", [
    ("tri2k", 1.0, FP64, 16), ("tri2k", 1.0, FP32, 23), ("tri2k", 1.0, FP32, 1),
    ("tri4m", 3e-3, FP32, 64), ("tet5m", 2e-3, FP32, 27), ("tet5m", 2e-3, FP64, 30),
])
def test_stratified_transfer_parity(orc, name, scale, prec, N):
    src, tgt, _ = W.config_meshes(name, scale)
    s, t = sft.mesh_source(src, device=DEV), sft.mesh_target(tgt, device=DEV)
    nf = src.nfields
    u = torch.zeros((nf, tgt.nnodes), dtype=torch.float64, device=DEV)
    b = torch.zeros_like(u)
    se = torch.zeros((tgt.nelems, N), dtype=torch.int32, device=DEV)
    _, st, _ = sft.sft_transfer(s, t, N, prec, seed=3, stream_id=1, cg_tol=1e-13, cg_max_iter=2000, u_out=u,
                                b_out=b, sample_elem_out=se, sampling=STRAT)
    o = orc.transfer(src, tgt, 1 if prec == FP32 else 0, N, seed=3, stream=1, cg_tol=1e-13, cg_max_iter=2000,
                     want_sample_elem=True, sampling=1)
    assert np.array_equal(se.cpu().numpy(), o["sample_elem"])
    assert st["fallback_queries"] == o["fallback_queries"]
    bh, uh = b.cpu().numpy(), u.cpu().numpy()
    for f in range(nf):
        if prec == FP64:
            assert _rel(bh[f], o["b"][f]) < 1e-13
            assert _rel(uh[f], o["u"][f]) < 1e-10
        else:
            assert _rel(bh[f], o["b"][f]) < 1e-5
            assert _rel(uh[f], o["u"][f]) < 1e-4
    # the scheme changes the samples (not a no-op)
    se_u = torch.zeros_like(se)
    sft.sft_transfer(s, t, N, prec, seed=3, stream_id=1, cg_tol=1e-13, cg_max_iter=2000, u_out=u,
                     sample_elem_out=se_u)
    if N > 1:
        assert not np.array_equal(se_u.cpu().numpy(), se.cpu().numpy())
    else:
        assert np.array_equal(se_u.cpu().numpy(), se.cpu().numpy())   # m = 1: no strata


def test_stratified_plan_and_batch_equal_transfer():
    src = W.as_precision(W.with_values(W.jittered_tri_mesh(24, 3), [W.paper_f2, W.field_sincos], np.float64),
                         np.float32)
    tgt = W.as_precision(W.jittered_tri_mesh(17, 4), np.float32)
    s, t = sft.mesh_source(src, device=DEV), sft.mesh_target(tgt, device=DEV)
    N = 18
    bs = np.zeros((2, tgt.nnodes))
    sft.sft_transfer(s, t, N, FP32, seed=7, b_out=bs, sampling=STRAT)
    pl = sft.sft_plan_create(s, t, N, seed=7, sampling=STRAT)
    bp = np.zeros((2, tgt.nnodes))
    sft.sft_plan_transfer(pl, b_out=bp)
    for f in range(2):
        assert _rel(bp[f], bs[f]) < 1e-14
    pl.close()
    # batch: the same request twice plus a 3D one
    src3 = W.as_precision(W.with_values(W.jittered_kuhn_mesh(6, 2), [lambda x: x[:, 0] * x[:, 2] + 1.0], np.float64),
                          np.float32)
    tgt3 = W.as_precision(W.morton_reorder(W.jittered_kuhn_mesh(4, 5)), np.float32)
    s3, t3 = sft.mesh_source(src3, device=DEV), sft.mesh_target(tgt3, device=DEV)
    opts = [dict(samples_per_elem=N, seed=7, sampling=STRAT), dict(samples_per_elem=N, seed=7, sampling=STRAT),
            dict(samples_per_elem=29, seed=2, sampling=STRAT)]
    bt = sft.sft_batch_create([s, s, s3], [t, t, t3], opts, autotune=False)
    sft.sft_batch_run(bt)
    for r in range(2):
        _, bb = sft.sft_batch_result(bt, r, b_out=np.zeros((2, tgt.nnodes)))
        for f in range(2):
            assert _rel(bb[f], bs[f]) < 1e-6
    _, bb3 = sft.sft_batch_result(bt, 2, b_out=np.zeros((1, tgt3.nnodes)))
    b3 = np.zeros((1, tgt3.nnodes))
    sft.sft_transfer(s3, t3, 29, FP32, seed=2, b_out=b3, sampling=STRAT)
    assert _rel(bb3[0], b3[0]) < 1e-6
    bt.close()


@pytest.mark.parametrize("dt,N", [(2, 16), (3, 27)])
def test_stratified_surrogate_exact_path(orc, dt, N):
    """The surrogate path's sampler with strata: exact-only transfer equals the
    oracle's (FP32 mesh queries, b within 1e-5)."""
    from oracle import surrogate as S
    src = W.with_values(W.jittered_tri_mesh(20, seed=31), [W.field_sincos])
    tgt = W.jittered_kuhn_mesh(3, seed=32) if dt == 3 else W.jittered_tri_mesh(10, seed=33)
    ref = S.surrogate_transfer(None, tgt.coords, tgt.conn, N, seed=5, exact=(src.coords, src.conn, src.values[0]),
                               sampling=1)
    b = np.zeros(len(tgt.coords))
    sf = np.zeros((len(tgt.conn), N), np.float32)
    sft.sft_transfer_surrogate(None, sft.mesh_source(src), sft.mesh_target(tgt), N, seed=5, subsample=0, b_out=b,
                               sample_f_out=sf, sampling=STRAT)
    assert np.abs(sf - ref["f"]).max() <= 1e-5 * np.abs(src.values[0]).max()
    assert np.linalg.norm(b - ref["b"]) <= 1e-5 * np.linalg.norm(ref["b"])


def test_stratified_rejects_unknown_scheme():
    src, tgt, _ = W.config_meshes("tri2k", 1.0)
    s, t = sft.mesh_source(src), sft.mesh_target(tgt)
    with pytest.raises(sft.SftError) as e:
        sft.sft_transfer(s, t, 8, FP32, sampling=5)
    assert e.value.status == sft.SFT_ERR_ARG
    with pytest.raises(sft.SftError) as e:   # digits exact only up to 2^20 samples per element
        sft.sft_transfer(s, t, (1 << 20) + 1, FP32, sampling=STRAT)
    assert e.value.status == sft.SFT_ERR_UNSUPPORTED
