"""Batched transfers (sft_batch_*): every request of a batch must equal the
same request run on its own (same samples and locations; the batch sums a
lane's few samples in plain FP32 before the compensated warp combine, so b
agrees to ~1e-7), the oracle within the FP32 bound, and repeated graph runs
must agree."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_00538_gb300 as sft  # noqa: E402

DEV = torch.device("cuda:0")
FIELDS2 = [W.paper_f1, W.paper_f2, W.paper_f3, W.field_sincos, W.field_gauss_jump_2d,
           W.linear_field([1, 2, -1]), lambda x: np.cos(3 * x[:, 0]) + x[:, 1], lambda x: x[:, 0] * x[:, 1]]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def batch_setup():
    src2 = W.as_precision(W.with_values(W.jittered_tri_mesh(40, 3), FIELDS2, np.float64), np.float32)
    f3 = [lambda x, f=f: f(x[:, :2]) + 0.5 * x[:, 2] for f in FIELDS2]
    src3 = W.as_precision(W.with_values(W.jittered_kuhn_mesh(9, 3), f3, np.float64), np.float32)
    s2, s3 = sft.mesh_source(src2, device=DEV), sft.mesh_source(src3, device=DEV)
    rng = np.random.default_rng(11)
    reqs = []
    for r in range(14):
        dim = 2 if r % 3 else 3
        if dim == 2:
            n = int(rng.integers(6, 30))
            tgt = W.as_precision(W.jittered_tri_mesh(n, 100 + r), np.float32)
        else:
            n = int(rng.integers(3, 8))
            tgt = W.as_precision(W.morton_reorder(W.jittered_kuhn_mesh(n, 100 + r)), np.float32)
        opt = dict(samples_per_elem=int(rng.choice([1, 7, 8, 16, 33, 64, 128])), seed=int(r), stream_id=r,
                   field_count=int(rng.integers(1, 9)), cg_tol=1e-12, cg_max_iter=2000,
                   alpha=float(rng.choice([1.0, 0.5])))
        reqs.append((dim, tgt, opt))
    srcs = [s2 if d == 2 else s3 for d, _, _ in reqs]
    tgts = [sft.mesh_target(t, device=DEV) for _, t, _ in reqs]
    return dict(src2=src2, src3=src3, srcs=srcs, tgts=tgts, reqs=reqs)


def test_batch_matches_single_transfers_and_oracle(batch_setup, orc):
    S = batch_setup
    b = sft.sft_batch_create(S["srcs"], S["tgts"], [o for _, _, o in S["reqs"]], autotune=True)
    status, st = sft.sft_batch_run(b)
    assert st["nreq"] == len(S["reqs"]) and st["nonconverged"] == 0
    assert st["empty_queries"] == 0
    for r, (dim, tgt, opt) in enumerate(S["reqs"]):
        nf = opt["field_count"]
        ub, bb = sft.sft_batch_result(b, r, b_out=np.zeros((nf, tgt.nnodes)))
        _, _, us = sft.sft_transfer(S["srcs"][r], S["tgts"][r], opt["samples_per_elem"], sft.SFT_PREC_FP32,
                                    seed=opt["seed"], stream_id=opt["stream_id"], alpha=opt["alpha"],
                                    cg_tol=1e-12, cg_max_iter=2000, field_count=nf,
                                    b_out=(bs := np.zeros((nf, tgt.nnodes))))
        for f in range(nf):
            assert _rel(bb[f], bs[f]) < 1e-6, (r, f)
            assert _rel(ub[f], us[f]) < 1e-5, (r, f)
        if r < 4:   # oracle on a few requests
            src = S["src2"] if dim == 2 else S["src3"]
            src_nf = W.Mesh(src.coords, src.conn, src.values[:nf])
            o = orc.transfer(src_nf, tgt, 1, opt["samples_per_elem"], seed=opt["seed"], stream=opt["stream_id"],
                             alpha=opt["alpha"], cg_tol=1e-12, cg_max_iter=2000)
            for f in range(nf):
                assert _rel(bb[f], o["b"][f]) < 1e-5
    # a second run replays the same work: same answers up to atomic ordering
    _, st2 = sft.sft_batch_run(b)
    for r, (_, tgt, opt) in enumerate(S["reqs"]):
        u1, _ = sft.sft_batch_result(b, r)
        assert np.isfinite(u1).all()
    assert st2["queries"] == st["queries"]
    b.close()


def test_batch_graph_and_tiles(batch_setup):
    S = batch_setup
    b = sft.sft_batch_create(S["srcs"], S["tgts"], [o for _, _, o in S["reqs"]], autotune=True)
    _, st = sft.sft_batch_run(b)
    assert st["graph"] in (0, 1)
    assert any(t > 0 for t in st["tile"])
    assert all(t in (0, 1, 2, 4, 8, 16) for t in st["tile"])
    b.close()


def test_batch_rejects_fp64_requests(batch_setup):
    S = batch_setup
    opts = [dict(o, precision=sft.SFT_PREC_FP64) for _, _, o in S["reqs"][:2]]
    with pytest.raises(sft.SftError) as ei:
        sft.sft_batch_create(S["srcs"][:2], S["tgts"][:2], opts)
    assert ei.value.status == 8


def _spmv(rp, col, val, x):
    rows = np.repeat(np.arange(len(rp) - 1), np.diff(rp))
    return np.bincount(rows, weights=val * x[col], minlength=len(rp) - 1)


@pytest.mark.parametrize("modes", ["mixed", "fp64", "one_fp64"])
def test_batch_cg_modes(batch_setup, orc, modes):
    """The batched solve in either CG mode: every (request, field) system's
    u has the true residual ||b - M u|| <= tol ||b|| (MIXED stops on it; the
    FP64 CG's recurrence residual may drift from it by rounding, 1e-11), and
    u equals the single transfer's in the same mode to the solve accuracy.
    One FP64 request makes the whole batch use the FP64 CG."""
    S = batch_setup
    reqs = S["reqs"][:8]
    mode = {"mixed": [0] * 8, "fp64": [1] * 8, "one_fp64": [0] * 7 + [1]}[modes]
    opts = [dict(o, cg_tol=1e-12, cg_mode=m) for (_, _, o), m in zip(reqs, mode)]
    b = sft.sft_batch_create(S["srcs"][:8], S["tgts"][:8], opts, autotune=False)
    _, st = sft.sft_batch_run(b)
    assert st["nonconverged"] == 0
    for r, (dim, tgt, opt) in enumerate(reqs):
        nf = opt["field_count"]
        ub, bb = sft.sft_batch_result(b, r, b_out=np.zeros((nf, tgt.nnodes)))
        rp, col, val = orc.mass_csr(tgt.coords, tgt.conn)
        for f in range(nf):
            res = np.linalg.norm(bb[f] - _spmv(rp, col, val, ub[f])) / np.linalg.norm(bb[f])
            assert res <= (2e-12 if modes == "mixed" else 1e-11), (r, f, res)
        _, _, us = sft.sft_transfer(S["srcs"][r], S["tgts"][r], opt["samples_per_elem"], sft.SFT_PREC_FP32,
                                    seed=opt["seed"], stream_id=opt["stream_id"], alpha=opt["alpha"],
                                    cg_tol=1e-12, cg_max_iter=2000, field_count=nf, cg_mode=mode[r])
        for f in range(nf):
            assert _rel(ub[f], us[f]) < 1e-5, (r, f)
    b.close()
