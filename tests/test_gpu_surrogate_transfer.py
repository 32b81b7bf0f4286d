"""The surrogate-source transfer (fused sampler -> tensor-core network ->
exact-subsample fallback -> scatter) and the surrogate training set, against
the oracle.

Bounds. The network's forward matches the FP64 oracle network (same BF16
weights, BF16 activations) within eps * S, eps = 1e-2, S = max |f_net|
(the forward tests). The fallback decision compares that value with tau, so
it is unique only where the oracle's margin is farther than eps * S from
tau; elsewhere either decision is valid and the test only checks the GPU's
choice is consistent with the margin. b at node i is a sum over its
elements of |T| (alpha M g / |T| + 1/N sum_j (f_j - alpha g(X_j)) psi_i):
an error eps * S in every f_j and g_m moves it by at most
(1 + 2 alpha) eps S int psi_i (times 1.5 for the sampling fluctuation of the
psi_i sample means); that is the bound on nodes whose elements took the same
fallback decision on both sides. Exact-only transfers are FP32 mesh queries:
b within 1e-5 relative (the FP32 transfer bound)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_00538_gb300 as sft  # noqa: E402

EPS = 1e-2


def _gpu_params(orc, p64):
    p = p64.astype(np.float32).astype(np.float64)
    parts = orc.mlp_split(p)
    for i in (2, 4, 6):
        parts[i][...] = np.vectorize(orc.bf16_round)(parts[i])
    return p


def _meshes(dt, n_tgt):
    src = W.with_values(W.jittered_tri_mesh(20, seed=31), [W.field_sincos])
    if dt == 3:
        tgt = W.jittered_kuhn_mesh(n_tgt, seed=32)
    else:
        tgt = W.jittered_tri_mesh(n_tgt, seed=33)
    return src, tgt


def _run(net, src_h, tgt_h, tgt, N, seed, tau, s, alpha=1.0):
    E = len(tgt.conn)
    b = np.zeros(len(tgt.coords))
    g = np.zeros(len(tgt.coords))
    fb = np.zeros(E, np.int32)
    sf = np.zeros((E, N), np.float32)
    st, stats, u = sft.sft_transfer_surrogate(net, src_h, tgt_h, N, seed=seed, alpha=alpha, subsample=s, tau=tau,
                                              b_out=b, g_out=g, fallback_out=fb, sample_f_out=sf)
    return u, b, g, fb.astype(bool), sf, stats


# (3, 4, 8) and (2, 40, 8): 16 elements per tile (no prefetch of element data);
# (2, 40, 8) and (2, 40, 16) have more work units than SMs, so CTAs run paired
# tiles (with and without the prefetch); (3, 2, 200):
# an element spans two tiles
@pytest.mark.parametrize("dt,n_tgt,N", [(3, 4, 16), (3, 3, 50), (3, 2, 200), (2, 10, 16), (3, 4, 8), (2, 40, 8), (2, 40, 16)])
def test_surrogate_transfer_matches_oracle(orc, dt, n_tgt, N):
    from oracle import surrogate as S
    src, tgt = _meshes(dt, n_tgt)
    p = _gpu_params(orc, W.mlp_init(41))
    s, seed, alpha = 4, 17, 1.0
    # tau at the median oracle margin: about half the elements fall back
    probe = S.surrogate_transfer(p, tgt.coords, tgt.conn, N, seed=seed, alpha=alpha,
                                 exact=(src.coords, src.conn, src.values[0]), tau=np.inf, s=s)
    tau = float(np.median(probe["margin"]))
    ref = S.surrogate_transfer(p, tgt.coords, tgt.conn, N, seed=seed, alpha=alpha,
                               exact=(src.coords, src.conn, src.values[0]), tau=tau, s=s)
    net = sft.sft_mlp_create(p.astype(np.float32))
    src_h, tgt_h = sft.mesh_source(src), sft.mesh_target(tgt)
    u, b, g, fb, sf, stats = _run(net, src_h, tgt_h, tgt, N, seed, tau, s, alpha)
    Snet = max(np.abs(probe["f"]).max(), np.abs(probe["g"]).max())
    E, nv = len(tgt.conn), len(tgt.coords)

    # control values: network at the target nodes
    assert np.abs(g - ref["g"]).max() <= EPS * Snet
    # fallback decisions: unique away from tau, consistent near it
    near = np.abs(ref["margin"] - tau) <= EPS * Snet
    assert np.array_equal(fb[~near], ref["fallback"][~near])
    assert np.all(ref["margin"][fb] > tau - EPS * Snet)
    assert np.all(ref["margin"][~fb] <= tau + EPS * Snet)
    assert 0.2 * E < fb.sum() < 0.8 * E
    agree = fb == ref["fallback"]
    # per-sample values: network within eps*S, exact within FP32 rounding
    net_rows = agree & ~fb
    ex_rows = agree & fb
    assert np.abs(sf[net_rows] - ref["f"][net_rows]).max() <= EPS * Snet
    fmax = np.abs(src.values[0]).max()
    assert np.abs(sf[ex_rows] - ref["f"][ex_rows]).max() <= 1e-5 * fmax
    # the fused network is the standalone forward, bit for bit
    Xs = np.zeros((int(net_rows.sum()) * N, 3), np.float32)
    k = 0
    for t in np.nonzero(net_rows)[0]:
        _, X = orc.sample_element(1, dt, seed, 0, int(t), N, tgt.coords[tgt.conn[t]])
        Xs[k:k + N, :dt] = X
        k += N
    y = sft.sft_mlp_forward(net, Xs)
    assert np.array_equal(y.reshape(-1, N), sf[net_rows])
    # b on nodes whose elements took the same decision on both sides
    m = orc.lumped_mass(tgt.coords, tgt.conn)
    touched = np.zeros(nv, bool)
    touched[tgt.conn[~agree].ravel()] = True
    bound = 1.5 * (1 + 2 * alpha) * EPS * Snet * m + 1e-5 * np.abs(ref["b"]).max()
    assert np.all(np.abs(b - ref["b"])[~touched] <= bound[~touched])
    # statistics
    # the network runs on the target nodes, the subsample of every element,
    # and all N samples of the elements that keep it
    assert stats["net_queries"] == nv + E * s + (E - fb.sum()) * N
    assert stats["fallback_elems"] == fb.sum()
    assert stats["exact_queries"] == E * s + fb.sum() * (N - s)
    assert stats["cg_rel_resid"] <= 1e-10


@pytest.mark.parametrize("dt,n_tgt,N", [(3, 4, 16), (3, 2, 130), (2, 12, 9)])
def test_exact_only_transfer_matches_oracle(orc, dt, n_tgt, N):
    """No network: the plain mesh-query transfer of the 2D source onto the
    target (extruded along z in 3D). FP32 mesh queries: b within 1e-5."""
    from oracle import surrogate as S
    src, tgt = _meshes(dt, n_tgt)
    ref = S.surrogate_transfer(None, tgt.coords, tgt.conn, N, seed=5, exact=(src.coords, src.conn, src.values[0]))
    src_h, tgt_h = sft.mesh_source(src), sft.mesh_target(tgt)
    u, b, g, fb, sf, stats = _run(None, src_h, tgt_h, tgt, N, 5, 0.0, 0)
    assert fb.all()
    assert np.abs(g - ref["g"]).max() <= 1e-6 * np.abs(ref["g"]).max()
    assert np.abs(sf - ref["f"]).max() <= 1e-5 * np.abs(src.values[0]).max()
    assert np.linalg.norm(b - ref["b"]) <= 1e-5 * np.linalg.norm(ref["b"])
    assert np.linalg.norm(u - ref["u"]) <= 1e-5 * np.linalg.norm(ref["u"])
    assert stats["net_queries"] == 0


def test_exact_only_2d_equals_mesh_transfer():
    """In 2D the exact-only surrogate path and sft_transfer (FP32) draw the
    same samples from the same source: b agrees to summation order."""
    src, tgt = _meshes(2, 14)
    src_h, tgt_h = sft.mesh_source(src), sft.mesh_target(tgt)
    _, b, _, _, _, _ = _run(None, src_h, tgt_h, tgt, 24, 8, 0.0, 0)
    b2 = np.zeros((1, len(tgt.coords)))
    sft.sft_transfer(src_h, tgt_h, 24, precision=sft.SFT_PREC_FP32, seed=8, b_out=b2)
    assert np.linalg.norm(b - b2[0]) <= 1e-6 * np.linalg.norm(b2[0])


def test_pure_network_transfer(orc):
    """Network only (no exact source): no fallback, every sample from the
    network."""
    from oracle import surrogate as S
    src, tgt = _meshes(3, 3)
    p = _gpu_params(orc, W.mlp_init(42))
    ref = S.surrogate_transfer(p, tgt.coords, tgt.conn, 32, seed=3)
    net = sft.sft_mlp_create(p.astype(np.float32))
    u, b, g, fb, sf, stats = _run(net, None, sft.mesh_target(tgt), tgt, 32, 3, 0.0, 0)
    Snet = max(np.abs(ref["f"]).max(), np.abs(ref["g"]).max())
    assert not fb.any()
    assert np.abs(sf - ref["f"]).max() <= EPS * Snet
    m = orc.lumped_mass(tgt.coords, tgt.conn)
    assert np.all(np.abs(b - ref["b"]) <= 4.5 * EPS * Snet * m + 1e-5 * np.abs(ref["b"]).max())
    assert stats["exact_queries"] == 0 and stats["fallback_elems"] == 0


def test_tau_extremes(orc):
    """tau = 0 with a generic network sends every element to exact queries
    (then b equals the exact-only transfer's); a huge tau sends none."""
    src, tgt = _meshes(3, 3)
    p = _gpu_params(orc, W.mlp_init(43))
    net = sft.sft_mlp_create(p.astype(np.float32))
    src_h, tgt_h = sft.mesh_source(src), sft.mesh_target(tgt)
    _, b0, _, fb0, sf0, _ = _run(net, src_h, tgt_h, tgt, 16, 2, 0.0, 4)
    _, bx, _, fbx, sfx, _ = _run(None, src_h, tgt_h, tgt, 16, 2, 0.0, 0)
    assert fb0.all()
    assert np.array_equal(sf0, sfx)
    _, _, _, fb1, _, st1 = _run(net, src_h, tgt_h, tgt, 16, 2, 1e30, 4)
    assert not fb1.any() and st1["fallback_elems"] == 0


def test_surrogate_dataset_matches_oracle(orc):
    from oracle import surrogate as S
    src, _ = _meshes(2, 4)
    lo, hi = (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    pts_ref, f_ref, _ = S.surrogate_dataset(src.coords, src.conn, src.values[0], 5000, seed=77, stream_id=2,
                                            box_lo=lo, box_hi=hi)
    pts, f, mx = sft.sft_surrogate_dataset(sft.mesh_source(src), 5000, seed=77, stream_id=2, box_lo=lo, box_hi=hi)
    torch.cuda.synchronize()
    assert np.array_equal(pts.cpu().numpy(), pts_ref)
    fmax = np.abs(src.values[0]).max()
    assert np.abs(f.cpu().numpy() - f_ref).max() <= 1e-5 * fmax
    assert abs(mx - np.abs(f_ref).max()) <= 1e-5 * fmax


def test_surrogate_argument_errors(orc):
    src, tgt = _meshes(3, 2)
    net = sft.sft_mlp_create(W.mlp_init(1).astype(np.float32))
    src_h, tgt_h = sft.mesh_source(src), sft.mesh_target(tgt)
    with pytest.raises(sft.SftError) as e:
        sft.sft_transfer_surrogate(None, None, tgt_h, 8)
    assert e.value.status == sft.SFT_ERR_ARG
    with pytest.raises(sft.SftError) as e:
        sft.sft_transfer_surrogate(net, src_h, tgt_h, 8, subsample=9)
    assert e.value.status == sft.SFT_ERR_ARG
    with pytest.raises(sft.SftError) as e:
        sft.sft_transfer_surrogate(net, src_h, tgt_h, 8, tau=-1.0)
    assert e.value.status == sft.SFT_ERR_ARG
    o = sft._options(8, precision=sft.SFT_PREC_FP64)
    so = sft.sft_surrogate_opts()
    u = np.zeros(len(tgt.coords))
    import ctypes
    st = sft.lib().sft_transfer_surrogate(net.h, src_h.h, tgt_h.h, ctypes.byref(o), ctypes.byref(so),
                                          u.ctypes.data, None, None, None)
    assert st == sft.SFT_ERR_UNSUPPORTED
