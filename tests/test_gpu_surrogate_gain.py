"""What the trained network gains over the method without it. The paper's
motivating case is a black-box source whose point queries are costly: the
surrogate transfer issues exact queries only for its fallback subsample and
for the elements that fall back, and the network answers the rest on the
tensor cores. Here the exact source is the tri4m mesh field (2D, 1/20 of the
benchmark's element counts) with a stand-in cost added to every exact query
(exact_cost dependent FMAs), and both transfers run on the same samples:

* at equal accuracy: the surrogate transfer's supermesh L2 error (exact 2D
  mesh-intersection judge) is within 25 % of the exact-query transfer's;
* it issues fewer exact queries (below 80 % of the exact path's);
* with the mesh query alone (cost 0) the exact path is faster, with a costly
  source the surrogate path is, and the crossover cost lies between.

The measured times, query counts and the crossover are printed (pytest -s)."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_00538_gb300 as sft  # noqa: E402

DEV = torch.device("cuda:0")
COSTS = (0, 50_000, 200_000)


def _time(fn, reps=3):
    fn()
    ms, st = [], None
    for _ in range(reps):
        st = fn()
        ms.append(st["ms_total"])
    return float(np.median(ms)), st


def test_surrogate_gain_over_a_costly_exact_source():
    src, tgt, p = W.config_meshes("tri4m", 0.05)
    N, tol = p["samples_per_elem"], p["cg_tol"]
    S = sft.mesh_source(src, device=DEV)
    T = sft.mesh_target(tgt, device=DEV)
    pts, f, fmax = sft.sft_surrogate_dataset(S, 1_000_000, seed=1, box_lo=(0.0, 0.0, 0.0), box_hi=(1.0, 1.0, 0.0))
    net = sft.sft_mlp_create(W.mlp_init(0).astype(np.float32))
    hist = sft.sft_mlp_train(net, pts, f, epochs=40, batch=16384, lr=2e-3, lr_final=1e-4)
    assert hist[-1] < hist[0]
    tau = 1e-2 * fmax
    u_plain = torch.zeros(tgt.nnodes, dtype=torch.float64, device=DEV)
    u_sur = torch.zeros_like(u_plain)

    def plain(cost):
        return lambda: sft.sft_transfer_surrogate(None, S, T, N, cg_tol=tol, u_out=u_plain, exact_cost=cost)[1]

    def sur(cost):
        return lambda: sft.sft_transfer_surrogate(net, S, T, N, cg_tol=tol, subsample=4, tau=tau, u_out=u_sur,
                                                  exact_cost=cost)[1]

    rows = []
    for c in COSTS:
        tp, sp = _time(plain(c))
        ts, ss = _time(sur(c))
        rows.append((c, tp, ts, sp["exact_queries"], ss["exact_queries"], ss["fallback_elems"]))
    # accuracy of both (the last runs): supermesh L2 error and conservation error
    e_p, n_p = sft.sft_mi_l2_error(S, T, u_plain, 0)
    e_s, n_s = sft.sft_mi_l2_error(S, T, u_sur, 0)
    m_p = sft.sft_conservation_error(S, T, u_plain)[0]
    m_s = sft.sft_conservation_error(S, T, u_sur)[0]
    q_plain, q_sur = rows[0][3], rows[0][4]
    # line fits T(c) = a + b c for both paths; crossover where they meet
    cs = np.array([r[0] for r in rows], float)
    ap, bp = np.polyfit(cs, [r[1] for r in rows], 1)[::-1]
    as_, bs = np.polyfit(cs, [r[2] for r in rows], 1)[::-1]
    c_star = (as_ - ap) / (bp - bs)
    # cost of one exact query at the crossover, in GPU time per query of the
    # exact path (its slope over its query count)
    ns_star = c_star * bp * 1e6 / q_plain
    print(f"\nsurrogate gain (2D, {tgt.nelems} target / {src.nelems} source triangles, N = {N}):")
    for c, tp, ts, qp, qs, fb in rows:
        print(f"  exact_cost {c:6d} FMA: exact path {tp:8.3f} ms ({qp} exact queries), "
              f"surrogate {ts:8.3f} ms ({qs} exact queries, {fb} fallback elements)")
    print(f"  E_L2 exact path {e_p / n_p:.5f}, surrogate {e_s / n_s:.5f}; E_mass {m_p:.2e} / {m_s:.2e}")
    print(f"  crossover: {c_star:.0f} FMA per exact query = {ns_star:.2f} ns of GPU time per query")
    assert q_sur < 0.8 * q_plain
    assert e_s / n_s <= 1.25 * e_p / n_p
    assert rows[0][2] > rows[0][1]            # a mesh query is cheaper than the network
    assert rows[-1][2] < rows[-1][1]          # a costly black box is not
    assert 0 < c_star < COSTS[-1]
