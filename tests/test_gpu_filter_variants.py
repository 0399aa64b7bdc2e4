"""Filter and degree-correction variants through the C-ABI (Sec. IV-D, Fig. 4, Table II).

* The sign of tau (Fig. 4): on a graph shaped like the paper's benchmark graphs (100,000 nodes,
  56 blocks, 2.5 within-block edges per between-block edge; Table II's L = 60, d = 32), the
  partition quality of the FFP embedding (k-means with the planted number of blocks, NMI and
  pairwise F1 against the planted blocks) is best for a negative tau and clearly worse for every
  tau >= 0, as the paper reports for its F1-score.
* Table II's settings: see test_table2_settings_error_budget.
"""
import numpy as np
import pytest

import oracle
from paper_2508_19737_gb300 import metrics, synth
from tests.checks import kmeans_labels, row_errs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_19737_gb300 import api as a
    torch.cuda.set_device(0)
    return a


TAUS = [-100.0, -80.0, -60.0, -40.0, -20.0, -1.0, 0.0, 1.0, 20.0, 60.0, 100.0]


def test_tau_sign_decides_quality_as_in_fig4(api):
    import torch
    g = synth.challenge_like(100_000, seed=2)
    K = int(g.blocks.max()) + 1
    gr = api.graph_build(g.src, g.dst, g.N)
    L, d = 60, 32
    curve = {}
    for tau in TAUS:
        out = torch.empty((g.N, d), dtype=torch.float32, device="cuda")
        api.embed(gr, tau, L, d, 0, out=out)
        lab = kmeans_labels(out.cpu().numpy(), K)
        curve[tau] = (metrics.nmi(g.blocks, lab), metrics.pairwise_scores(g.blocks, lab)[2])
    gr.free()
    print("tau -> (NMI, F1):", {t: (round(a, 3), round(b, 3)) for t, (a, b) in curve.items()})
    best_neg = max(curve[t][1] for t in TAUS if t < 0)
    best_nonneg = max(curve[t][1] for t in TAUS if t >= 0)
    assert best_neg >= 0.9 and best_neg >= best_nonneg + 0.2, (best_neg, best_nonneg)
    assert max(curve, key=lambda t: curve[t][1]) < 0


def _ffp_job(a):
    rp, col, X, tau, L, storage = a
    return oracle.ffp(rp, col, X, tau, L, storage=storage)


TABLE2 = [(5_000, -6.0, 10, 64), (10_000, -3.0, 9, 64), (50_000, -80.0, 40, 32), (100_000, -80.0, 60, 32),
          (200_000, -100.0, 20, 16)]


@pytest.mark.parametrize("N,tau,L,d", TABLE2)
def test_table2_settings_error_budget(api, N, tau, L, d):
    """Table II's (tau, L, d) on graphs shaped like the paper's benchmark graphs of N nodes (the
    1M-node streaming setting tau = -100, L = 20, d = 16 on 200,000 nodes), host-drawn input, fp32
    and bf16 storage, against the FP64 oracle.

    Moderate |tau| (Table II's 5K and 10K rows): fp32 within 1e-4 on every row; bf16 within 5e-3
    of the bf16 storage model on every row. Large |tau| (-80, -100): Eq. 1 clamps D_tau to eps
    for every node of degree up to |tau| (almost all of them), the layer gains reach 1 / eps, tanh
    saturates and rows near its switching point amplify any rounding; there fp32 stays within 1e-4
    on at least 99.5 % of rows, and every row beyond that is one the FP64 oracle itself moves by
    more than 1e-6 when its input is perturbed by 2^-20 relative (the row is ill-conditioned, not
    mis-computed); bf16 stays within 5e-3 of its storage model on at least 97 % of rows (its storage
    error alone exceeds 2e-2 on many rows: bf16 is outside its error budget at such tau)."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import torch
    g = synth.challenge_like(N, seed=1)
    gr = api.graph_build(g.src, g.dst, g.N)
    rp, col = oracle.build_csr(g.src, g.dst, g.N)
    X = torch.from_numpy(synth.gaussian_input(0, N, d))
    X32, Xb = X.to(torch.float32), X.to(torch.bfloat16)
    x32, xb = X32.double().numpy(), Xb.double().numpy()
    sign = np.random.default_rng(5).choice([-1.0, 1.0], size=x32.shape)
    jobs = {"ref": (x32, "f64"), "pert": (x32 * (1 + sign * 2.0 ** -20), "f64"), "refb": (xb, "f64"),
            "emu": (xb, "bf16")}
    with cf.ProcessPoolExecutor(max_workers=4, mp_context=mp.get_context("spawn")) as ex:
        fut = {k: ex.submit(_ffp_job, (rp, col, v[0], tau, L, v[1])) for k, v in jobs.items()}
        res = {k: f.result() for k, f in fut.items()}
    out = {}
    for storage, xin in (("f32", X32), ("bf16", Xb)):
        o = torch.empty((N, d), dtype=torch.float32, device="cuda")
        api.embed(gr, tau, L, d, 0, out=o, storage=storage, x_in=xin.cuda())
        out[storage] = o.cpu().numpy()
    gr.free()
    e32 = row_errs(out["f32"], res["ref"])
    sens = row_errs(res["pert"], res["ref"])
    eb = row_errs(out["bf16"], res["emu"])
    store = row_errs(res["emu"], res["refb"])
    bad = e32 > 1e-4
    print(f"N={N} tau={tau} L={L} d={d}: fp32 rows beyond 1e-4: {int(bad.sum())} (max {e32.max():.2e}); "
          f"bf16 rows beyond 5e-3 of the model: {int((eb > 5e-3).sum())}; rows where bf16 storage alone "
          f"exceeds 2e-2: {int((store > 2e-2).sum())}")
    if abs(tau) <= 6:
        assert e32.max() <= 1e-4
        assert eb.max() <= 5e-3
    else:
        assert bad.mean() <= 0.005
        assert np.all(sens[bad] > 1e-6), float(sens[bad].min())
        assert (eb <= 5e-3).mean() >= 0.97
