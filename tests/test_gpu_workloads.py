"""The named single-graph workloads at full size and full depth, through the C-ABI, against the
FP64 oracle on the same input.

The input Theta is drawn on the host (synth.gaussian_input, N(0, 1/d)) and given to both sides:
to the GPU as igp_embed_opts.x_in in the storage type, to the oracle as the same values (the
fp32 or bf16 rounding of the host draw, widened to fp64). So the comparison measures the FFP
alone, not the device's own Theta generator (that one is checked against the oracle's generator
in test_gpu_parity.py).
"""
import numpy as np
import pytest

import oracle
from paper_2508_19737_gb300 import synth
from tests.checks import TOL, check_bf16, nmi_gap, row_errs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_19737_gb300 import api as a
    torch.cuda.set_device(0)
    return a


def _input(N, d, storage):
    """Host draw -> (device tensor in the storage type, the same values as fp64 for the oracle)."""
    import torch
    X = torch.from_numpy(synth.gaussian_input(0, N, d))
    Xs = X.to(torch.bfloat16 if storage == "bf16" else torch.float32)
    return Xs.cuda(), Xs.to(torch.float64).numpy()


def test_200k_config_both_storages_full_depth(api):
    """dcsbm-200k (N = 200,000, d = 64, tau = -0.5, L = 10): fp32 storage within 1e-4 of FP64 on
    every row; bf16 storage within 2e-2 of FP64 on every row and within 5e-3 of the bf16 storage
    model; for both, k-means NMI against the planted partition within 0.01 of FP64's."""
    import torch
    wl = synth.WORKLOADS["dcsbm-200k"]
    g = synth.workload_graph("dcsbm-200k")
    d, tau, L = wl["d"], wl["tau"], wl["L"]
    gr = api.graph_build(g.src, g.dst, g.N)
    rp, col = oracle.build_csr(g.src, g.dst, g.N)
    for storage in ("f32", "bf16"):
        xd, x64 = _input(g.N, d, storage)
        out = torch.empty((g.N, d), dtype=torch.float32, device="cuda")
        api.embed(gr, tau, L, d, 0, out=out, storage=storage, x_in=xd)
        got = out.cpu().numpy()
        if storage == "f32":
            ref = oracle.ffp(rp, col, x64, tau, L)
            err = row_errs(got, ref)
            gap, n_got, n_ref = nmi_gap(got, ref, g.blocks)
            print(f"fp32: max row error {err.max():.3e}, NMI {n_got:.4f} vs FP64 {n_ref:.4f}")
            assert err.max() <= TOL["f32"]
            assert gap <= 0.01
        else:
            check_bf16(got, rp, col, x64, tau, L, blocks=g.blocks, strict=True)
    gr.free()


def test_2m_config_full_size_full_depth(api):
    """dcsbm-2m in the configuration the benchmark times (N = 2,000,000, about 80M CSR entries,
    d = 64, bf16 storage, tau = -0.5, L = 10): bit-exact CSR and degree factors; the embedding
    compared with FP64 and with the bf16 storage model on every row; k-means NMI (128 planted
    blocks) on a fixed sample of 200,000 nodes within 0.01 of FP64's; logits with column mean 0
    and sample standard deviation 1."""
    import torch
    wl = synth.WORKLOADS["dcsbm-2m"]
    g = synth.workload_graph("dcsbm-2m")
    d, tau, L, storage = wl["d"], wl["tau"], wl["L"], wl["storage"]
    src = torch.from_numpy(g.src).cuda()
    dst = torch.from_numpy(g.dst).cuda()
    gr = api.graph_build(src, dst, g.N)
    del src, dst
    rp, col = oracle.build_csr(g.src, g.dst, g.N)
    rpg, colg = gr.export()
    assert np.array_equal(rpg, rp) and np.array_equal(colg, col)
    del rpg, colg
    ref_dinv = oracle.inv_sqrt_degrees(oracle.degree_correction(oracle.degrees(rp), tau)).astype(np.float32)
    assert np.array_equal(api.degree_factors(gr, tau).view(np.uint32), ref_dinv.view(np.uint32))
    xd, x64 = _input(g.N, d, storage)
    out = torch.empty((g.N, d), dtype=torch.float32, device="cuda")
    api.embed(gr, tau, L, d, 0, out=out, storage=storage, x_in=xd)
    got = out.cpu().numpy()
    del xd
    check_bf16(got, rp, col, x64, tau, L, blocks=g.blocks, strict=True, nmi_sample=200_000)
    z = out.double()
    z = torch.log(z) - torch.log1p(-z)
    assert torch.isfinite(z).all()
    assert float(z.mean(0).abs().max()) < 1e-2
    assert float((z.std(0) - 1).abs().max()) < 2e-2
    gr.free()
