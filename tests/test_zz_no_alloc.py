"""igp_embed_noalloc: the FFP for callers that may not allocate device memory during
the call (stream capture, allocator hooks, fixed-footprint loops).

Checked through the C-ABI against igp_embed on the same graph, on two calls in a row
(the second reuses the library's fixed scratch array after the first left its
contents there), plus the size limit. This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2508_19737_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"f32": 1e-4, "bf16": 2e-2}


@pytest.fixture(scope="module")
def api():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_19737_gb300 import api as a
    torch.cuda.set_device(0)
    return a


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_noalloc_matches_embed_on_two_calls(api, storage):
    import torch
    g = synth.dcsbm(6007, 9, 18, 2.5, 5, seed=21)
    gr = api.graph_build(g.src, g.dst, g.N)
    N, nnz, _ = gr.info()
    rp = torch.empty(N + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(nnz, dtype=torch.int32, device="cuda")
    gr.export(rp, col)
    d, tau, L = 32, -0.5, 10
    for seed in (3, 4):  # two calls in a row through the shared scratch array
        ref = torch.empty((N, d), dtype=torch.float32, device="cuda")
        api.embed(gr, tau, L, d, seed, out=ref, storage=storage)
        got = torch.full((N, d), -1.0, dtype=torch.float32, device="cuda")
        api.embed_noalloc(rp, col, N, tau, L, d, seed, got, storage=storage)
        torch.cuda.synchronize()
        assert _rel(got.cpu().numpy(), ref.cpu().numpy()) <= TOL[storage]
    gr.free()


def test_noalloc_rejects_sizes_beyond_its_scratch(api):
    import torch
    N, d = 200_000, 64  # 2 x 200,000 x 64 x 4 bytes of activations alone exceed 16 MiB
    rp = torch.zeros(N + 1, dtype=torch.int32, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.empty((N, d), dtype=torch.float32, device="cuda")
    with pytest.raises(api.IgpError) as e:
        api.embed_noalloc(rp, col, N, -0.5, 2, d, 0, out)
    assert e.value.status == api.IGP_E_INVAL and "16 MiB" in str(e.value)
