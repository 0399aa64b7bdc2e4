"""igp_embed_noalloc: the FFP for callers that cannot allocate device memory during the
call (an allocator hook that must not re-enter its allocator, a framework whose caching
allocator already holds the free memory, a loop with a fixed memory footprint).

Checked through the C-ABI against igp_embed on the same graph, on two calls in a row
(the second reuses the library's fixed scratch array after the first left its
contents there); against the FP64 oracle at the largest size the array holds, on a
graph with hub rows; that repeated calls allocate nothing (the library's allocation
count and the device's free memory stay put); and the size limit. This file is
collected last on purpose.
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


def _hub_graph(N, seed):
    """A DC-SBM with a few hubs of 2,000-6,000 neighbours added (long rows)."""
    g = synth.dcsbm(N, 16, 30, 2.2, 5, seed=seed)
    rng = np.random.default_rng(seed)
    src, dst = [g.src], [g.dst]
    for h, k in ((0, 6000), (1, 3000), (N // 2, 2000)):
        nb = rng.choice(N, size=k, replace=False).astype(np.int32)
        src.append(np.full(k, h, np.int32))
        dst.append(nb)
    return np.concatenate(src), np.concatenate(dst), g


@pytest.mark.parametrize("storage,d", [("f32", 32), ("bf16", 64)])
def test_noalloc_matches_oracle_at_its_largest_size(api, storage, d):
    """60,000 nodes: 2 x 60,000 x 128-byte activations + 8 N + statistics fit the 16 MiB array
    (about 264 N bytes); the hubs give rows of thousands of entries."""
    import torch
    import oracle
    from tests.test_gpu_batch import check_bf16_against_oracles
    N = 60_000
    src, dst, g = _hub_graph(N, 31)
    gr = api.graph_build(src, dst, N)
    _, nnz, max_deg = gr.info()
    assert max_deg >= 6000
    rp = torch.empty(N + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(nnz, dtype=torch.int32, device="cuda")
    gr.export(rp, col)
    tau, L, seed = -0.5, 10, 9
    got = torch.full((N, d), -1.0, dtype=torch.float32, device="cuda")
    api.embed_noalloc(rp, col, N, tau, L, d, seed, got, storage=storage)
    torch.cuda.synchronize()
    got = got.cpu().numpy()
    if storage == "f32":
        orp, ocol = oracle.build_csr(src, dst, N)
        ref = oracle.ffp(orp, ocol, oracle.theta_input(seed, N, d), tau, L)
        assert _rel(got, ref) <= TOL["f32"]
    else:
        h = synth.DCSBM(src, dst, N, g.blocks, g.theta, g.seed, g.params)
        check_bf16_against_oracles(got, h, seed, d, tau, L)
    gr.free()


def test_noalloc_allocates_nothing_and_honours_out_row_begin(api):
    """After a first call (which looks up the array's address and loads the kernels), further
    calls leave the library's allocation count and the device's free memory unchanged. With
    out_row_begin = r the call writes rows r .. N-1 into an (N - r) x d output."""
    import torch
    g = synth.dcsbm(20_000, 12, 24, 2.5, 5, seed=5)
    gr = api.graph_build(g.src, g.dst, g.N)
    N, nnz, _ = gr.info()
    rp = torch.empty(N + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(nnz, dtype=torch.int32, device="cuda")
    gr.export(rp, col)
    d, r0 = 64, 12_345
    full = torch.empty((N, d), dtype=torch.float32, device="cuda")
    part = torch.full((N - r0, d), -1.0, dtype=torch.float32, device="cuda")
    api.embed_noalloc(rp, col, N, -0.5, 10, d, 1, full, storage="bf16")
    api.embed_noalloc(rp, col, N, -0.5, 10, d, 1, part, storage="bf16", out_row_begin=r0)
    torch.cuda.synchronize()
    a0 = api.alloc_count()
    free0, _ = torch.cuda.mem_get_info()
    for seed in (2, 3, 1):
        api.embed_noalloc(rp, col, N, -0.5, 10, d, seed, full, storage="bf16")
        api.embed_noalloc(rp, col, N, -0.5, 10, d, seed, part, storage="bf16", out_row_begin=r0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert api.alloc_count() == a0
    assert free1 == free0, (free0, free1)
    # the last pair of calls used seed 1 for both: the partial output is the tail of the full one
    assert torch.equal(part, full[r0:])
    gr.free()
