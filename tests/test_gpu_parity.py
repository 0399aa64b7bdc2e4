"""CUDA path (through the C-ABI) against the FP64 oracle on the same seeded inputs.

Bars: CSR, degrees and the fp32 degree factors bit-exact; Theta within a few
fp32 ulps; embeddings within 1e-4 max per-row relative L2 error for fp32
storage and 2e-2 for bf16 storage (max over rows of ||z_gpu - z_ref|| / ||z_ref||).
"""
import math

import numpy as np
import pytest

import oracle
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


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def row_rel_err(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)))


def _random_multigraph(seed, N, M, loops=True):
    rng = np.random.default_rng(seed)
    src = rng.integers(0, N, M).astype(np.int32)
    dst = rng.integers(0, N, M).astype(np.int32)
    if loops and M:
        k = rng.integers(0, M, max(1, M // 50))
        dst[k] = src[k]
    rep = rng.integers(0, M, M // 10) if M else np.zeros(0, dtype=np.int64)
    return np.concatenate([src, dst[rep]]), np.concatenate([dst, src[rep]])  # some reversed repeats


# ---------------------------------------------------------------------------- CSR + Eq. 1
CSR_CASES = {
    "dcsbm-1k": lambda: (lambda g: (g.src, g.dst, g.N))(synth.dcsbm(1000, 11, 20, 2.5, 10, seed=0)),
    "multigraph": lambda: (*_random_multigraph(1, 5003, 40000), 5003),
    "single-node": lambda: (np.zeros(3, np.int32), np.zeros(3, np.int32), 1),
    "no-edges": lambda: (np.zeros(0, np.int32), np.zeros(0, np.int32), 77),
    "hub-rows": lambda: (  # rows longer than a warp's sort capacity and than shared memory
        np.concatenate([np.zeros(60000, np.int32), np.full(3000, 7, np.int32), np.arange(1, 5000, dtype=np.int32)]),
        np.concatenate([np.random.default_rng(2).integers(1, 70000, 60000).astype(np.int32),
                        np.random.default_rng(3).integers(0, 70000, 3000).astype(np.int32),
                        np.arange(2, 5001, dtype=np.int32)]), 70000),
    # 2^22 nodes: the partitioned build packs (local row, column) into all 32 bits
    "wide-ids": lambda: (*_random_multigraph(4, 1 << 22, 30000), 1 << 22),
    # more than 2^24 nodes: the atomic build
    "huge-N": lambda: (*_random_multigraph(5, (1 << 24) + 5, 30000), (1 << 24) + 5),
}


@pytest.mark.parametrize("case", sorted(CSR_CASES))
@pytest.mark.parametrize("where", ["host", "device"])
def test_csr_bit_exact(api, case, where):
    src, dst, N = CSR_CASES[case]()
    rp_ref, col_ref = oracle.build_csr(src, dst, N)
    s, d = (src, dst) if where == "host" else (_dev(src), _dev(dst))
    g = api.graph_build(s, d, N)
    n, nnz, maxdeg = g.info()
    rp, col = g.export()
    assert n == N and nnz == col_ref.size
    assert np.array_equal(rp, rp_ref) and np.array_equal(col, col_ref)
    assert maxdeg == (int(np.diff(rp_ref).max()) if N else 0)
    g.free()


def test_csr_rejects_out_of_range_ids(api):
    with pytest.raises(api.IgpError) as e:
        api.graph_build(np.array([0, 1, 2], np.int32), np.array([1, 9, 0], np.int32), 5)
    assert e.value.status == api.IGP_E_INVAL and "edge 1" in str(e.value)
    with pytest.raises(api.IgpError):
        api.graph_build(np.array([-1], np.int32), np.array([0], np.int32), 5)


@pytest.mark.parametrize("tau", [-0.5, -1.5, -6.0, -80.0, 0.0, 3.0])
def test_degree_factors_bit_exact(api, tau):
    src, dst, N = CSR_CASES["multigraph"]()
    src = np.concatenate([src, np.array([N - 1], np.int32)])  # plus an isolated node below
    dst = np.concatenate([dst, np.array([N - 1], np.int32)])
    g = api.graph_build(src, dst, N + 1)
    rp, _ = oracle.build_csr(src, dst, N + 1)
    ref = oracle.inv_sqrt_degrees(oracle.degree_correction(oracle.degrees(rp), tau)).astype(np.float32)
    got = api.degree_factors(g, tau)
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))
    g.free()


# ---------------------------------------------------------------------------- Theta
@pytest.mark.parametrize("N,d,seed", [(1000, 32, 0), (4099, 64, 12345), (17, 8, 2**63 + 5), (300, 128, 7)])
def test_theta_matches_oracle(api, N, d, seed):
    got = api.generate_x(seed, N, d).astype(np.float64)
    ref = oracle.theta_input(seed, N, d)
    xs = 1.0 / math.sqrt(d)
    np.testing.assert_allclose(got, ref, rtol=2e-6, atol=1e-6 * xs)
    # device output equals host output bit for bit
    import torch
    dev = torch.empty((N, d), dtype=torch.float32, device="cuda")
    api.generate_x(seed, N, d, out=dev)
    assert np.array_equal(dev.cpu().numpy(), got.astype(np.float32))


# ---------------------------------------------------------------------------- FFP
def _ffp_case(api, src, dst, N, d, tau, L, storage="f32", seed=0, device_out=True, **kw):
    import torch
    g = api.graph_build(_dev(src), _dev(dst), N)
    if device_out:
        out = torch.empty((N, d), dtype=torch.float32, device="cuda")
        api.embed(g, tau, L, d, seed, out=out, storage=storage, **kw)
        got = out.cpu().numpy()
    else:
        got = api.embed(g, tau, L, d, seed, storage=storage, **kw)
    g.free()
    rp, col = oracle.build_csr(src, dst, N)
    okw = {k: v for k, v in kw.items() if k in ("alpha", "theta", "eps", "out_row_l2")}
    if "znorm_ddof" in kw:
        okw["ddof"] = kw["znorm_ddof"]
    X = oracle.theta_input(seed, N, d, x_scale=kw.get("x_scale") or None)
    ref = oracle.ffp(rp, col, X, tau, L, **okw)
    return got, ref, (rp, col, X, okw)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_small_config_parity(api, storage):
    g = synth.dcsbm(1000, 11, 20, 2.5, 10, seed=0)
    got, ref, _ = _ffp_case(api, g.src, g.dst, g.N, 32, -0.5, 10, storage=storage)
    assert row_rel_err(got, ref) <= TOL[storage]


@pytest.mark.parametrize("d", [8, 16, 32, 64, 128])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_every_width_parity(api, d, storage):
    # ragged sizes: N not a multiple of any tile, rows from degree 0 to a few hundred
    g = synth.dcsbm(4099, 13, 18, 2.5, 5, seed=d)
    got, ref, _ = _ffp_case(api, g.src, g.dst, g.N, d, -0.5, 6, storage=storage, seed=d + 1)
    assert row_rel_err(got, ref) <= TOL[storage]


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_chunked_layers_equal_unchunked(api, storage):
    import torch
    g = synth.dcsbm(20000, 16, 20, 2.5, 5, seed=11)
    gr = api.graph_build(g.src, g.dst, g.N)
    outs = []
    for cc in (0, 32, 16, 8):
        o = torch.empty((g.N, 64), dtype=torch.float32, device="cuda")
        api.embed(gr, -0.5, 8, 64, 5, out=o, storage=storage, chunk_cols=cc)
        outs.append(o.cpu().numpy())
    gr.free()
    # column passes change only the fp32 summation order of the heavy rows (the whole-warp
    # gather depends on the lanes per row); the statistics are exact integer sums
    for o in outs[1:]:
        assert row_rel_err(o, outs[0]) <= {"f32": 1e-5, "bf16": 2e-2}[storage]
    with pytest.raises(api.IgpError):
        api.embed(api.graph_build(g.src, g.dst, g.N), -0.5, 2, 64, 0, chunk_cols=24)


@pytest.mark.parametrize("opts", [
    dict(chunk_cols=16),                  # four column passes per layer
    dict(chunk_cols=8),                   # one 32-byte slice per row, four passes
    dict(znorm_ddof=0),
    dict(out_row_l2=True),
    dict(alpha=-0.5, theta=0.7),          # high-pass filter (Eq. 2, alpha < 0)
    dict(x_scale=1.0),                    # Theta ~ N(0, 1)
    dict(eps=1e-2),
])
def test_option_parity(api, opts):
    g = synth.dcsbm(3001, 9, 16, 2.5, 6, seed=4)
    got, ref, _ = _ffp_case(api, g.src, g.dst, g.N, 32, -1.0, 5, **opts)
    assert row_rel_err(got, ref) <= TOL["f32"]


@pytest.mark.parametrize("tau,L", [(0.0, 4), (3.0, 4), (-6.0, 10), (-80.0, 5), (-0.5, 0), (-0.5, 1)])
def test_tau_and_depth_parity(api, tau, L):
    g = synth.dcsbm(2500, 7, 30, 2.5, 6, seed=5)
    got, ref, _ = _ffp_case(api, g.src, g.dst, g.N, 32, tau, L)
    assert row_rel_err(got, ref) <= TOL["f32"]


def test_degenerate_graphs(api):
    # edgeless graph (Ahat = 0), a single node (std of one value -> column 0), isolated nodes
    got, ref, _ = _ffp_case(api, np.zeros(0, np.int32), np.zeros(0, np.int32), 50, 16, -0.5, 3)
    assert row_rel_err(got, ref) <= TOL["f32"]
    got, ref, _ = _ffp_case(api, np.zeros(0, np.int32), np.zeros(0, np.int32), 1, 16, -0.5, 3)
    assert np.array_equal(got, np.full((1, 16), 0.5, np.float32)) and np.allclose(ref, 0.5)
    src = np.array([0, 1, 5], np.int32)
    dst = np.array([1, 2, 6], np.int32)
    got, ref, _ = _ffp_case(api, src, dst, 40, 8, -1.5, 4)
    assert row_rel_err(got, ref) <= TOL["f32"]


def test_host_output_and_x_in(api):
    import torch
    g = synth.dcsbm(2000, 5, 12, 2.5, 5, seed=6)
    got, ref, (rp, col, X, _) = _ffp_case(api, g.src, g.dst, g.N, 32, -0.5, 5, device_out=False)
    assert row_rel_err(got, ref) <= TOL["f32"]
    # a caller-supplied Z^(0)
    Xc = np.random.default_rng(0).standard_normal((g.N, 32)).astype(np.float32)
    gr = api.graph_build(g.src, g.dst, g.N)
    out = api.embed(gr, -0.5, 5, 32, 0, x_in=torch.from_numpy(Xc).cuda())
    gr.free()
    assert row_rel_err(out, oracle.ffp(rp, col, Xc.astype(np.float64), -0.5, 5)) <= TOL["f32"]


def test_pinned_host_output_equals_device_output(api):
    """A page-locked host output is written by the output kernel directly; the result is the
    device-output result, bit for bit (pageable outputs are staged through the device)."""
    import torch
    g = synth.dcsbm(30011, 20, 24, 2.4, 5, seed=12)
    gr = api.graph_build(g.src, g.dst, g.N)
    for storage in ("f32", "bf16"):
        dev = torch.empty((g.N, 64), dtype=torch.float32, device="cuda")
        api.embed(gr, -0.5, 6, 64, 4, out=dev, storage=storage)
        pinned = torch.full((g.N, 64), -1.0, dtype=torch.float32).pin_memory()
        api.embed(gr, -0.5, 6, 64, 4, out=pinned, storage=storage)
        pageable = np.full((g.N, 64), -1.0, dtype=np.float32)
        api.embed(gr, -0.5, 6, 64, 4, out=pageable, storage=storage)
        d = dev.cpu().numpy()
        assert np.array_equal(pinned.numpy(), d) and np.array_equal(pageable, d)
    gr.free()


def test_host_async_output_equals_synchronous_output(api):
    """opts.host_async: the call returns once the work is enqueued and a page-locked output is
    filled in stream order (through a device temporary and a copy engine); after
    igp_graph_sync it holds the synchronous result bit for bit. Two graphs on two streams are in
    flight at once, as in a pipelined caller; a pageable output ignores the option."""
    import torch
    gs = [synth.dcsbm(30011, 20, 24, 2.4, 5, seed=12), synth.dcsbm(20011, 16, 20, 2.5, 5, seed=13)]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for storage in ("f32", "bf16"):
        refs, grs, outs = [], [], []
        for g in gs:
            gr = api.graph_build(g.src, g.dst, g.N)
            ref = torch.empty((g.N, 64), dtype=torch.float32, device="cuda")
            api.embed(gr, -0.5, 6, 64, 4, out=ref, storage=storage)
            refs.append(ref.cpu().numpy())
            grs.append(gr)
        torch.cuda.synchronize()
        for k, (g, gr) in enumerate(zip(gs, grs)):
            out = torch.full((g.N, 64), -1.0, dtype=torch.float32).pin_memory()
            api.embed(gr, -0.5, 6, 64, 4, out=out, storage=storage, host_async=True, stream=streams[k])
            outs.append(out)
        for gr, out, ref in zip(grs, outs, refs):
            gr.sync()
            assert np.array_equal(out.numpy(), ref)
        pageable = np.full((gs[0].N, 64), -1.0, dtype=np.float32)
        api.embed(grs[0], -0.5, 6, 64, 4, out=pageable, storage=storage, host_async=True)
        assert np.array_equal(pageable, refs[0])
        for gr in grs:
            gr.free()


def test_bf16_against_bf16_emulating_oracle(api):
    g = synth.dcsbm(20011, 32, 25, 2.5, 4, seed=7, dirichlet_alpha=2.0)
    got, ref, (rp, col, X, _) = _ffp_case(api, g.src, g.dst, g.N, 64, -0.5, 10, storage="bf16")
    e64 = row_rel_err(got, ref)
    emu = oracle.ffp(rp, col, X, -0.5, 10, storage="bf16")
    e_emu = row_rel_err(got, emu)
    assert e64 <= TOL["bf16"]
    assert e_emu <= e64  # the storage-rounding model explains most of the difference


def test_deterministic_and_stream_ordered(api):
    import torch
    g = synth.dcsbm(30000, 20, 25, 2.5, 4, seed=8)
    gr = api.graph_build(_dev(g.src), _dev(g.dst), g.N)
    s = torch.cuda.Stream()
    outs = []
    for _ in range(2):
        o = torch.empty((g.N, 64), dtype=torch.float32, device="cuda")
        with torch.cuda.stream(s):
            api.embed(gr, -0.5, 10, 64, 3, out=o, storage="bf16", stream=s)
        s.synchronize()
        outs.append(o.cpu().numpy())
    gr.free()
    assert np.array_equal(outs[0], outs[1])


# The named workloads at full size and depth: tests/test_gpu_workloads.py


# ---------------------------------------------------------------------------- gather modes
@pytest.mark.parametrize("d,storage", [(64, "bf16"), (64, "f32"), (32, "bf16"), (128, "bf16"), (16, "f32")])
def test_gather_modes_agree(api, d, storage):
    """The two bulk-copy gathers add the same rows in the same order; the register-load gather
    agrees with them to fp32 rounding (it gathers the highest-degree rows with a whole warp)."""
    import torch
    g = synth.dcsbm(7001, 12, 22, 2.4, 5, seed=13)
    gr = api.graph_build(g.src, g.dst, g.N)
    outs = {}
    for mode in ("lsu", "bulk", "tma4"):
        o = torch.empty((g.N, d), dtype=torch.float32, device="cuda")
        api.embed(gr, -0.5, 6, d, 9, out=o, storage=storage, gather=mode)
        outs[mode] = o.cpu().numpy()
    gr.sync()
    gr.free()
    assert np.array_equal(outs["bulk"], outs["tma4"])
    assert row_rel_err(outs["lsu"], outs["bulk"]) <= {"f32": 1e-5, "bf16": 2e-2}[storage]
    rp, col = oracle.build_csr(g.src, g.dst, g.N)
    ref = oracle.ffp(rp, col, oracle.theta_input(9, g.N, d), -0.5, 6)
    assert row_rel_err(outs["lsu"], ref) <= TOL[storage]


def test_bounded_device_wait_reports_timeout(api):
    """A bulk-copy wait that cannot complete gives up after about a second: the host reads
    IGP_E_TIMEOUT and the context stays usable (no trap, no hang)."""
    import torch
    g = synth.dcsbm(3000, 6, 16, 2.5, 5, seed=17)
    gr = api.graph_build(g.src, g.dst, g.N)
    out = torch.empty((g.N, 64), dtype=torch.float32, device="cuda")
    api.embed(gr, -0.5, 2, 64, 1, out=out, storage="bf16", gather="bulk", reserved_test=1)
    with pytest.raises(api.IgpError) as e:
        gr.sync()
    assert e.value.status == api.IGP_E_TIMEOUT
    with pytest.raises(api.IgpError) as e:  # host output: reported by the call itself
        api.embed(gr, -0.5, 1, 64, 1, storage="bf16", gather="tma4", reserved_test=1)
    assert e.value.status == api.IGP_E_TIMEOUT
    # the same handle and context work normally afterwards
    api.embed(gr, -0.5, 3, 64, 2, out=out, storage="bf16", gather="tma4")
    gr.sync()
    rp, col = oracle.build_csr(g.src, g.dst, g.N)
    ref = oracle.ffp(rp, col, oracle.theta_input(2, g.N, 64), -0.5, 3)
    assert row_rel_err(out.cpu().numpy(), ref) <= TOL["bf16"]
    gr.free()


# ---------------------------------------------------------------------------- import
def test_import_restores_an_exported_graph(api):
    """igp_graph_export -> igp_graph_import (host and device arrays, validated or trusted) gives a
    graph whose CSR, degree factors and embeddings equal the original's bit for bit."""
    import torch
    g = synth.dcsbm(20011, 16, 22, 2.4, 5, seed=31)
    gr = api.graph_build(g.src, g.dst, g.N)
    rp, col = gr.export()
    ref = torch.empty((g.N, 32), dtype=torch.float32, device="cuda")
    api.embed(gr, -0.5, 6, 32, 3, out=ref, storage="bf16")
    for where, validate in (("host", True), ("device", True), ("device", False)):
        a, b = (rp, col) if where == "host" else (_dev(rp), _dev(col))
        h = api.graph_import(a, b, g.N, validate=validate)
        assert h.info() == gr.info()
        rp2, col2 = h.export()
        assert np.array_equal(rp2, rp) and np.array_equal(col2, col)
        out = torch.empty((g.N, 32), dtype=torch.float32, device="cuda")
        api.embed(h, -0.5, 6, 32, 3, out=out, storage="bf16")
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        h.free()
    gr.free()


def test_import_rejects_what_is_not_a_simple_undirected_csr(api):
    rp, col = oracle.build_csr([0, 0, 1, 2], [1, 2, 2, 3], 5)  # path-like graph + isolated node 4
    rp = rp.astype(np.int32)
    col = col.astype(np.int32)
    ok = api.graph_import(rp, col, 5)
    assert ok.info()[:2] == (5, 8)
    ok.free()
    cases = {
        "row_ptr": (np.array([1, 2, 4, 6, 8, 8], np.int32), col),
        "column out of range": (rp, np.where(np.arange(col.size) == 3, 9, col).astype(np.int32)),
        "row not sorted": (rp, col[[1, 0, 2, 3, 4, 5, 6, 7]]),
        "self-loop": (rp, np.where(np.arange(col.size) == 0, 0, col).astype(np.int32)),
        "not symmetric": (rp, np.where(np.arange(col.size) == 7, 1, col).astype(np.int32)),
    }
    for name, (a, b) in cases.items():
        with pytest.raises(api.IgpError) as e:
            api.graph_import(a, b, 5)
        assert e.value.status == api.IGP_E_INVAL and name.split()[0] in str(e.value), (name, str(e.value))
