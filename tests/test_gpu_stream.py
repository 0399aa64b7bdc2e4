"""Streaming (the merge and FFP of each step of Alg. 2): a device-resident graph grown by edge increments equals, after
every step, the graph built from scratch from all edges so far (CSR bit-exact against the FP64
oracle's cumulative snapshot), and its embedding equals the fresh build's bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2508_19737_gb300 import synth

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("mode", ["snowball", "random"])
def test_appended_graph_equals_static_rebuild(api, mode):
    g = synth.dcsbm(6000, 12, 20, 2.5, 5, seed=31)
    incs = synth.split_increments(g, T=10, mode=mode, seed=2)
    snaps = list(oracle.stream_snapshots(incs))
    s0, d0, n0 = incs[0]
    gr = api.graph_build(s0, d0, n0)
    acc_s, acc_d = [s0], [d0]
    for t, ((s, d, n), (rp_ref, col_ref, n_ref)) in enumerate(zip(incs, snaps)):
        if t > 0:
            gr.append(s, d, n)
            acc_s.append(s)
            acc_d.append(d)
        N, nnz, maxdeg = gr.info()
        rp, col = gr.export()
        assert N == n_ref and nnz == col_ref.size
        assert np.array_equal(rp, rp_ref) and np.array_equal(col, col_ref), t
        assert maxdeg == (int(np.diff(rp_ref).max()) if N else 0)
        if t in (0, 4, 9):
            fresh = api.graph_build(np.concatenate(acc_s), np.concatenate(acc_d), n)
            for storage in ("f32", "bf16"):
                a = api.embed(gr, -0.5, 5, 32, 7 + t, storage=storage)
                b = api.embed(fresh, -0.5, 5, 32, 7 + t, storage=storage)
                assert np.array_equal(a, b)
            fresh.free()
            ref = oracle.ffp(rp_ref, col_ref, oracle.theta_input(7 + t, n, 32), -0.5, 5)
            assert _rel(api.embed(gr, -0.5, 5, 32, 7 + t), ref) <= 1e-4
    gr.free()


def test_append_rejects_bad_input_and_keeps_graph(api):
    gr = api.graph_build(np.array([0, 1], np.int32), np.array([1, 2], np.int32), 4)
    before = gr.export()
    with pytest.raises(api.IgpError) as e:
        gr.append(np.array([0], np.int32), np.array([1], np.int32), 3)  # shrinking
    assert e.value.status == api.IGP_E_INVAL
    with pytest.raises(api.IgpError):
        gr.append(np.array([0], np.int32), np.array([9], np.int32), 6)  # id outside [0, 6)
    after = gr.export()
    assert all(np.array_equal(x, y) for x, y in zip(before, after)) and gr.info()[0] == 4
    gr.append(np.zeros(0, np.int32), np.zeros(0, np.int32), 7)  # new isolated nodes only
    rp, col = gr.export()
    assert rp.size == 8 and np.array_equal(col, before[1])
    gr.free()


def test_new_node_rows_extracted_on_the_device(api):
    """Alg. 2 extracts the new nodes' rows: with out_row_begin = N_(t-1) igp_embed writes only the new nodes' rows, bit for bit
    the rows N_(t-1).. of the whole embedding, into device, page-locked and pageable outputs."""
    import torch
    g = synth.dcsbm(9000, 10, 18, 2.5, 5, seed=51)
    incs = synth.split_increments(g, T=4, mode="snowball", seed=5)
    gr = api.graph_build(*incs[0])
    for s, d, n in incs[1:]:
        n_old = gr.N
        gr.append(s, d, n)
        for storage in ("f32", "bf16"):
            full = api.embed(gr, -0.5, 6, 64, 3, storage=storage)
            for r0 in (0, n_old, n - 1, n):
                pageable = api.embed(gr, -0.5, 6, 64, 3, storage=storage, out_row_begin=r0)
                assert pageable.shape == (n - r0, 64)
                if r0 == n:  # no rows: a NULL output is allowed too
                    o = api.embed_opts(storage=storage, out_row_begin=r0)
                    assert api.lib().igp_embed(gr.handle, -0.5, 6, 64, 3, None, api.ctypes.byref(o), None) == 0
                    continue
                dev = torch.full((n - r0, 64), -1.0, dtype=torch.float32, device="cuda")
                api.embed(gr, -0.5, 6, 64, 3, out=dev, storage=storage, out_row_begin=r0)
                pinned = torch.full((n - r0, 64), -1.0, dtype=torch.float32).pin_memory()
                api.embed(gr, -0.5, 6, 64, 3, out=pinned, storage=storage, out_row_begin=r0)
                for got in (dev.cpu().numpy(), pinned.numpy(), pageable):
                    assert np.array_equal(got, full[r0:]), (storage, r0)
    for r0 in (-1, gr.N + 1):
        with pytest.raises(api.IgpError) as e:
            api.embed(gr, -0.5, 6, 64, 3, out=np.empty((4, 64), np.float32), out_row_begin=r0)
        assert e.value.status == api.IGP_E_INVAL
    gr.free()


def test_new_node_rows_through_the_server_and_noalloc(api):
    import torch
    g = synth.dcsbm(7000, 8, 16, 2.5, 5, seed=52)
    incs = synth.split_increments(g, T=3, mode="snowball", seed=6)
    sv = api.Server(slots=2)
    t0 = sv.submit(*incs[0], -0.5, 5, 32, 1, kind="embed", graph_id=5, keep=True, storage="bf16")
    (s1, d1, n1), n0 = incs[1], incs[0][2]
    t1 = sv.submit(s1, d1, n1, -0.5, 5, 32, 2, kind="append", graph_id=5, storage="bf16", out_row_begin=n0)
    for t in (t0, t1):
        assert sv.wait(t)[0] == "done"
    ref = api.graph_build(np.concatenate([incs[0][0], s1]), np.concatenate([incs[0][1], d1]), n1)
    full = api.embed(ref, -0.5, 5, 32, 2, storage="bf16")
    assert sv.result(t1).shape == (n1 - n0, 32) and np.array_equal(sv.result(t1), full[n0:])
    sv.close()
    N, nnz, _ = ref.info()
    rp = torch.empty(N + 1, dtype=torch.int32, device="cuda")
    col = torch.empty(nnz, dtype=torch.int32, device="cuda")
    ref.export(rp, col)
    whole = torch.empty((N, 32), dtype=torch.float32, device="cuda")
    api.embed_noalloc(rp, col, N, -0.5, 5, 32, 2, whole)
    tail = torch.full((N - n0, 32), -1.0, dtype=torch.float32, device="cuda")
    api.embed_noalloc(rp, col, N, -0.5, 5, 32, 2, tail, out_row_begin=n0)
    torch.cuda.synchronize()
    assert torch.equal(tail, whole[n0:])
    ref.free()


class _Leader:
    """Threshold leader clustering: a row joins the nearest centre within `radius`, else starts one;
    predict gives the nearest centre. Deterministic in its input rows."""

    def __init__(self, radius):
        self.radius, self.C = radius, None

    def partial_fit(self, X):
        for x in X:
            if self.C is None or np.min(np.linalg.norm(self.C - x, axis=1)) > self.radius:
                self.C = x[None].copy() if self.C is None else np.vstack([self.C, x])
        return self

    def predict(self, X):
        out = np.empty(X.shape[0], dtype=np.int64)
        c2 = (self.C.astype(np.float64) ** 2).sum(1)
        for a in range(0, X.shape[0], 4096):
            x = X[a:a + 4096].astype(np.float64)
            out[a:a + 4096] = np.argmin(c2[None] - 2 * x @ self.C.T.astype(np.float64), axis=1)
        return out


def test_streaming_partitioner_equals_fresh_runs_step_by_step(api):
    """Alg. 2 end to end: the pipeline (append, FFP, new rows only, clustering on a host thread)
    gives at every step the partition of a step-by-step run on freshly built snapshots whose whole
    embedding is sliced on the host."""
    from paper_2508_19737_gb300 import stream
    g = synth.dcsbm(12000, 12, 20, 2.5, 5, seed=61)
    incs = synth.split_increments(g, T=5, mode="snowball", seed=7)
    with stream.StreamingPartitioner(_Leader(1.2), tau=-0.5, L=6, d=32, seed=9, storage="bf16") as sp:
        labs = [sp.labels(sp.step(*inc), timeout=300) for inc in incs]
        assert [sp.timings[t]["new_rows"] for t in range(len(incs))] == \
            [incs[0][2]] + [incs[t][2] - incs[t - 1][2] for t in range(1, len(incs))]
    ref = _Leader(1.2)
    acc_s, acc_d, kept, n_prev = [], [], [], 0
    for t, (s, d, n) in enumerate(incs):
        acc_s.append(s)
        acc_d.append(d)
        fresh = api.graph_build(np.concatenate(acc_s), np.concatenate(acc_d), n)
        Z = api.embed(fresh, -0.5, 6, 32, 9, storage="bf16")
        fresh.free()
        ref.partial_fit(Z[n_prev:])
        kept.append(Z[n_prev:])
        assert np.array_equal(labs[t], ref.predict(np.concatenate(kept))), t
        n_prev = n
    lab, gpu_s, host_s = stream.static_partition(np.concatenate(acc_s), np.concatenate(acc_d), n_prev, _Leader(1.2),
                                                 tau=-0.5, L=6, d=32, seed=9, storage="bf16")
    assert lab.shape == (n_prev,) and gpu_s > 0 and host_s > 0
