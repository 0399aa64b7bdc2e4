"""Streaming (Alg. 2, lines 1-7): a device-resident graph grown by edge increments equals, after
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
