"""Serving loop: concurrent, memory-admitted requests give exactly the results the same requests
give alone (to fp32 rounding when small requests are embedded in shared batches: igp_embed alone
gathers the highest-degree rows with a whole warp, in another summation order); resident graphs
are grown by increments in submission order."""
import numpy as np
import pytest

from paper_2508_19737_gb300 import synth

pytestmark = pytest.mark.gpu

AGREE = {"f32": 1e-5, "bf16": 2e-2}


def _rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(b, axis=1)))


@pytest.fixture(scope="module")
def api():
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2508_19737_gb300 import api as a
    torch.cuda.set_device(0)
    return a


def _requests():
    reqs = []
    for k in range(12):
        g = synth.dcsbm(2000 + 1500 * k, 5 + k, 12 + k, 2.5, 5, seed=100 + k)
        reqs.append(dict(src=g.src, dst=g.dst, N=g.N, tau=-0.5 - 0.1 * k, L=4 + k % 5, d=(32, 64, 16)[k % 3],
                         seed=k, storage=("f32", "bf16")[k % 2]))
    return reqs


def test_results_same_alone_and_in_the_mix(api):
    reqs = _requests()
    alone = []
    sv1 = api.Server(slots=1)
    for r in reqs:  # one at a time
        t = sv1.submit(**r)
        assert sv1.wait(t)[0] == "done"
        alone.append(sv1.result(t).copy())
    sv1.close()
    sv = api.Server(slots=4)
    tickets = [sv.submit(**r) for r in reqs]  # all at once: they overlap on the GPU
    for t in tickets:
        assert sv.wait(t)[0] == "done"
    for k, t in enumerate(tickets):
        assert np.array_equal(sv.result(t), alone[k]), k
    # and both equal the direct library call
    r = reqs[5]
    g = api.graph_build(r["src"], r["dst"], r["N"])
    direct = api.embed(g, r["tau"], r["L"], r["d"], r["seed"], storage=r["storage"])
    g.free()
    assert np.array_equal(direct, alone[5])
    st = sv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["latency_p99_s"] >= st["latency_p50_s"] > 0
    sv.close()


def test_streaming_requests_on_a_resident_graph(api):
    g = synth.dcsbm(8000, 10, 18, 2.5, 5, seed=41)
    incs = synth.split_increments(g, T=6, mode="snowball", seed=3)
    sv = api.Server(slots=3)
    tickets = []
    for t, (s, d, n) in enumerate(incs):
        tickets.append(sv.submit(s, d, n, -0.5, 5, 32, 9 + t, kind="embed" if t == 0 else "append",
                                 graph_id=77, keep=(t == 0), storage="bf16"))
    # a second, independent request in the middle
    h = synth.dcsbm(3000, 4, 10, 2.5, 5, seed=42)
    other = sv.submit(h.src, h.dst, h.N, -0.5, 5, 32, 1)
    for t in tickets + [other]:
        assert sv.wait(t)[0] == "done"
    ref = api.graph_build(*incs[0])
    for t, (s, d, n) in enumerate(incs):
        if t:
            ref.append(s, d, n)
        assert np.array_equal(sv.result(tickets[t]), api.embed(ref, -0.5, 5, 32, 9 + t, storage="bf16")), t
    ref.free()
    assert sv.stats()["resident_graphs"] == 1
    sv.release(77)
    assert sv.stats()["resident_graphs"] == 0
    sv.close()


def test_cancel_and_failures(api):
    g = synth.dcsbm(20000, 8, 20, 2.5, 5, seed=43)
    sv = api.Server(slots=1)
    ts = [sv.submit(g.src, g.dst, g.N, -0.5, 10, 64, k) for k in range(12)]
    sv.cancel(ts[-1])
    assert sv.poll(ts[-1])[0] == "cancelled"
    bad = sv.submit(g.src, g.dst, g.N, -0.5, 3, 32, 0, kind="append", graph_id=12345)
    with pytest.raises(api.IgpError) as e:
        sv.wait(bad)
    assert e.value.status == api.IGP_E_INVAL
    for t in ts[:-1]:
        assert sv.wait(t)[0] == "done"
    oob = sv.submit(g.src, np.full(g.M, 10 ** 9, np.int32), g.N, -0.5, 3, 32, 0)  # fails in the CSR build
    with pytest.raises(api.IgpError) as e:
        sv.wait(oob)
    assert e.value.status == api.IGP_E_INVAL
    with pytest.raises(api.IgpError) as e:  # larger than any device
        sv.submit(g.src, g.dst, 2 ** 31 - 1, -0.5, 3, 128, 0, out=np.empty((1, 128), np.float32))
    assert e.value.status == api.IGP_E_NOMEM
    with pytest.raises(api.IgpError) as e:  # a served result is final when its request completes
        sv.submit(g.src, g.dst, g.N, -0.5, 3, 32, 0, host_async=True)
    assert e.value.status == api.IGP_E_INVAL
    ok = sv.submit(g.src, g.dst, g.N, -0.5, 3, 32, 0)  # the server still serves
    assert sv.wait(ok)[0] == "done"
    st = sv.stats()
    assert st["cancelled"] == 1 and st["completed"] == 12 and st["failed"] == 2
    sv.close()



def test_forget_finished_requests(api):
    """A long-running server drops the records of requests whose results were read: a finished
    request can be forgotten (its output stays as it was), a queued one cannot, and a forgotten
    ticket is unknown afterwards."""
    g = synth.dcsbm(20000, 8, 20, 2.5, 5, seed=44)
    sv = api.Server(slots=1)
    ts = [sv.submit(g.src, g.dst, g.N, -0.5, 10, 64, k) for k in range(16)]
    with pytest.raises(api.IgpError) as e:  # still queued behind fifteen others on one slot
        sv.forget(ts[-1])
    assert e.value.status == api.IGP_E_BUSY
    for t in ts:
        assert sv.wait(t)[0] == "done"
    first = sv.result(ts[0]).copy()
    out = sv.forget(ts[0])
    assert np.array_equal(out, first)
    assert sv.poll(ts[0])[2] == api.IGP_E_INVAL
    with pytest.raises(api.IgpError) as e:
        sv.forget(ts[0])
    assert e.value.status == api.IGP_E_INVAL
    for t in ts[1:]:
        sv.forget(t)
    t = sv.submit(g.src, g.dst, g.N, -0.5, 10, 64, 0)  # the same request as the first, served again
    assert sv.wait(t)[0] == "done"
    assert np.array_equal(sv.forget(t), first)
    assert sv.stats()["completed"] == 17
    sv.close()

def test_continuous_batches_equal_each_request_alone(api):
    """Many compatible small requests in flight at once are embedded in shared batches; each
    result equals igp_embed of that graph alone (to fp32 rounding)."""
    gs = [synth.dcsbm(3000 + 997 * k, 6 + k % 4, 14 + k % 7, 2.4, 5, seed=300 + k) for k in range(16)]
    sv = api.Server(slots=8, batch_rows=100_000)
    tickets = [sv.submit(g.src, g.dst, g.N, -0.5, 6, 64, 50 + k, storage="bf16") for k, g in enumerate(gs)]
    for t in tickets:
        assert sv.wait(t)[0] == "done"
    st = sv.stats()
    assert st["completed"] == len(gs) and st["failed"] == 0
    assert st["batches"] >= 1 and st["batched"] >= 2, st
    for k, (g, t) in enumerate(zip(gs, tickets)):
        gr = api.graph_build(g.src, g.dst, g.N)
        assert _rel(sv.result(t), api.embed(gr, -0.5, 6, 64, 50 + k, storage="bf16")) <= AGREE["bf16"], k
        gr.free()
    sv.close()
