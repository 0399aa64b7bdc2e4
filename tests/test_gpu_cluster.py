"""The device clusterer (igp_clusterer_*, BIRCH's leaf level in batches) against its oracle
(oracle/cluster.py): labels, entry counts and centroids bit for bit, on random points and on FFP
embeddings computed by the FP64 oracle, with partial fits, predict and the error paths."""
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


def _blobs(seed, N, d, k=12, sd=0.1):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, size=(k, d))
    return np.clip(centres[rng.integers(0, k, N)] + rng.normal(0, sd, size=(N, d)), 0, 1).astype(np.float32)


def _same(api, cl, lab, st, got):
    K, C, n = cl.info(centroids=True, counts=True)
    assert np.array_equal(got, lab)
    assert K == st.K
    assert np.array_equal(n, st.n)
    assert np.array_equal(C.view(np.uint32), st.C.view(np.uint32))


@pytest.mark.parametrize("d,batch,T", [(8, 1, 0.3), (16, 37, 0.35), (32, 512, 0.5), (64, 4096, 1.0),
                                       (128, 300, 0.9), (32, 1024, 0.05)])
def test_fit_equals_oracle_bit_for_bit(api, d, batch, T):
    E = _blobs(d + batch, 3000 if batch > 1 else 600, d)
    lab, st = oracle.cf_cluster(E, T, batch=batch)
    cl = api.Clusterer(d, T, batch=batch)
    got = cl.fit(E)
    _same(api, cl, lab, st, got)
    cl.free()


def test_fit_on_ffp_embeddings_device_buffers_and_partial_fits(api):
    """Embeddings of a graph shaped like the paper's benchmark graphs (5,000 nodes, Table II's
    tau = -6, L = 10, d = 64), computed by the FP64 oracle and rounded to fp32; given to the
    device clusterer in device memory, in two partial fits."""
    import torch
    g = synth.challenge_like(5000, seed=3)
    rp, col = oracle.build_csr(g.src, g.dst, g.N)
    tau, L, d = synth.TABLE2_STATIC[5000]
    E = oracle.ffp(rp, col, oracle.theta_input(0, g.N, d), tau, L).astype(np.float32)
    T, B = 1.3, 512
    lab, st = oracle.cf_cluster(E, T, batch=B)
    cl = api.Clusterer(d, T, batch=B)
    Ed = torch.from_numpy(E).cuda()
    out = torch.full((g.N,), -7, dtype=torch.int32, device="cuda")
    cl.fit(Ed[:2048], labels=out[:2048])
    cl.fit(Ed[2048:], labels=out[2048:])
    torch.cuda.synchronize()
    _same(api, cl, lab, st, out.cpu().numpy())
    # predict on the device and on the host
    P = _blobs(9, 777, d, sd=0.2)
    ref = oracle.cf_predict(P, st)
    assert np.array_equal(cl.predict(P), ref)
    pd = torch.empty(777, dtype=torch.int32, device="cuda")
    cl.predict(torch.from_numpy(P).cuda(), labels=pd)
    torch.cuda.synchronize()
    assert np.array_equal(pd.cpu().numpy(), ref)
    cl.free()


def test_fit_errors(api):
    d = 16
    cl = api.Clusterer(d, 0.3, batch=64, max_entries=10)
    with pytest.raises(api.IgpError) as e:
        cl.predict(_blobs(1, 5, d))
    assert e.value.status == api.IGP_E_INVAL  # nothing fitted yet
    bad = _blobs(2, 100, d)
    bad[37, 3] = 1.5
    with pytest.raises(api.IgpError) as e:
        cl.fit(bad)
    assert e.value.status == api.IGP_E_INVAL
    assert cl.info()[0] == 0  # nothing fitted
    bad[37, 3] = np.nan
    with pytest.raises(api.IgpError):
        cl.fit(bad)
    # more than max_entries entries: the batches before the overflowing one stay fitted
    E = np.random.default_rng(3).uniform(0, 1, size=(640, d)).astype(np.float32)
    with pytest.raises(api.IgpError) as e:
        cl.fit(E)
    assert e.value.status == api.IGP_E_NOMEM
    assert cl.info()[0] <= 10
    cl.free()
    with pytest.raises(api.IgpError):
        api.Clusterer(24, 0.3)
    with pytest.raises(api.IgpError):
        api.Clusterer(32, 0.0)


def test_large_fit_matches_oracle(api):
    """100,000 points of d = 16 in batches of 1,024 (98 batches, several hundred entries)."""
    E = _blobs(11, 100_000, 16, k=20, sd=0.04)
    T = 0.2
    lab, st = oracle.cf_cluster(E, T, batch=1024)
    cl = api.Clusterer(16, T, batch=1024)
    got = cl.fit(E)
    _same(api, cl, lab, st, got)
    print(f"100K points: K = {st.K}")
    cl.free()
