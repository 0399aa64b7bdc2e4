"""Host logic of the streaming partitioner (the extraction of new rows and the clustering steps of Alg. 2), with the library calls replaced by the
FP64 oracle: each step hands exactly the new nodes' rows of that step's FFP to partial_fit, keeps
the old rows, predicts every node, runs the clustering of step t while step t+1's FFP is under way,
and reports clustering failures on the caller's thread. (The CUDA path itself is covered by the
GPU tests of the same pipeline.)"""
import threading

import numpy as np
import pytest

import oracle
from paper_2508_19737_gb300 import stream, synth


class _OracleGraph:
    def __init__(self, src, dst, N):
        self.src, self.dst, self.n = [np.asarray(src)], [np.asarray(dst)], int(N)

    @property
    def N(self):
        return self.n

    def append(self, src, dst, N, stream=None):
        self.src.append(np.asarray(src))
        self.dst.append(np.asarray(dst))
        self.n = int(N)

    def free(self):
        pass


class _OracleApi:
    """graph_build / embed with the library's signatures, computed by the FP64 oracle."""

    def __init__(self):
        self.embedded = []  # (seed, out_row_begin) per call
        self.events = {}

    def graph_build(self, src, dst, N, stream=None):
        return _OracleGraph(src, dst, N)

    def embed(self, g, tau, L, d, seed, stream=None, storage="f32", out_row_begin=0, **kw):
        self.embedded.append((seed, out_row_begin))
        self.events.setdefault(len(self.embedded) - 1, threading.Event()).set()
        X = oracle.theta_input(seed, g.N, d)
        Z = oracle.ffp_from_edges(np.concatenate(g.src), np.concatenate(g.dst), g.N, X, tau, L)
        return Z[out_row_begin:].astype(np.float32)


class _Recorder:
    """Nearest-centre clusterer with a fixed radius; records what it was given and on which thread."""

    def __init__(self, radius, wait_for=None):
        self.radius, self.C, self.fits, self.threads, self.wait_for, self.overlapped = radius, None, [], [], wait_for, []

    def partial_fit(self, X):
        if self.wait_for is not None:  # step t waits (bounded) for step t+1's FFP to start
            ev = self.wait_for(len(self.fits))
            self.overlapped.append(ev.wait(10.0) if ev is not None else None)
        self.fits.append(X.copy())
        self.threads.append(threading.current_thread().name)
        for x in X:
            if self.C is None:
                self.C = x[None].copy()
                continue
            dist = np.linalg.norm(self.C - x, axis=1)
            if dist.min() > self.radius:
                self.C = np.vstack([self.C, x])
        return self

    def predict(self, X):
        return np.argmin(((X[:, None, :] - self.C[None]) ** 2).sum(-1), axis=1)


def _increments():
    g = synth.dcsbm(600, 4, 10, 2.5, 5, seed=3)
    return g, synth.split_increments(g, T=4, mode="snowball", seed=1)


def test_each_step_fits_the_new_rows_and_predicts_every_node(monkeypatch):
    fake = _OracleApi()
    monkeypatch.setattr(stream, "api", fake)
    g, incs = _increments()
    cl = _Recorder(radius=1.5)
    sp = stream.StreamingPartitioner(cl, tau=-0.5, L=3, d=8, seed=40, storage="f32")
    steps = [sp.step(*inc) for inc in incs]
    labs = [sp.labels(t, timeout=60) for t in steps]
    sp.close()
    n_prev = 0
    acc_s, acc_d = [], []
    for t, (s, d, n) in enumerate(incs):
        acc_s.append(s)
        acc_d.append(d)
        Z = oracle.ffp_from_edges(np.concatenate(acc_s), np.concatenate(acc_d), n, oracle.theta_input(40, n, 8),
                                  -0.5, 3).astype(np.float32)
        assert fake.embedded[t] == (40, n_prev)  # one seed: old nodes keep their Theta rows; new rows only
        assert np.array_equal(cl.fits[t], Z[n_prev:])  # partial fit on the new rows
        assert labs[t].shape == (n,)
        n_prev = n
    kept = np.concatenate(cl.fits)  # old nodes keep the rows of the step that added them
    assert np.array_equal(labs[-1], cl.predict(kept))  # every node assigned
    assert set(cl.threads) == {"igp-stream-cluster"}
    assert all(sp.timings[t]["ffp_s"] >= 0 and sp.timings[t]["cluster_s"] >= 0 for t in steps)


def test_clustering_of_a_step_overlaps_the_next_ffp(monkeypatch):
    fake = _OracleApi()
    monkeypatch.setattr(stream, "api", fake)
    _, incs = _increments()
    cl = _Recorder(radius=1.5, wait_for=lambda t: fake.events.setdefault(t + 1, threading.Event())
                   if t + 1 < len(incs) else None)
    sp = stream.StreamingPartitioner(cl, L=2, d=8, storage="f32")
    for inc in incs:
        sp.step(*inc)
    sp.labels(len(incs) - 1, timeout=120)
    sp.close()
    assert cl.overlapped == [True] * (len(incs) - 1) + [None]


def test_a_failing_clusterer_is_reported_to_the_caller(monkeypatch):
    monkeypatch.setattr(stream, "api", _OracleApi())
    _, incs = _increments()

    class Broken(_Recorder):
        def partial_fit(self, X):
            raise ValueError("planted")

    sp = stream.StreamingPartitioner(Broken(1.0), L=2, d=8, storage="f32")
    t = sp.step(*incs[0])
    with pytest.raises(RuntimeError) as e:
        sp.labels(t, timeout=60)
    assert isinstance(e.value.__cause__, ValueError)
    with pytest.raises(RuntimeError):
        sp.step(*incs[1])
    sp.close()
    with pytest.raises(ValueError):
        sp.labels(7)


def test_birch_in_the_pipeline_equals_birch_run_step_by_step(monkeypatch):
    pytest.importorskip("sklearn")
    monkeypatch.setattr(stream, "api", _OracleApi())
    _, incs = _increments()
    sp = stream.StreamingPartitioner(stream.birch(threshold=0.6), L=3, d=8, seed=2, storage="f32")
    got = [sp.labels(sp.step(*inc), timeout=120) for inc in incs]
    sp.close()
    ref_cl = stream.birch(threshold=0.6)
    acc_s, acc_d, kept = [], [], []
    n_prev = 0
    for t, (s, d, n) in enumerate(incs):
        acc_s.append(s)
        acc_d.append(d)
        Z = oracle.ffp_from_edges(np.concatenate(acc_s), np.concatenate(acc_d), n, oracle.theta_input(2, n, 8),
                                  -0.5, 3).astype(np.float32)
        ref_cl.partial_fit(Z[n_prev:])
        kept.append(Z[n_prev:])
        assert np.array_equal(got[t], ref_cl.predict(np.concatenate(kept)))
        n_prev = n
