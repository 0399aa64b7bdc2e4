"""Streaming graph partitioning (Alg. 2) around the CUDA FFP, with the clustering of each step
overlapped with the next step's FFP.

Step t, for an increment (V_t, E_t) whose new nodes carry the ids N_(t-1) .. N_t - 1 (the snowball
model of Sec. II numbers nodes in arrival order):

* merge: the increment is merged into the device-resident cumulative CSR (igp_graph_append; the
  first step builds it, which is Alg. 1 on (V_1, E_1));
* embed: one FFP over all N_t nodes with Theta of the cumulative size from the same seed at
  every step, so each old node keeps its row of Theta and each new node gets a fresh one (row i
  of Theta depends on the seed and i alone); a fresh draw of every row at every step would put
  the rows kept from earlier steps and the new rows into unrelated coordinates;
* extract: only the new nodes' rows leave the device (igp_embed with out_row_begin = N_(t-1));
* fit: the clusterer is partially fitted on those rows;
* keep: they are appended to the rows kept from earlier steps (old nodes keep the rows of the step
  that added them);
* assign: the clusterer assigns a block to every node so far.

Merge, embed and extract run on the calling thread (the library call releases the interpreter lock
while the GPU works); fit, keep and assign run in step order on one host thread, so step t's
clustering overlaps step t+1's FFP. Any object with `partial_fit(X)` and `predict(X)` is a clusterer; `birch()` makes the
scikit-learn BIRCH the paper uses (Sec. IV-A) when that package is installed.
"""
import queue
import threading
import time

import numpy as np

from . import api

__all__ = ["StreamingPartitioner", "static_partition", "birch"]


def birch(threshold=0.5, branching_factor=50):
    """A K-agnostic BIRCH (n_clusters=None) from scikit-learn."""
    try:
        from sklearn.cluster import Birch
    except ImportError as e:  # pragma: no cover - depends on the host
        raise ImportError("BIRCH needs scikit-learn; pass any object with partial_fit and predict instead") from e
    return Birch(threshold=threshold, branching_factor=branching_factor, n_clusters=None)


class StreamingPartitioner:
    """Alg. 2 over a stream of edge increments; see the module docstring.

    step(src, dst, N_t) runs merge, embed and extract and queues fit, keep and assign, returning
    the step index t;
    labels(t) waits for step t's partition C^(t) (one block id per node 0 .. N_t - 1).
    timings[t] holds the seconds of the GPU part ("ffp_s": merge, embed and extract, including the
    copy of the new rows) and of the host part ("cluster_s": fit, keep and assign) of each finished
    step.
    """

    def __init__(self, clusterer, tau=-0.5, L=10, d=64, seed=0, storage="bf16", stream=None, **opts):
        self.clusterer = clusterer
        self.tau, self.L, self.d, self.seed = float(tau), int(L), int(d), int(seed)
        self.storage, self.stream, self.opts = storage, stream, opts
        self.graph = None
        self._t = 0
        self._rows = []
        self._labels = {}
        self.timings = {}
        self._error = None
        self._done = threading.Condition()
        self._q = queue.Queue()
        self._worker = threading.Thread(target=self._cluster_loop, name="igp-stream-cluster", daemon=True)
        self._worker.start()

    # merge, embed, extract -----------------------------------------------------------------
    def step(self, src, dst, N_t):
        self._raise_pending()
        t = self._t
        t0 = time.perf_counter()
        if self.graph is None:
            self.graph = api.graph_build(src, dst, N_t, stream=self.stream)
            row0 = 0
        else:
            row0 = self.graph.N
            self.graph.append(src, dst, N_t, stream=self.stream)
        rows = api.embed(self.graph, self.tau, self.L, self.d, self.seed, stream=self.stream,
                         storage=self.storage, out_row_begin=row0, **self.opts)
        self.timings[t] = {"ffp_s": time.perf_counter() - t0, "new_rows": rows.shape[0]}
        self._t += 1
        self._q.put((t, rows))
        return t

    # fit, keep, assign ---------------------------------------------------------------------
    def _cluster_loop(self):
        while True:
            item = self._q.get()
            if item is None:
                return
            t, rows = item
            try:
                t0 = time.perf_counter()
                if rows.shape[0]:
                    self.clusterer.partial_fit(rows)  # fit
                self._rows.append(rows)  # keep
                kept = np.concatenate(self._rows) if len(self._rows) > 1 else self._rows[0]
                if len(self._rows) > 1:
                    self._rows = [kept]
                lab = np.asarray(self.clusterer.predict(kept))  # assign
                dt = time.perf_counter() - t0
                with self._done:
                    self.timings[t]["cluster_s"] = dt
                    self._labels[t] = lab
                    self._done.notify_all()
            except BaseException as e:  # reported by the next step() / labels() call
                with self._done:
                    self._error = e
                    self._done.notify_all()
                return

    def labels(self, t, timeout=None):
        """Block ids of step t (waits for its clustering)."""
        if not 0 <= t < self._t:
            raise ValueError(f"step {t} was not submitted")
        with self._done:
            ok = self._done.wait_for(lambda: t in self._labels or self._error is not None, timeout)
            if self._error is not None:
                raise RuntimeError("clustering failed") from self._error
            if not ok:
                raise TimeoutError(f"step {t} not clustered within {timeout} s")
            return self._labels[t]

    def _raise_pending(self):
        with self._done:
            if self._error is not None:
                raise RuntimeError("clustering failed") from self._error

    def close(self):
        """Finish queued clustering, stop the host thread and free the device graph."""
        if self._worker.is_alive():
            self._q.put(None)
            self._worker.join()
        if self.graph is not None:
            self.graph.free()
            self.graph = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def static_partition(src, dst, N, clusterer, tau=-0.5, L=10, d=64, seed=0, storage="bf16", stream=None, **opts):
    """Alg. 1 from scratch (the baseline the streaming variant is compared with): build, one FFP over
    all nodes, fit the clusterer to every row and predict. Returns (labels, seconds of the GPU part,
    seconds of the clustering)."""
    t0 = time.perf_counter()
    g = api.graph_build(src, dst, N, stream=stream)
    try:
        Z = api.embed(g, tau, L, d, seed, stream=stream, storage=storage, **opts)
    finally:
        g.free()
    t1 = time.perf_counter()
    clusterer.partial_fit(Z)
    lab = np.asarray(clusterer.predict(Z))
    return lab, t1 - t0, time.perf_counter() - t1
