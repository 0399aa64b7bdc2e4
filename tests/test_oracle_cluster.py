"""Pins of the clusterer oracle (oracle/cluster.py, BIRCH's leaf level in batches) to facts that do
not come from its own code: cases whose partition is known, BIRCH's radius invariant, the
clustering features as plain sums of the members, a pure-Python sequential BIRCH leaf loop that
the batch-of-one case reduces to, and the partition quality of scikit-learn's BIRCH on the same
embeddings."""
import math

import numpy as np
import pytest

import oracle
from oracle import cluster as oc
from paper_2508_19737_gb300 import metrics, synth


def _groups(seed, g, per, d, spread, gap):
    """g groups of `per` points: centres on a grid `gap` apart, points within `spread` of them,
    shuffled; returns (points in [0, 1], group of each point)."""
    rng = np.random.default_rng(seed)
    centres = 0.1 + gap * np.arange(g)[:, None] * np.eye(d)[0][None, :] + 0.05
    grp = np.repeat(np.arange(g), per)
    pts = centres[grp] + rng.uniform(-spread, spread, size=(g * per, d))
    order = rng.permutation(g * per)
    return np.clip(pts[order], 0, 1).astype(np.float32), grp[order]


def _same_partition(a, b):
    # a relabelling: one-to-one map between the label sets
    pairs = set(zip(a.tolist(), b.tolist()))
    return len(pairs) == len(set(a.tolist())) == len(set(b.tolist()))


@pytest.mark.parametrize("batch", [1, 7, 64, 4096])
def test_separated_groups_are_recovered(batch):
    """Groups 0.2 apart, each within a box of half-width 0.01 in 8 dims (diameter < 0.06), T = 0.05:
    every group is one entry, whatever the batch size."""
    E, grp = _groups(0, 5, 40, 8, 0.01, 0.2)
    lab, st = oracle.cf_cluster(E, 0.05, batch=batch)
    assert st.K == 5 and _same_partition(lab, grp)


def test_huge_threshold_gives_one_entry_and_tiny_threshold_one_per_distinct_point():
    rng = np.random.default_rng(1)
    E = rng.uniform(0, 1, size=(300, 16)).astype(np.float32)
    E[100:110] = E[5]  # ten repeats of one point
    lab, st = oracle.cf_cluster(E, 10.0, batch=64)
    assert st.K == 1 and np.all(lab == 0)
    lab, st = oracle.cf_cluster(E, 1e-6, batch=64)
    distinct = np.unique(np.rint(E.astype(np.float64) * 65536), axis=0).shape[0]
    assert st.K == distinct == 290
    assert len(set(lab[[5] + list(range(100, 110))].tolist())) == 1


def _seq_leaf_birch(E, T):
    """BIRCH's leaf rule, one point at a time, in pure Python (lists, math): the point joins the
    entry with the closest centroid if the merged radius is at most T, else starts an entry."""
    entries = []  # [n, LS (list of ints), SS (int)]
    labels = []
    for row in E:
        xq = [round(float(v) * 65536) for v in row]  # Python's round: half to even
        x = [v / 65536 for v in xq]
        best, bd = -1, math.inf
        for c, (n, LS, SS) in enumerate(entries):
            dd = sum((x[k] - LS[k] / n / 65536) ** 2 for k in range(len(x)))
            if dd < bd:
                best, bd = c, dd
        if best >= 0:
            n, LS, SS = entries[best]
            n1 = n + 1
            L1 = [LS[k] + xq[k] for k in range(len(x))]
            S1 = SS + sum(v * v for v in xq)
            r2 = S1 / n1 - sum((v / n1) ** 2 for v in L1)
            if math.sqrt(max(r2, 0.0)) / 65536 <= T:
                entries[best] = [n1, L1, S1]
                labels.append(best)
                continue
        entries.append([1, xq, sum(v * v for v in xq)])
        labels.append(len(entries) - 1)
    return np.array(labels)


@pytest.mark.parametrize("seed,T", [(0, 0.3), (1, 0.5), (2, 0.8)])
def test_batch_of_one_is_the_sequential_birch_leaf_rule(seed, T):
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.2, 0.8, size=(6, 8))
    E = np.clip(centres[rng.integers(0, 6, 250)] + rng.normal(0, 0.12, size=(250, 8)), 0, 1).astype(np.float32)
    lab, st = oracle.cf_cluster(E, T, batch=1)
    ref = _seq_leaf_birch(E, T)
    assert np.array_equal(lab, ref)
    assert st.K == ref.max() + 1


@pytest.mark.parametrize("batch", [1, 32, 500])
def test_entries_are_member_sums_and_one_by_one_keep_the_radius_bound(batch):
    rng = np.random.default_rng(3)
    E = rng.uniform(0, 1, size=(700, 16)).astype(np.float32)
    T = 0.45
    lab, st = oracle.cf_cluster(E, T, batch=batch)
    xq = np.rint(E.astype(np.float64) * 65536).astype(np.int64)
    for c in range(st.K):
        mem = xq[lab == c]
        assert st.n[c] == len(mem) > 0
        assert np.array_equal(st.LS[c], mem.sum(axis=0))
        assert int(st.SS[c]) == int((mem * mem).sum())
        cen = mem.mean(axis=0) / 65536
        np.testing.assert_allclose(st.C[c], cen, rtol=1e-6, atol=1e-7)
        if batch == 1:  # point by point, BIRCH's bound holds; in batches several joins of one
            # batch are each tested alone and may take an entry past T together
            radius = math.sqrt(max(0.0, ((mem / 65536 - cen) ** 2).sum(axis=1).mean()))
            assert radius <= T + 1e-9, (c, radius)


def test_partial_fits_equal_one_fit_when_batches_align():
    rng = np.random.default_rng(4)
    E = rng.uniform(0, 1, size=(1000, 8)).astype(np.float32)
    lab, st = oracle.cf_cluster(E, 0.4, batch=100)
    a, sa = oracle.cf_cluster(E[:600], 0.4, batch=100)
    b, sb = oracle.cf_cluster(E[600:], 0.4, batch=100, state=sa)
    assert np.array_equal(lab, np.concatenate([a, b]))
    assert np.array_equal(st.LS, sb.LS) and np.array_equal(st.C, sb.C)


def test_predict_is_the_closest_centroid():
    rng = np.random.default_rng(5)
    E = rng.uniform(0, 1, size=(400, 8)).astype(np.float32)
    _, st = oracle.cf_cluster(E, 0.35, batch=50)
    P = rng.uniform(0, 1, size=(300, 8)).astype(np.float32)
    got = oracle.cf_predict(P, st)
    xp = np.rint(P.astype(np.float64) * 65536) / 65536
    D = ((xp[:, None, :] - st.C.astype(np.float64)[None, :, :]) ** 2).sum(axis=2)
    ref = D.argmin(axis=1)
    gap = np.sort(D, axis=1)[:, 1] - np.sort(D, axis=1)[:, 0]
    clear = gap > 1e-5  # away from fp32-level near-ties
    assert clear.mean() > 0.95 and np.array_equal(got[clear], ref[clear])


def test_quality_matches_scikit_learn_birch():
    """On the FFP embeddings of a graph shaped like the paper's benchmark graphs (10,000 nodes,
    25 blocks, Table II's tau = -3, L = 9, d = 64), at thresholds 1.0 and 1.3 the partition's NMI
    and pairwise F1 against the planted blocks are within 0.05 of scikit-learn's BIRCH
    (n_clusters=None, the same threshold)."""
    skc = pytest.importorskip("sklearn.cluster")
    g = synth.challenge_like(10_000, seed=1)
    rp, col = oracle.build_csr(g.src, g.dst, g.N)
    tau, L, d = synth.TABLE2_STATIC[10_000]
    E = oracle.ffp(rp, col, oracle.theta_input(0, g.N, d), tau, L).astype(np.float32)
    for T in (1.0, 1.3):
        lab, _ = oracle.cf_cluster(E, T, batch=512)
        ref = skc.Birch(threshold=T, n_clusters=None).fit_predict(E)
        ours = metrics.nmi(g.blocks, lab), metrics.pairwise_scores(g.blocks, lab)[2]
        theirs = metrics.nmi(g.blocks, ref), metrics.pairwise_scores(g.blocks, ref)[2]
        assert ours[0] >= theirs[0] - 0.05 and ours[1] >= theirs[1] - 0.05, (T, ours, theirs)
