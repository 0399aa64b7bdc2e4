"""Graph Challenge quality measures (precision, recall, F1, ARI; Sec. IV "Evaluation Protocols") and
NMI, pinned against brute force over all node pairs on small labelings, the pair-confusion form of
the ARI, closed forms, and scikit-learn's implementations where that library is importable."""
import itertools
import math

import numpy as np
import pytest

from paper_2508_19737_gb300 import metrics


def _labelings():
    rng = np.random.default_rng(5)
    cases = [(np.zeros(1, int), np.zeros(1, int)), (np.arange(7), np.arange(7)), (np.zeros(9, int), np.arange(9)),
             (np.zeros(8, int), np.zeros(8, int)), (np.arange(8) % 2, np.arange(8) // 4)]
    for n in (2, 3, 10, 25, 40):
        for kt, kp in ((2, 3), (5, 5), (n, 2)):
            cases.append((rng.integers(0, kt, n) * 7 + 3, rng.integers(0, kp, n) - 11))
    return cases


def _brute_pairs(t, p):
    tp = fp = fn = tn = 0
    for i, j in itertools.combinations(range(len(t)), 2):
        st, sp = t[i] == t[j], p[i] == p[j]
        tp += st and sp
        fp += sp and not st
        fn += st and not sp
        tn += not st and not sp
    return tp, fp, fn, tn


@pytest.mark.parametrize("k", range(len(_labelings())))
def test_pair_measures_equal_brute_force(k):
    t, p = _labelings()[k]
    tp, fp, fn, tn = _brute_pairs(t, p)
    both, pt, pp, total = metrics.pair_counts(t, p)
    assert (both, pt, pp, total) == (tp, tp + fn, tp + fp, tp + fp + fn + tn)
    precision, recall, f1 = metrics.pairwise_scores(t, p)
    assert precision == (tp / (tp + fp) if tp + fp else 1.0)
    assert recall == (tp / (tp + fn) if tp + fn else 1.0)
    if precision + recall:
        assert f1 == pytest.approx(2 * precision * recall / (precision + recall), rel=1e-12)
    # ARI in its pair-confusion form (Steinley 2004), an independent algebraic route
    den = (tp + fn) * (fn + tn) + (tp + fp) * (fp + tn)
    ari = 2 * (tp * tn - fn * fp) / den if den else 1.0
    assert metrics.adjusted_rand_index(t, p) == pytest.approx(ari, abs=1e-12)


def _brute_nmi(t, p):
    n = len(t)
    pt = {a: np.mean(t == a) for a in set(t.tolist())}
    pp = {b: np.mean(p == b) for b in set(p.tolist())}
    ht = -sum(v * math.log(v) for v in pt.values())
    hp = -sum(v * math.log(v) for v in pp.values())
    if ht == 0 and hp == 0:
        return 1.0
    if ht == 0 or hp == 0:
        return 0.0
    mi = 0.0
    for a in pt:
        for b in pp:
            pab = sum(1 for i in range(n) if t[i] == a and p[i] == b) / n
            if pab > 0:
                mi += pab * math.log(pab / (pt[a] * pp[b]))
    return mi / ((ht + hp) / 2)


@pytest.mark.parametrize("k", range(len(_labelings())))
def test_nmi_equals_brute_force(k):
    t, p = _labelings()[k]
    assert metrics.nmi(t, p) == pytest.approx(_brute_nmi(t, p), abs=1e-12)


def test_closed_forms_and_invariances():
    t = np.repeat(np.arange(6), 50)
    s = metrics.scores(t, t)
    assert s["precision"] == s["recall"] == s["f1"] == 1.0 and s["ari"] == 1.0 and s["nmi"] == pytest.approx(1.0)
    # a relabelling of the blocks changes nothing
    perm = np.random.default_rng(0).permutation(6)
    assert metrics.scores(t, perm[t] + 100) == s
    # independent partitions of a balanced grid: mutual information exactly 0
    g = np.arange(400)
    assert metrics.nmi(g % 4, g // 100) == pytest.approx(0.0, abs=1e-12)
    # every node alone: no together pair in pred -> precision 1 (claims nothing), recall 0
    assert metrics.pairwise_scores(t, np.arange(t.size)) == (1.0, 0.0, 0.0)
    # one block in pred: recall 1, precision = fraction of together pairs in truth
    prec, rec, _ = metrics.pairwise_scores(t, np.zeros_like(t))
    assert rec == 1.0 and prec == pytest.approx(6 * math.comb(50, 2) / math.comb(300, 2))
    with pytest.raises(ValueError):
        metrics.scores(t, t[:-1])


def test_agree_with_scikit_learn():
    skm = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(9)
    for _ in range(20):
        n = int(rng.integers(2, 3000))
        t = rng.integers(0, int(rng.integers(1, 40)), n)
        p = np.where(rng.random(n) < 0.7, t, rng.integers(0, 50, n))
        assert metrics.adjusted_rand_index(t, p) == pytest.approx(skm.adjusted_rand_score(t, p), abs=1e-10)
        assert metrics.nmi(t, p) == pytest.approx(skm.normalized_mutual_info_score(t, p), abs=1e-10)
