"""Partition quality measures of the Graph Challenge protocol (Sec. IV, "Evaluation Protocols"):
pairwise precision, recall and their F1-score, the adjusted Rand index (ARI), and normalised mutual
information (NMI) as a clusterer-independent check of embedding quality.

All of them are functions of the contingency table n_ab = |{i : truth_i = a, pred_i = b}| of two
labelings of the same nodes; nothing here runs on the GPU. Definitions:

* A node pair is "together" in a labeling when both nodes carry the same label. With
  P_true = sum_a C(n_a., 2), P_pred = sum_b C(n_.b, 2) and P_both = sum_ab C(n_ab, 2):
  precision = P_both / P_pred, recall = P_both / P_true, F1 = their harmonic mean
  (a labeling with no together pair has precision or recall 1 by convention: it claims nothing).
* ARI (Hubert and Arabie, 1985): (P_both - E) / ((P_true + P_pred) / 2 - E),
  E = P_true P_pred / C(n, 2); 1 when both labelings put every pair alike.
* NMI: I(truth; pred) / ((H(truth) + H(pred)) / 2) in nats, 1 for identical partitions; 1 as
  well when both are a single block, 0 when exactly one of them is.
"""
import numpy as np

__all__ = ["contingency", "pair_counts", "pairwise_scores", "adjusted_rand_index", "nmi", "scores"]


def _table(truth, pred):
    """Nonzero cells of the contingency table as (row index, column index, count), with the row
    sums n_a. and column sums n_.b."""
    t = np.asarray(truth).ravel()
    p = np.asarray(pred).ravel()
    if t.shape != p.shape:
        raise ValueError("truth and pred must label the same nodes")
    _, ti = np.unique(t, return_inverse=True)
    _, pi = np.unique(p, return_inverse=True)
    ncol = int(pi.max()) + 1 if pi.size else 1
    key, cnt = np.unique(ti.astype(np.int64) * ncol + pi, return_counts=True)
    return key // ncol, key % ncol, cnt.astype(np.int64), np.bincount(ti).astype(np.int64), \
        np.bincount(pi).astype(np.int64)


def contingency(truth, pred):
    """Nonzero cells of the contingency table: (counts n_ab, row sums n_a., column sums n_.b)."""
    _, _, cnt, a, b = _table(truth, pred)
    return cnt, a, b


def _c2(x):
    x = np.asarray(x, dtype=np.int64)
    return int(np.sum(x * (x - 1) // 2))


def pair_counts(truth, pred):
    """(P_both, P_true, P_pred, C(n, 2)): pairs together in both, in truth, in pred, and all pairs."""
    cells, a, b = contingency(truth, pred)
    n = int(a.sum())
    return _c2(cells), _c2(a), _c2(b), n * (n - 1) // 2


def pairwise_scores(truth, pred):
    """Graph Challenge pairwise precision, recall and F1-score."""
    both, pt, pp, _ = pair_counts(truth, pred)
    precision = both / pp if pp else 1.0
    recall = both / pt if pt else 1.0
    f1 = 2 * precision * recall / (precision + recall) if precision + recall > 0 else 0.0
    return precision, recall, f1


def adjusted_rand_index(truth, pred):
    both, pt, pp, total = pair_counts(truth, pred)
    if total == 0:
        return 1.0
    expected = pt * pp / total
    top = (pt + pp) / 2 - expected
    if top == 0:  # both labelings trivial in the same way (all singletons or one block)
        return 1.0
    return (both - expected) / top


def nmi(truth, pred):
    ri, ci, cnt, a, b = _table(truth, pred)
    n = float(a.sum())
    if n == 0:
        return 1.0
    ha = -float(np.sum(a / n * np.log(a / n)))
    hb = -float(np.sum(b / n * np.log(b / n)))
    if ha == 0.0 and hb == 0.0:
        return 1.0
    if ha == 0.0 or hb == 0.0:
        return 0.0
    # I = sum_ab (n_ab / n) log(n n_ab / (n_a. n_.b))
    mi = float(np.sum(cnt / n * (np.log(cnt * n) - np.log(a[ri].astype(np.float64) * b[ci]))))
    return max(0.0, mi / ((ha + hb) / 2))


def scores(truth, pred):
    """All measures of the protocol as a dict."""
    precision, recall, f1 = pairwise_scores(truth, pred)
    return {"precision": precision, "recall": recall, "f1": f1, "ari": adjusted_rand_index(truth, pred),
            "nmi": nmi(truth, pred), "blocks_true": int(np.unique(truth).size),
            "blocks_pred": int(np.unique(pred).size)}
