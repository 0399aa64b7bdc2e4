"""Plain reference of the library's K-agnostic clusterer (the GPU stand-in for BIRCH).

TEST INFRASTRUCTURE ONLY (see the package docstring). The paper clusters the FFP embeddings with
BIRCH (Alg. 1's last step, Alg. 2's fit and assign; Sec. IV-A), whose leaf entries are clustering
features CF = (n, LS, SS) (the point count, the linear sum and the sum of squared norms of the
members; Zhang, Ramakrishnan, Livny, SIGMOD 1996): a point joins the closest leaf entry if the
merged entry's radius sqrt(SS/n - |LS/n|^2) stays within the threshold T, and otherwise starts a
new entry; without a global clustering step at the end the leaf entries are the clusters, so
their number K is not fixed in advance. The library keeps that leaf level and drops the tree:
the closest entry is found by an exhaustive search, points are taken in batches of B against
the entries as they stood at the start of the batch, and the new entries a batch needs are
chosen by a threshold-leader rule among its leftover points. For the batch of points
b*B .. (b+1)*B - 1 (in index order):

  1. quantise: xq = round-half-even(x * 2^16) as integers; x' = xq / 2^16 (exact in fp32);
  2. each point: the closest entry c* (smallest fp32 squared distance |x' - C_c|^2, the sum over
     coordinates taken in coordinate order, each difference, product and sum rounded to fp32;
     ties go to the smaller c); it joins c* if the radius of CF(c*) + x, evaluated in fp64 from
     the exact integer sums as SS'/n' - sum_k (LS'_k / n')^2 (coordinates in order; every
     conversion, division, product and difference rounded to fp64), is at most (T 2^16)^2;
     otherwise it is a candidate;
  3. among the candidates: two candidates are close if they lie within T of each other
     (|x'_i - x'_j|^2 <= fp32(T^2), the same fp32 distance); a candidate is a leader if no
     earlier candidate of the batch is close to it; every other candidate joins the closest
     leader of the batch that is close to it (ties to the smaller index), or, with none, starts
     an entry of its own. (An entry made of a leader and members within T of it has radius at
     most T, as BIRCH's entries do: the centroid minimises the mean squared distance.)
  4. the new entries (leaders and the candidates left alone) are numbered on from K in index
     order and take their members' sums; the joins of step 2 are added to their entries' sums;
     every entry's centroid is C_c = fp32((double) LS_c / n_c / 2^16).

With batches of one point this is BIRCH's leaf rule, and no entry's radius exceeds T; in larger
batches the points that join one entry are each tested against it alone, so together they may
take its radius past T (the price of deciding a batch at once).

Integer sums make the entries independent of the order of additions, and every decision is taken
in fixed-order fp32 (distances) or fp64 (radii) arithmetic, so the GPU reproduces the labels
exactly. predict() gives each point its closest entry by the distance of step 2, without the
radius test and without changing the entries. Inputs must lie in [-1, 1] (FFP outputs are
sigmoids in (0, 1)).
"""
import numpy as np

__all__ = ["CFState", "cf_cluster", "cf_predict", "quantize", "QBITS"]

QBITS = 16
_Q = float(1 << QBITS)


class CFState:
    """The entries: counts n [K] int64, linear sums LS [K, d] int64, square sums SS [K] uint64
    (in units of 2^-16 and 2^-32), centroids C [K, d] fp32."""

    def __init__(self, d):
        self.d = d
        self.n = np.zeros(0, dtype=np.int64)
        self.LS = np.zeros((0, d), dtype=np.int64)
        self.SS = np.zeros(0, dtype=np.uint64)
        self.C = np.zeros((0, d), dtype=np.float32)

    @property
    def K(self):
        return int(self.n.size)


def quantize(E):
    """xq = round-half-even(x * 2^16) (int64) and x' = xq / 2^16 (fp32) of fp32 points."""
    E = np.asarray(E, dtype=np.float32)
    if E.size and (not np.all(np.isfinite(E)) or np.abs(E).max() > 1.0):
        raise ValueError("points must be finite and within [-1, 1]")
    xq = np.rint(E * np.float32(_Q)).astype(np.int64)
    return xq, (xq.astype(np.float32) / np.float32(_Q))


def _dist2(X, C):
    """fp32 squared distances (m x K), summed over coordinates in order, every op rounded."""
    s = np.zeros((X.shape[0], C.shape[0]), dtype=np.float32)
    for k in range(X.shape[1]):
        diff = X[:, k:k + 1] - C[None, :, k]
        s = s + diff * diff
    return s


def _merged_r2(n, LS, SS, xq):
    """Radius^2 * 2^32 of entries (n, LS, SS) each merged with its point xq (arrays over points):
    fp64 from the exact integer sums, SS'/n' minus the squares of LS'_k/n' added in order."""
    n1 = (n + 1).astype(np.float64)
    ss = (SS + (xq * xq).sum(axis=1).astype(np.uint64)).astype(np.float64)
    r2 = ss / n1
    b = np.zeros_like(r2)
    L1 = LS + xq
    for k in range(xq.shape[1]):
        m = L1[:, k].astype(np.float64) / n1
        b = b + m * m
    return r2 - b


def _centroids(n, LS):
    return ((LS.astype(np.float64) / n.astype(np.float64)[:, None]) / _Q).astype(np.float32)


def _add_u64(out, lab, vals):
    np.add.at(out, lab, vals.astype(np.uint64))


def cf_cluster(E, threshold, batch=4096, state=None, max_entries=1 << 20):
    """Fit the points E (N x d) in index order, starting from `state` (a CFState; None: no
    entries yet). Returns (labels int32 [N], state)."""
    xq, xp = quantize(E)
    N, d = xq.shape
    st = CFState(d) if state is None else state
    t2r = float(threshold) * _Q
    t2r = t2r * t2r                               # radius bound of step 2 (fp64, 2^-32 units)
    t2d = np.float32(float(threshold) * float(threshold))  # distance bound of step 3 (fp32)
    ssq = (xq * xq).sum(axis=1).astype(np.uint64)
    labels = np.full(N, -1, dtype=np.int64)
    for b0 in range(0, N, batch):
        idx = np.arange(b0, min(N, b0 + batch))
        K0 = st.K
        # step 2: the closest entry at the start of the batch, and BIRCH's radius test
        if K0:
            cstar = np.argmin(_dist2(xp[idx], st.C), axis=1)  # first minimum: the smaller id on ties
            ok = _merged_r2(st.n[cstar], st.LS[cstar], st.SS[cstar], xq[idx]) <= t2r
            labels[idx[ok]] = cstar[ok]
        cand = idx[labels[idx] < 0]
        # step 3: leaders among the candidates, then the others
        if cand.size:
            Dc = _dist2(xp[cand], xp[cand])
            close = Dc <= t2d
            earlier = np.tril(np.ones((cand.size, cand.size), dtype=bool), -1)
            leader = ~np.any(close & earlier, axis=1)
            own = leader.copy()                   # candidates that start an entry
            target = np.arange(cand.size)         # candidate whose entry each one joins
            lead_pos = np.nonzero(leader)[0]
            for p in np.nonzero(~leader)[0]:
                reach = lead_pos[close[p, lead_pos]]
                if reach.size:
                    target[p] = reach[np.argmin(Dc[p, reach])]  # first minimum: smaller index
                else:
                    own[p] = True
            # step 4 (new entries): numbered in index order
            if K0 + int(own.sum()) > max_entries:
                raise ValueError("more than max_entries entries")
            eid = np.full(cand.size, -1, dtype=np.int64)
            eid[own] = K0 + np.arange(int(own.sum()))
            labels[cand] = eid[target]
        # step 4: the sums
        K1 = max(K0, int(labels[idx].max()) + 1)  # every point of the batch has its entry now
        n = np.zeros(K1, dtype=np.int64)
        n[:K0] = st.n
        LS = np.zeros((K1, d), dtype=np.int64)
        LS[:K0] = st.LS
        SS = np.zeros(K1, dtype=np.uint64)
        SS[:K0] = st.SS
        lab = labels[idx]
        np.add.at(n, lab, 1)
        np.add.at(LS, lab, xq[idx])
        _add_u64(SS, lab, ssq[idx])
        st.n, st.LS, st.SS = n, LS, SS
        st.C = _centroids(n, LS)
    return labels.astype(np.int32), st


def cf_predict(E, state):
    """The closest entry of every point (fp32 distance of step 2; ties to the smaller id)."""
    _, xp = quantize(E)
    if state.K == 0:
        raise ValueError("no entries")
    return np.argmin(_dist2(xp, state.C), axis=1).astype(np.int32)
