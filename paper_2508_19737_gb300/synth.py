"""Seeded synthetic inputs: degree-corrected stochastic block model (DC-SBM) graphs.

This module only draws inputs. It holds none of the method's arithmetic, imports
neither the CUDA library nor the CPU checker, and both sides are fed from it.

The paper evaluates on the IEEE HPEC Graph Challenge graphs (Sec. IV-A, Table I:
planted blocks, heterogeneous block sizes, power-law degrees, mean degree ~40).
Those files are not available here, so a seeded DC-SBM with the same kind of
structure stands in for them:

* node propensities theta_i from a power law p(x) ~ x^-gamma on [1, 100]
  (inverse CDF);
* block sizes equal (largest-remainder split) or Dirichlet(alpha) * N rounded
  by largest remainder, every block non-empty;
* M = round(N * mean_deg / 2) undirected edge draws with
  P(u, v) ~ theta_u theta_v w(b_u, b_v), w = ratio inside a block and 1 across:
  u is drawn with weight theta_u (ratio Th_{b_u} + Th_tot - Th_{b_u}), then the
  draw is intra-block with probability ratio Th_{b_u} / (ratio Th_{b_u} +
  Th_tot - Th_{b_u}), and v is drawn with weight theta_v inside the chosen side.
  Self-loops and repeated pairs are left in; the CSR build drops and merges them.
* node labels: a random permutation ("random"), or block-major with nodes in
  decreasing drawn degree inside each block ("block_degree").
"""
import numpy as np

__all__ = ["DCSBM", "dcsbm", "powerlaw_propensities", "block_sizes", "batch_dcsbm",
           "split_increments", "log_uniform_sizes"]


class DCSBM:
    """A drawn graph: int32 edge arrays (src, dst), N, and per-node block labels."""

    def __init__(self, src, dst, N, blocks, theta, seed, params):
        self.src = src
        self.dst = dst
        self.N = N
        self.blocks = blocks
        self.theta = theta
        self.seed = seed
        self.params = params

    @property
    def M(self):
        return int(self.src.size)

    def __repr__(self):
        return f"DCSBM(N={self.N}, M={self.M}, blocks={int(self.blocks.max()) + 1}, seed={self.seed})"


def powerlaw_propensities(rng, n, gamma, lo=1.0, hi=100.0):
    """n draws from p(x) ~ x^-gamma on [lo, hi] (inverse CDF, gamma != 1)."""
    a = 1.0 - gamma
    u = rng.random(n)
    return (lo ** a + u * (hi ** a - lo ** a)) ** (1.0 / a)


def _largest_remainder(p, N):
    raw = p * N
    base = np.floor(raw).astype(np.int64)
    short = N - int(base.sum())
    if short > 0:
        order = np.argsort(-(raw - base), kind="stable")
        base[order[:short]] += 1
    return base


def block_sizes(rng, N, B, dirichlet_alpha=None):
    """Sizes of B non-empty blocks summing to N."""
    if B > N:
        raise ValueError("more blocks than nodes")
    if dirichlet_alpha is None:
        p = np.full(B, 1.0 / B)
    else:
        p = rng.dirichlet(np.full(B, float(dirichlet_alpha)))
    sizes = _largest_remainder(p, N)
    while (sizes == 0).any():  # give every empty block one node from the largest
        k = int(np.argmin(sizes))
        j = int(np.argmax(sizes))
        sizes[k] += 1
        sizes[j] -= 1
    return sizes


def dcsbm(N, B, mean_deg, gamma, ratio, seed=0, dirichlet_alpha=None, order="random",
          theta_range=(1.0, 100.0), intra_fraction=None):
    """Draw one DC-SBM graph (see the module docstring). With intra_fraction, `ratio` is ignored
    and the per-pair ratio r is solved from the drawn block masses Tb so that the expected share
    of within-block edge draws is intra_fraction: r sum Tb^2 / (r sum Tb^2 + Ttot^2 - sum Tb^2)."""
    rng = np.random.default_rng(seed)
    sizes = block_sizes(rng, N, B, dirichlet_alpha)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    blk = np.repeat(np.arange(B), sizes)  # internal order: block-contiguous
    th = powerlaw_propensities(rng, N, gamma, *theta_range)
    cum = np.concatenate([[0.0], np.cumsum(th)])
    Tb = cum[starts[1:]] - cum[starts[:-1]]
    Ttot = cum[-1]
    M = int(round(N * mean_deg / 2.0))
    if intra_fraction is not None:
        S2 = float((Tb * Tb).sum())
        f = float(intra_fraction)
        ratio = f * (Ttot * Ttot - S2) / ((1.0 - f) * S2)

    # u with weight theta_u * (ratio*Tb + Ttot - Tb)
    wu = th * (ratio * Tb[blk] + Ttot - Tb[blk])
    cw = np.cumsum(wu)
    u = np.searchsorted(cw, rng.random(M) * cw[-1], side="right")
    u = np.minimum(u, N - 1)
    bu = blk[u]
    p_in = ratio * Tb[bu] / (ratio * Tb[bu] + Ttot - Tb[bu])
    intra = rng.random(M) < p_in
    x = rng.random(M)
    s0 = cum[starts[bu]]
    s1 = cum[starts[bu + 1]]
    # intra: a point in [cum[start_b], cum[end_b]); inter: a point in the rest
    y_in = s0 + x * (s1 - s0)
    y_out = x * (Ttot - Tb[bu])
    y_out = np.where(y_out >= s0, y_out + Tb[bu], y_out)
    y = np.where(intra, y_in, y_out)
    v = np.searchsorted(cum, y, side="right") - 1
    v = np.clip(v, 0, N - 1)
    lo_b = starts[bu]
    hi_b = starts[bu + 1] - 1
    v = np.where(intra, np.clip(v, lo_b, hi_b), v)  # rounding at a block edge

    if order == "random":
        label = rng.permutation(N)
    elif order == "block_degree":
        drawn = np.bincount(u, minlength=N) + np.bincount(v, minlength=N)
        # block-major, then decreasing drawn degree, then internal index
        idx = np.lexsort((np.arange(N), -drawn, blk))
        label = np.empty(N, dtype=np.int64)
        label[idx] = np.arange(N)
    elif order == "internal":
        label = np.arange(N)
    else:
        raise ValueError(order)
    src = label[u].astype(np.int32)
    dst = label[v].astype(np.int32)
    blocks = np.empty(N, dtype=np.int32)
    blocks[label] = blk
    theta_l = np.empty(N)
    theta_l[label] = th
    params = dict(N=N, B=B, mean_deg=mean_deg, gamma=gamma, ratio=float(ratio),
                  dirichlet_alpha=dirichlet_alpha, order=order, intra_fraction=intra_fraction)
    return DCSBM(src, dst, N, blocks, theta_l, seed, params)


# Blocks of the paper's benchmark graphs per N (Table I) and InfraredGP's settings (tau, L, d)
# per N (Table II), static and streaming.
TABLE1_BLOCKS = {5_000: 19, 10_000: 25, 50_000: 44, 100_000: 56, 500_000: 98, 1_000_000: 125}
TABLE2_STATIC = {5_000: (-6.0, 10, 64), 10_000: (-3.0, 9, 64), 50_000: (-80.0, 40, 32),
                 100_000: (-80.0, 60, 32), 500_000: (-80.0, 70, 32), 1_000_000: (-80.0, 60, 32)}
TABLE2_STREAMING = {100_000: (-100.0, 20, 32), 1_000_000: (-100.0, 20, 16)}


def challenge_like(N, K=None, seed=0, mean_deg=40.0, count_ratio=2.5, dirichlet_alpha=2.0):
    """A DC-SBM shaped like the benchmark graphs of the paper's experiments (Sec. IV-A, Table I):
    K blocks (Table I's count for N by default) of Dirichlet(2) sizes, mean degree 40, degree
    propensities from a power law of exponent 1.5 on [1, 12] (degrees roughly 10-140 around the
    mean, like Table I's spread), and about count_ratio within-block edges per between-block edge
    (the benchmark's 2.5), i.e. an expected within-block share of edge draws of
    count_ratio / (count_ratio + 1)."""
    if K is None:
        K = TABLE1_BLOCKS.get(N, max(2, int(round(N ** 0.4))))
    return dcsbm(N, K, mean_deg, 1.5, 1.0, seed=seed, dirichlet_alpha=dirichlet_alpha, theta_range=(1.0, 12.0),
                 intra_fraction=count_ratio / (count_ratio + 1.0))


def gaussian_input(seed, N, d, x_scale=None):
    """A seeded N x d fp64 Gaussian matrix, N(0, 1) times x_scale (1/sqrt(d) by default: the
    N(0, 1/d) random input of Alg. 1), drawn on the host with numpy's PCG64. Tests feed it to the
    GPU (as igp_embed_opts.x_in, in the storage type) and to the oracle alike, so that both start
    from the same values."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), int(N), int(d), 0x7E7A]))
    xs = 1.0 / np.sqrt(d) if x_scale is None else float(x_scale)
    return rng.standard_normal((N, d)) * xs


def log_uniform_sizes(rng, n, lo, hi):
    """n integers log-uniform on [lo, hi]."""
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n)).round().astype(np.int64)


def batch_dcsbm(G, n_lo, n_hi, deg_lo, deg_hi, gamma, ratio, seed=0, block_exp=0.4):
    """G independent graphs: N log-uniform on [n_lo, n_hi], blocks = round(N^block_exp),
    mean degree uniform on [deg_lo, deg_hi]; graph g uses SeedSequence(seed).spawn(G)[g]."""
    return [batch_dcsbm_one(G, n_lo, n_hi, deg_lo, deg_hi, gamma, ratio, g, seed, block_exp) for g in range(G)]


def batch_dcsbm_one(G, n_lo, n_hi, deg_lo, deg_hi, gamma, ratio, k, seed=0, block_exp=0.4):
    """Graph k of batch_dcsbm(G, ...), drawn alone (the same graph)."""
    ss = np.random.SeedSequence(seed)
    rng = np.random.default_rng(ss)
    Ns = log_uniform_sizes(rng, G, n_lo, n_hi)
    degs = rng.uniform(deg_lo, deg_hi, size=G)
    kid = ss.spawn(G)[k]
    N = int(Ns[k])
    B = max(1, int(round(N ** block_exp)))
    return dcsbm(N, B, float(degs[k]), gamma, ratio, seed=kid)


def split_increments(graph, T=10, mode="random", seed=0, return_order=False):
    """Cut a drawn graph into T edge increments.

    mode="random": edges in a uniformly random order, T equal slices; every
    slice carries the full node count N.
    mode="snowball": nodes ordered by breadth-first search from a random start
    (unreached nodes appended in random order), split into T equal node groups
    V_1..V_T (the snowball model of Sec. II); increment t holds the edges whose
    later-visited endpoint lies in V_t, and node ids are relabelled to the visit
    order so that the nodes present after step t are 0..N_t-1.
    Returns a list of (src, dst, N_t); with return_order, also the node order (order[new id] =
    id in the drawn graph; the identity for mode="random").
    """
    rng = np.random.default_rng(seed)
    src = graph.src.astype(np.int64)
    dst = graph.dst.astype(np.int64)
    N = graph.N
    if mode == "random":
        perm = rng.permutation(src.size)
        cuts = np.linspace(0, src.size, T + 1).round().astype(np.int64)
        incs = [(src[perm[a:b]].astype(np.int32), dst[perm[a:b]].astype(np.int32), N)
                for a, b in zip(cuts[:-1], cuts[1:])]
        return (incs, np.arange(N)) if return_order else incs
    if mode != "snowball":
        raise ValueError(mode)
    # breadth-first visit order; a component not reached from the start is entered at its
    # first node in a random node order once everything reachable has been visited
    import scipy.sparse as sp
    from scipy.sparse.csgraph import breadth_first_order, connected_components
    keep = src != dst
    adj = sp.csr_matrix((np.ones(int(keep.sum()), dtype=np.int8), (src[keep], dst[keep])), shape=(N, N))
    ncomp, comp = connected_components(adj, directed=False)
    sizes = np.bincount(comp, minlength=ncomp)
    start = int(rng.integers(N))
    rest = rng.permutation(N)
    entries = [start]
    seen = np.zeros(ncomp, dtype=bool)
    seen[comp[start]] = True
    for b_ in rest[np.sort(np.unique(comp[rest], return_index=True)[1])]:  # each component's first node
        if not seen[comp[b_]]:
            seen[comp[b_]] = True
            entries.append(int(b_))
    parts = []
    for e in entries:
        parts.append(np.array([e]) if sizes[comp[e]] == 1 else
                     breadth_first_order(adj, e, directed=False, return_predecessors=False))
    order = np.concatenate(parts).astype(np.int64)
    visit = np.empty(N, dtype=np.int64)
    visit[order] = np.arange(N)
    pos = visit  # relabel: node -> visit position
    su, sv = pos[src], pos[dst]
    later = np.maximum(su, sv)
    bounds = np.linspace(0, N, T + 1).round().astype(np.int64)
    step = np.searchsorted(bounds[1:], later, side="right")
    out = []
    for t in range(T):
        m = step == t
        out.append((su[m].astype(np.int32), sv[m].astype(np.int32), int(bounds[t + 1])))
    return (out, order) if return_order else out


# ---------------------------------------------------------------------------
# Named workloads (graph recipe + FFP settings). tau, L, d follow the paper's
# settings where it fixes them (Table II gives tau < 0, L ~ 10, d in {16..64}).
# ---------------------------------------------------------------------------
WORKLOADS = {
    # 1,000 nodes, 11 equal blocks, mean degree 20, gamma 2.5, per-pair ratio 10
    "dcsbm-1k": dict(graph=dict(N=1000, B=11, mean_deg=20, gamma=2.5, ratio=10, seed=0),
                     d=32, tau=-0.5, L=10, storage="f32"),
    # 200,000 nodes, 64 Dirichlet(2) blocks, mean degree 25, gamma 2.5, ratio 4
    "dcsbm-200k": dict(graph=dict(N=200_000, B=64, mean_deg=25, gamma=2.5, ratio=4, seed=0, dirichlet_alpha=2.0),
                       d=64, tau=-0.5, L=10, storage="f32"),
    # 2,000,000 nodes, 128 Dirichlet(5) blocks, mean degree 40, gamma 2.2, ratio 6,
    # node ids ordered block-major then by decreasing degree
    "dcsbm-2m": dict(graph=dict(N=2_000_000, B=128, mean_deg=40, gamma=2.2, ratio=6, seed=0, dirichlet_alpha=5.0,
                                order="block_degree"),
                     d=64, tau=-0.5, L=10, storage="bf16"),
}


# 512 independent graphs, N log-uniform on [1,000, 50,000], blocks round(N^0.4), mean degree
# uniform on [10, 40], gamma 2.5, ratio 5 (embedded together as one batch)
BATCH_WORKLOADS = {
    "dcsbm-batch512": dict(batch=dict(G=512, n_lo=1000, n_hi=50000, deg_lo=10, deg_hi=40, gamma=2.5, ratio=5,
                                      seed=0),
                           d=64, tau=-0.5, L=10, storage="bf16"),
}


def workload_graph(name):
    return dcsbm(**WORKLOADS[name]["graph"])


def workload_batch(name):
    b = BATCH_WORKLOADS[name]["batch"]
    return batch_dcsbm(b["G"], b["n_lo"], b["n_hi"], b["deg_lo"], b["deg_hi"], b["gamma"], b["ratio"], seed=b["seed"])


def workload_batch_graph(name, k):
    """Graph k of a batch workload, drawn alone."""
    b = BATCH_WORKLOADS[name]["batch"]
    return batch_dcsbm_one(b["G"], b["n_lo"], b["n_hi"], b["deg_lo"], b["deg_hi"], b["gamma"], b["ratio"], k,
                           seed=b["seed"])


def workload_batch_sizes(name):
    """Node counts of every graph of a batch workload (without drawing the graphs)."""
    b = BATCH_WORKLOADS[name]["batch"]
    rng = np.random.default_rng(np.random.SeedSequence(b["seed"]))
    return log_uniform_sizes(rng, b["G"], b["n_lo"], b["n_hi"])


# A served stream: G graphs, N log-uniform on [5,000, 1,000,000], blocks round(N^0.4), mean
# degree 25, gamma 2.5, ratio 5; each graph arrives as T = 10 equal edge increments (even
# graphs in uniformly random edge order, odd graphs in snowball order); requests arrive as a
# Poisson process of the given rate, each the next increment of a uniformly chosen graph
# that still has increments left.
SERVE_WORKLOADS = {
    "dcsbm-serve": dict(stream=dict(G=32, n_lo=5000, n_hi=1_000_000, mean_deg=25, gamma=2.5, ratio=5, T=10,
                                    rate=200.0, seed=0),
                        d=64, tau=-0.5, L=10, storage="bf16"),
}


# Alg. 2 on a graph shaped like the paper's benchmark graphs: 10 snowball increments of a
# 100,000-node graph, Table II's streaming setting for N = 100K (tau = -100, L = 20, d = 32),
# the device clusterer with threshold 1.0 in batches of 1,024.
STREAM_WORKLOADS = {
    "challenge-stream-100k": dict(N=100_000, T=10, seed=5, tau=-100.0, L=20, d=32, storage="f32", threshold=1.0,
                                  batch=1024),
}


# The clusterer on the FFP output of a graph shaped like the paper's 1M-node benchmark graphs, at
# Table II's static setting for N = 1M (tau = -80, L = 60, d = 32); threshold 1.0, batches of 4,096.
CLUSTER_WORKLOADS = {
    "challenge-cluster-1m": dict(N=1_000_000, seed=4, tau=-80.0, L=60, d=32, storage="f32", threshold=1.0,
                                 batch=4096),
}


def serve_graph(params, k):
    """Increments of graph k of a served stream: list of (src, dst, N_t)."""
    ss = np.random.SeedSequence(params["seed"])
    rng = np.random.default_rng(ss)
    Ns = log_uniform_sizes(rng, params["G"], params["n_lo"], params["n_hi"])
    kid = ss.spawn(params["G"])[k]
    N = int(Ns[k])
    g = dcsbm(N, max(1, int(round(N ** 0.4))), params["mean_deg"], params["gamma"], params["ratio"], seed=kid)
    mode = "random" if k % 2 == 0 else "snowball"
    return split_increments(g, params["T"], mode, seed=int(kid.generate_state(1)[0]))


def serve_schedule(params):
    """Arrival times (s, from 0) and the (graph, increment) each request carries."""
    rng = np.random.default_rng(np.random.SeedSequence([params["seed"], 1]))
    G, T = params["G"], params["T"]
    R = G * T
    times = np.cumsum(rng.exponential(1.0 / params["rate"], size=R))
    times -= times[0]
    left = [T] * G
    live = list(range(G))
    order = []
    for _ in range(R):
        k = live[int(rng.integers(len(live)))]
        order.append((k, T - left[k]))
        left[k] -= 1
        if left[k] == 0:
            live.remove(k)
    return times, order
