"""Plain FP64 reference of InfraredGP's feed-forward propagation (FFP).

TEST INFRASTRUCTURE ONLY (see the package docstring). Slow on purpose: every
step is the paper's definition written out, in the paper's order, with numpy
and scipy.sparse primitives (sort/unique, sparse-times-dense product, tanh) and
no blocking, fusion or reordering.

What is computed (Qin, Li, Cui, Pei, "InfraredGP", arXiv 2508.19737):
  * A: symmetric binary adjacency of an undirected, unweighted, simple graph
    (Sec. II, problem statement). Self-loops in the input are dropped and
    repeated edges merged.
  * D_tau: degree correction. tau < 0 uses Eq. 1,
        (D_tau)_ii = deg_i - min(|tau|, deg_i - eps),  eps = 1e-3 by default;
    tau >= 0 uses the definition D_tau = D + tau I (Sec. I).
  * Eq. 3 (general (alpha, theta) form of the Eq. 2 filter):
        phi * Z = theta Z + alpha D_tau^{-1/2} A D_tau^{-1/2} Z,
    the paper's low-pass setting being (alpha, theta) = (1, 0.1).
  * Eq. 4: Z^(l) = ZNorm(tanh(phi * Z^(l-1))), l = 1..L, with ZNorm the
    column-wise z-score; output Z~ = sigmoid(Z^(L)). Z^(0) = Theta (Alg. 1).

Readings where the paper is silent (each is an option here and on the GPU):
  * ZNorm's standard deviation uses ddof=1 by default (ddof=0 on request).
    Parity unpinned as to which divisor the authors used: the paper does not
    say, and no printed value decides it (both are pinned against the closed
    forms of their own divisor).
  * A column with zero standard deviation normalises to 0.
  * A node with D_tau == 0 (tau = 0, isolated) gets D_tau^{-1/2} = 0; its row
    of A is empty, so nothing else depends on it.
  * out_row_l2 optionally divides each output row by its L2 norm.
"""
import numpy as np
import scipy.sparse as sp

__all__ = [
    "build_csr", "degrees", "degree_correction", "inv_sqrt_degrees",
    "normalized_adjacency", "conv", "conv_rows", "znorm", "sigmoid", "round_bf16", "bf16_store",
    "ffp", "ffp_from_edges", "stream_snapshots", "dense_adjacency",
    "corrected_laplacian",
]


# ----------------------------------------------------------------------------
# Graph (Sec. II) -> CSR
# ----------------------------------------------------------------------------
def build_csr(src, dst, N):
    """Undirected edge list -> CSR (row_ptr int64[N+1], col int64[nnz]).

    Both directions of every edge are entered, self-loops dropped, duplicates
    merged; columns of each row come out in increasing order. Raises
    ValueError on an id outside [0, N).
    """
    src = np.asarray(src, dtype=np.int64).ravel()
    dst = np.asarray(dst, dtype=np.int64).ravel()
    if src.shape != dst.shape:
        raise ValueError("src and dst differ in length")
    if N <= 0:
        raise ValueError("N must be positive")
    if src.size and (src.min() < 0 or dst.min() < 0 or src.max() >= N or dst.max() >= N):
        raise ValueError("node id outside [0, N)")
    keep = src != dst
    u = np.concatenate([src[keep], dst[keep]])
    v = np.concatenate([dst[keep], src[keep]])
    keys = np.unique(u * np.int64(N) + v)  # sorted by (row, col), duplicates merged
    rows = keys // N
    col = keys % N
    counts = np.bincount(rows, minlength=N)  # row lengths
    row_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    return row_ptr, col


def degrees(row_ptr):
    """deg_i = number of neighbours of node i = row length of A."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    return np.diff(row_ptr)


def degree_correction(deg, tau, eps=1e-3):
    """Diagonal of D_tau in fp64: Eq. 1 for tau < 0, deg + tau otherwise."""
    deg = np.asarray(deg, dtype=np.float64)
    tau = float(tau)
    if tau < 0:
        return deg - np.minimum(abs(tau), deg - eps)
    return deg + tau


def inv_sqrt_degrees(Dtau):
    """D_tau^{-1/2} as a vector (fp64); 0 where D_tau == 0."""
    Dtau = np.asarray(Dtau, dtype=np.float64)
    out = np.zeros_like(Dtau)
    pos = Dtau > 0
    out[pos] = 1.0 / np.sqrt(Dtau[pos])
    return out


def normalized_adjacency(row_ptr, col, dinv):
    """scipy CSR matrix D_tau^{-1/2} A D_tau^{-1/2} (fp64)."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    N = row_ptr.size - 1
    A = sp.csr_matrix((np.ones(col.size), col, row_ptr), shape=(N, N))
    Dm = sp.diags(np.asarray(dinv, dtype=np.float64))
    return (Dm @ A @ Dm).tocsr()


def conv(Ahat, Z, alpha=1.0, theta=0.1):
    """Eq. 3 in its spatial form: theta Z + alpha Ahat Z."""
    return theta * Z + alpha * (Ahat @ Z)


def conv_rows(Ahat, Z, r0, r1, alpha=1.0, theta=0.1):
    """Rows r0..r1-1 of Eq. 3 (the same definition as conv, on a row range)."""
    return theta * Z[r0:r1] + alpha * (Ahat[r0:r1] @ Z)


def znorm(T, ddof=1):
    """Column-wise z-score (Eq. 4): (x - mean(x)) / std(x), two-pass, fp64.

    Returns (Z, mean, std). A column whose std is 0 maps to 0.
    """
    T = np.asarray(T, dtype=np.float64)
    n = T.shape[0]
    mu = T.sum(axis=0) / n
    dev = T - mu
    denom = n - ddof
    var = (dev * dev).sum(axis=0) / denom if denom > 0 else np.zeros(T.shape[1])
    s = np.sqrt(var)
    Z = np.zeros_like(T)
    nz = s > 0
    Z[:, nz] = dev[:, nz] / s[nz]
    return Z, mu, s


def sigmoid(x):
    """sigma(x) = 1 / (1 + e^{-x}) (Eq. 4)."""
    return 1.0 / (1.0 + np.exp(-np.asarray(x, dtype=np.float64)))


def round_bf16(x):
    """Round to the nearest bfloat16 (ties to even) via fp32, returned as fp64.

    Emulates the points where the GPU stores a value in BF16: the value is first
    held in fp32 and then rounded.
    """
    f = np.asarray(x, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ----------------------------------------------------------------------------
# Alg. 1 up to its clustering step
# ----------------------------------------------------------------------------
def bf16_store(a, dinv, layout="row_scaled"):
    """The values read back after rows of `a` (N x d) were stored in BF16.

    layout="row_scaled": row i is held as dinv_i * a_i (a_i where dinv_i = 0),
    so the rounding acts on that product and is undone by the division.
    layout="plain": each value a_ij is rounded on its own.
    """
    if layout == "plain":
        return round_bf16(a)
    sc = np.where(np.asarray(dinv) > 0, dinv, 1.0)[:, None]
    return round_bf16(sc * a) / sc


def ffp(row_ptr, col, X, tau, L, alpha=1.0, theta=0.1, eps=1e-3, ddof=1,
        out_row_l2=False, storage="f64", return_layers=False):
    """One FFP over the graph given in CSR form, on the input X = Theta.

    storage="bf16" rounds to BF16 where the GPU stores in BF16: Theta and each
    layer's tanh output T^(l), in the row-scaled layout of bf16_store; the column
    statistics of a layer are those of its unrounded T^(l). storage="bf16_plain"
    rounds the same values one by one instead (bf16_store's plain layout), a
    second storage of the same precision to compare against. Both only separate
    storage error from bugs; the fp64 result is the contract.
    Returns Z~ (N x d, fp64), plus per-layer (T, mean, std) if asked.
    """
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    N = row_ptr.size - 1
    X = np.asarray(X, dtype=np.float64)
    if X.shape[0] != N:
        raise ValueError("X must have N rows")
    # degree correction: D_tau via Eq. 1, and the normalised adjacency of Eq. 3
    dinv = inv_sqrt_degrees(degree_correction(degrees(row_ptr), tau, eps))
    Ahat = normalized_adjacency(row_ptr, col, dinv)
    if storage in ("bf16", "bf16_plain"):
        layout = "row_scaled" if storage == "bf16" else "plain"
        store = lambda a: bf16_store(a, dinv, layout)  # noqa: E731
    elif storage == "f64":
        store = lambda a: a  # noqa: E731
    else:
        raise ValueError("storage is one of f64, bf16, bf16_plain")
    # random input: Z^(0) = Theta
    Z = store(X)
    layers = []
    # L layers of Eq. 4
    for _ in range(L):
        T = np.tanh(conv(Ahat, Z, alpha, theta))
        _, mu, s = znorm(T, ddof)
        Ts = store(T)
        Z = np.zeros_like(Ts)
        nz = s > 0
        Z[:, nz] = (Ts[:, nz] - mu[nz]) / s[nz]
        if return_layers:
            layers.append((T, mu, s))
    # output: sigmoid of the last ZNorm
    out = sigmoid(Z)
    if out_row_l2:
        out = out / np.linalg.norm(out, axis=1, keepdims=True)
    if return_layers:
        return out, layers
    return out


def ffp_from_edges(src, dst, N, X, tau, L, **kw):
    """build_csr followed by ffp."""
    row_ptr, col = build_csr(src, dst, N)
    return ffp(row_ptr, col, X, tau, L, **kw)


# ----------------------------------------------------------------------------
# Alg. 2 (streaming): the cumulative graph after each increment
# ----------------------------------------------------------------------------
def stream_snapshots(increments):
    """Cumulative topology of Alg. 2 (each step adds its increment to the graph so far).

    increments: list of (src, dst, N_t) with N_t the node count after step t.
    Yields (row_ptr, col, N_t) of the merged graph after each step.
    """
    acc_s, acc_d = [], []
    for s, d, n in increments:
        acc_s.append(np.asarray(s, dtype=np.int64))
        acc_d.append(np.asarray(d, dtype=np.int64))
        row_ptr, col = build_csr(np.concatenate(acc_s), np.concatenate(acc_d), n)
        yield row_ptr, col, n


# ----------------------------------------------------------------------------
# Dense forms used only by the spectral checks (Sec. I, Sec. II)
# ----------------------------------------------------------------------------
def dense_adjacency(row_ptr, col):
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    N = row_ptr.size - 1
    A = np.zeros((N, N))
    for i in range(N):
        A[i, col[row_ptr[i]:row_ptr[i + 1]]] = 1.0
    return A


def corrected_laplacian(A, tau, eps=1e-3):
    """L_tau = I - D_tau^{-1/2} A D_tau^{-1/2} (dense), D_tau as in Eq. 1 / Sec. I."""
    A = np.asarray(A, dtype=np.float64)
    dinv = inv_sqrt_degrees(degree_correction(A.sum(axis=1), tau, eps))
    return np.eye(A.shape[0]) - (dinv[:, None] * A * dinv[None, :])
