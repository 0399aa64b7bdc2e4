"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test checks the oracle against something the paper or mathematics fixes:
values printed in the paper, closed forms worked by hand, identities between
two formulations (spectral vs spatial), invariants, independent library
routines, and brute force on tiny inputs.
"""
import math
import os
import statistics

import numpy as np
import pytest

import oracle
from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v = line.split()
            vals[k] = float(v)
    return vals


# ---------------------------------------------------------------------------
# Philox4x64-10 and the Gaussian input (the random input of Alg. 1)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("ctr,key", [
    ([0, 0, 0, 0], [0, 0]),
    ([5, 7, 0, 0], [123, 456]),
    ([2**64 - 2, 3, 9, 11], [2**63 + 17, 99]),
    ([12345678901234, 0, 0, 0], [0xDEADBEEFCAFEF00D, 0]),
])
def test_philox_matches_numpy_bitgenerator(ctr, key):
    # numpy's Philox bit generator increments its counter before each block,
    # so its first four raw outputs are Philox4x64-10(counter + 1, key).
    bg = np.random.Philox(counter=np.array(ctr, dtype=np.uint64), key=np.array(key, dtype=np.uint64))
    ref = bg.random_raw(4)
    c = list(ctr)
    c[0] = (c[0] + 1) % 2**64
    if c[0] == 0:
        c[1] += 1
    got = philox.philox4x64_10(np.array(c, dtype=np.uint64), np.array(key, dtype=np.uint64))
    assert [int(x) for x in got] == [int(x) for x in ref]


def test_philox_vectorised_equals_scalar():
    ctr = np.array([[i, j, 0, 0] for i in range(5) for j in range(3)], dtype=np.uint64)
    key = np.array([42, 0], dtype=np.uint64)
    vec = philox.philox4x64_10(ctr, key)
    for r in range(ctr.shape[0]):
        assert np.array_equal(vec[r], philox.philox4x64_10(ctr[r], key))


def test_uniform_map_closed_form():
    words = np.array([[0, 0xFFFFFFFF << 32 | 0x100, 0xFFFFFFFFFFFFFFFF, 0x00000000000000FF]], dtype=np.uint64)
    u = philox.uniforms_from_words(words)[0]
    # low half first, then high half of each 64-bit word
    assert u[0] == 2.0 ** -24 and u[1] == 2.0 ** -24
    assert u[2] == 2 * 2.0 ** -24  # 0x100 >> 8 = 1
    assert u[3] == 1.0              # 0xFFFFFFFF -> (2^24 - 1 + 1) * 2^-24
    assert u[4] == 1.0 and u[5] == 1.0
    assert u[6] == 2.0 ** -24       # 0xFF >> 8 = 0
    assert np.all(u > 0) and np.all(u <= 1)


def test_box_muller_closed_form():
    a = math.exp(-0.5)  # r = sqrt(-2 ln a) = 1
    u = np.array([a, 0.25, a, 0.5, 1.0, 0.3, a, 1.0])
    z = philox.box_muller(u)
    np.testing.assert_allclose(z[:2], [0.0, 1.0], atol=1e-15)    # angle pi/2
    np.testing.assert_allclose(z[2:4], [-1.0, 0.0], atol=1e-15)  # angle pi
    np.testing.assert_allclose(z[4:6], [0.0, 0.0], atol=1e-15)   # r = 0
    np.testing.assert_allclose(z[6:8], [1.0, 0.0], atol=1e-15)   # angle 2 pi


def test_theta_is_gaussian_with_variance_one_over_d():
    from scipy import stats
    d = 32
    X = oracle.theta_input(7, 4096, d)
    assert X.shape == (4096, d)
    flat = X.ravel() * math.sqrt(d)
    assert abs(flat.mean()) < 0.01
    assert abs(flat.var() - 1.0) < 0.02
    assert stats.kstest(flat, "norm").pvalue > 1e-3
    # columns uncorrelated
    C = np.corrcoef(X.T)
    assert np.max(np.abs(C - np.eye(d))) < 0.08


def test_theta_rows_depend_only_on_seed_and_row():
    big = oracle.theta_input(3, 100, 16)
    part = oracle.theta_input(3, 40, 16, row0=60)
    assert np.array_equal(big[60:], part)
    other = oracle.theta_input(4, 100, 16)
    assert not np.allclose(big, other)
    with pytest.raises(ValueError):
        oracle.theta_input(0, 4, 12)


# ---------------------------------------------------------------------------
# CSR (Sec. II: symmetric binary simple adjacency) -- brute force
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("seed", range(5))
def test_csr_equals_brute_force_sets(seed):
    rng = np.random.default_rng(seed)
    N = int(rng.integers(1, 40))
    M = int(rng.integers(0, 200))
    src = rng.integers(0, N, M)
    dst = rng.integers(0, N, M)
    row_ptr, col = oracle.build_csr(src, dst, N)
    adj = {i: set() for i in range(N)}
    for a, b in zip(src.tolist(), dst.tolist()):
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    assert row_ptr[0] == 0 and row_ptr.size == N + 1
    for i in range(N):
        assert list(col[row_ptr[i]:row_ptr[i + 1]]) == sorted(adj[i])
    assert np.array_equal(oracle.degrees(row_ptr), [len(adj[i]) for i in range(N)])


def test_csr_rejects_bad_ids():
    with pytest.raises(ValueError):
        oracle.build_csr([0, 1], [1, 5], 5)
    with pytest.raises(ValueError):
        oracle.build_csr([-1], [0], 3)


# ---------------------------------------------------------------------------
# Eq. 1 (negative correction) and D_tau = D + tau I (Sec. I)
# ---------------------------------------------------------------------------
def test_degree_correction_closed_forms():
    deg = np.array([0, 1, 2, 5, 40])
    # tau = -1.5, eps = 1e-3: deg - min(1.5, deg - eps)
    # (exact up to the rounding of deg - eps, e.g. 1 - (1 - 1e-3) != 1e-3 in fp64)
    np.testing.assert_allclose(oracle.degree_correction(deg, -1.5), [1e-3, 1e-3, 0.5, 3.5, 38.5], rtol=1e-14)
    # tau = -0.5
    np.testing.assert_allclose(oracle.degree_correction(deg, -0.5), [1e-3, 0.5, 1.5, 4.5, 39.5], rtol=1e-14)
    # tau = 0 and tau > 0 use D + tau I
    np.testing.assert_array_equal(oracle.degree_correction(deg, 0.0), deg)
    np.testing.assert_array_equal(oracle.degree_correction(deg, 2.0), deg + 2.0)
    # for tau < 0 the clamp equals max(deg + tau, eps), up to rounding
    for tau in (-0.3, -1.0, -6.0, -80.0):
        np.testing.assert_allclose(oracle.degree_correction(deg, tau), np.maximum(deg + tau, 1e-3), rtol=1e-14, atol=1e-13)
    dinv = oracle.inv_sqrt_degrees([0.0, 4.0, 1e-3])
    np.testing.assert_array_equal(dinv[:2], [0.0, 0.5])
    assert abs(dinv[2] - 1.0 / math.sqrt(1e-3)) < 1e-12


# ---------------------------------------------------------------------------
# Karate Club (Sec. I, Fig. 1): values printed in the paper
# ---------------------------------------------------------------------------
def _karate_csr():
    nx = pytest.importorskip("networkx")
    G = nx.karate_club_graph()
    e = np.array(list(G.edges()))
    return oracle.build_csr(e[:, 0], e[:, 1], G.number_of_nodes())


def test_karate_laplacian_matches_paper_values():
    gold = _golden("karate_tau0.txt")
    row_ptr, col = _karate_csr()
    assert row_ptr.size - 1 == gold["N"]
    L = oracle.corrected_laplacian(oracle.dense_adjacency(row_ptr, col), 0.0)
    lam, U = np.linalg.eigh(L)
    tol = gold["print_precision"]
    assert abs(lam[0] - gold["lambda_min"]) < 1e-10
    assert lam[-1] <= gold["lambda_max_upper"] + 1e-12
    assert np.all(U[:, 0] > 0) or np.all(U[:, 0] < 0)
    u33 = U[:, 33]
    sign = np.sign(u33[33]) * np.sign(gold["u33_node34"])  # eigenvector sign is arbitrary
    assert abs(sign * u33[33] - gold["u33_node34"]) < tol
    assert abs(sign * u33[22] - gold["u33_node23"]) < tol


def test_karate_spectrum_vs_tau_as_in_fig1():
    row_ptr, col = _karate_csr()
    A = oracle.dense_adjacency(row_ptr, col)
    lam0 = np.linalg.eigvalsh(oracle.corrected_laplacian(A, 0.0))
    # tau < 0 (Fig. 1 d, e): frequencies leave [0, 2] on both sides
    for tau in (-1.0, -1.5):
        lam = np.linalg.eigvalsh(oracle.corrected_laplacian(A, tau))
        assert lam.min() < 0 and lam.max() > 2
    # tau > 0 (Fig. 1 g, h): inside [0, 2] and pulled towards 1 as tau grows
    w_prev = lam0.max() - lam0.min()
    for tau in (5.0, 10.0):
        lam = np.linalg.eigvalsh(oracle.corrected_laplacian(A, tau))
        assert lam.min() >= 0 and lam.max() <= 2
        assert lam.max() - lam.min() < w_prev
        w_prev = lam.max() - lam.min()
        # Theorem 1 applied to I - D_tau^{-1} A (similar to L_tau): |lam - 1| <= max deg/(deg+tau)
        deg = A.sum(1)
        assert np.max(np.abs(lam - 1)) <= np.max(deg / (deg + tau)) + 1e-12


@pytest.mark.parametrize("tau", [0.0, -0.5, -1.5, 3.0])
def test_corrected_laplacian_on_sqrt_degree_vector(tau):
    rng = np.random.default_rng(1)
    N = 30
    A = np.triu((rng.random((N, N)) < 0.15).astype(float), 1)
    A = A + A.T
    A[0, :] = A[:, 0] = 0  # an isolated node
    A[1, :] = A[:, 1] = 0
    A[1, 2] = A[2, 1] = 1  # a degree-1 node
    L = oracle.corrected_laplacian(A, tau)
    deg = A.sum(1)
    Dt = oracle.degree_correction(deg, tau)
    v = np.sqrt(Dt)
    # (L_tau D_tau^{1/2} 1)_i = (Dtau_i - deg_i) / sqrt(Dtau_i), zero at tau = 0
    expect = np.where(Dt > 0, (Dt - deg) / np.where(Dt > 0, v, 1), 0)
    np.testing.assert_allclose(L @ v, expect, atol=1e-11)
    if tau < 0:  # Rayleigh quotient of v is negative: infrared frequencies exist
        assert np.linalg.eigvalsh(L).min() < 0


# ---------------------------------------------------------------------------
# Eq. 3: spectral form U phi(Lambda) U^T Z equals the spatial form
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("tau", [-1.5, -0.5, 0.0, 3.0])
@pytest.mark.parametrize("alpha,theta", [(1.0, 0.1), (-0.5, 0.7), (0.3, 0.0)])
def test_eq3_spectral_equals_spatial(tau, alpha, theta):
    rng = np.random.default_rng(2)
    N, d = 40, 8
    src = rng.integers(0, N, 120)
    dst = rng.integers(0, N, 120)
    row_ptr, col = oracle.build_csr(src, dst, N)
    A = oracle.dense_adjacency(row_ptr, col)
    Lt = oracle.corrected_laplacian(A, tau)
    lam, U = np.linalg.eigh(Lt)
    phi = (theta + alpha) - alpha * lam               # Eq. 2
    Z = rng.standard_normal((N, d))
    spectral = U @ (phi[:, None] * (U.T @ Z))         # graph convolution, Sec. II
    dinv = oracle.inv_sqrt_degrees(oracle.degree_correction(oracle.degrees(row_ptr), tau))
    spatial = oracle.conv(oracle.normalized_adjacency(row_ptr, col, dinv), Z, alpha, theta)
    np.testing.assert_allclose(spatial, spectral, atol=1e-10)


@pytest.mark.parametrize("tau", [0.0, 2.5, -1.5, -10.0])
def test_regular_graph_normalized_adjacency_of_ones(tau):
    """On a d-regular graph every D_tau is the same number c (Eq. 1: d + tau for tau >= 0, and
    d - min(|tau|, d - eps) for tau < 0), so D_tau^{-1/2} A D_tau^{-1/2} 1 = (d / c) 1."""
    N, offs = 30, (1, 2, 5)  # circulant: node i joined to i +- 1, 2, 5, so d = 6
    src = np.array([i for i in range(N) for _ in offs])
    dst = np.array([(i + o) % N for i in range(N) for o in offs])
    row_ptr, col = oracle.build_csr(src, dst, N)
    d = 2 * len(offs)
    assert np.all(np.diff(row_ptr) == d)
    c = d + tau if tau >= 0 else d - min(abs(tau), d - 1e-3)
    dinv = oracle.inv_sqrt_degrees(oracle.degree_correction(oracle.degrees(row_ptr), tau))
    Ahat = oracle.normalized_adjacency(row_ptr, col, dinv)
    np.testing.assert_allclose(Ahat @ np.ones(N), np.full(N, d / c), rtol=1e-14)


@pytest.mark.parametrize("tau", [-1.5, -0.5, 0.0, 3.0])
def test_ffp_through_the_spectral_form_equals_the_oracle(tau):
    """Alg. 1 written with the spectral form of Eq. 3 at every layer (an eigendecomposition of
    L_tau, the filter of Eq. 2 on its eigenvalues), numpy's column mean and sample standard
    deviation for ZNorm and scipy's logistic function for the output, against the oracle's
    spatial FFP: the assembly of Eq. 4's steps must agree, not only one convolution."""
    from scipy.special import expit
    rng = np.random.default_rng(5)
    N, d, L, alpha, theta = 36, 6, 4, 1.0, 0.1
    src = rng.integers(0, N, 110)
    dst = rng.integers(0, N, 110)
    row_ptr, col = oracle.build_csr(src, dst, N)
    lam, U = np.linalg.eigh(oracle.corrected_laplacian(oracle.dense_adjacency(row_ptr, col), tau))
    phi = (theta + alpha) - alpha * lam
    X = rng.standard_normal((N, d)) / math.sqrt(d)
    Z = X
    for _ in range(L):
        T = np.tanh(U @ (phi[:, None] * (U.T @ Z)))
        Z = (T - T.mean(axis=0)) / T.std(axis=0, ddof=1)
    np.testing.assert_allclose(oracle.ffp(row_ptr, col, X, tau, L), expit(Z), atol=1e-11)


# ---------------------------------------------------------------------------
# Eq. 4 and Alg. 1 on hand-worked cases
# ---------------------------------------------------------------------------
def _logit(p):
    return np.log(p) - np.log1p(-p)


def _check_znorm_tanh_pattern(out):
    """logit(out) = Z^(L): columns of mean 0 and sample std 1; rows follow
    tanh(0) = 0, tanh(ln 2) = 3/5, tanh(ln 3) = 4/5, so (z_2 - z_0)/(z_1 - z_0) = 4/3."""
    z = _logit(out)
    np.testing.assert_allclose(z.mean(0), 0, atol=1e-12)
    np.testing.assert_allclose(z.std(0, ddof=1), 1, atol=1e-12)
    np.testing.assert_allclose((z[2] - z[0]) / (z[1] - z[0]), 4.0 / 3.0, rtol=1e-12)


def test_one_layer_edgeless_graph_closed_form():
    # no edges: every node has D_tau = eps, A = 0, so phi * Z = theta Z
    theta = 0.1
    X = np.tile(np.array([[0.0], [math.log(2) / theta], [math.log(3) / theta]]), (1, 8))
    out = oracle.ffp(np.zeros(4, dtype=np.int64), np.zeros(0, dtype=np.int64), X, -0.5, 1)
    _check_znorm_tanh_pattern(out)


def test_one_layer_path_graph_closed_form():
    # path 0-1-2 at tau = -0.5: deg = (1, 2, 1), Eq. 1 gives D_tau = (0.5, 1.5, 0.5),
    # so Ahat_01 = Ahat_12 = (0.5 * 1.5)^{-1/2} = 2/sqrt(3). Choose X so that
    # theta X + alpha Ahat X = (0, ln 2, ln 3) in every column.
    theta, alpha = 0.1, 1.0
    a = 2.0 / math.sqrt(3.0)
    B = np.array([[theta, alpha * a, 0.0], [alpha * a, theta, alpha * a], [0.0, alpha * a, theta]])
    x = np.linalg.solve(B, [0.0, math.log(2), math.log(3)])
    X = np.tile(x[:, None], (1, 8))
    row_ptr, col = oracle.build_csr([0, 1], [1, 2], 3)
    _check_znorm_tanh_pattern(oracle.ffp(row_ptr, col, X, -0.5, 1, alpha=alpha, theta=theta))
    # the same with a high-pass filter (alpha < 0) and another theta
    theta, alpha = 0.7, -0.5
    B = np.array([[theta, alpha * a, 0.0], [alpha * a, theta, alpha * a], [0.0, alpha * a, theta]])
    x = np.linalg.solve(B, [0.0, math.log(2), math.log(3)])
    X = np.tile(x[:, None], (1, 8))
    _check_znorm_tanh_pattern(oracle.ffp(row_ptr, col, X, -0.5, 1, alpha=alpha, theta=theta))


def test_zero_layers_is_sigmoid_of_input():
    X = np.random.default_rng(0).standard_normal((5, 8))
    out = oracle.ffp(np.array([0, 1, 2, 2, 2, 2]), np.array([1, 0]), X, -0.5, 0)
    np.testing.assert_allclose(_logit(out), X, atol=1e-12)


def test_constant_column_maps_to_zero():
    X = np.zeros((4, 8))
    X[:, 1] = [1, 2, 3, 4]
    out = oracle.ffp(np.zeros(5, dtype=np.int64), np.zeros(0, dtype=np.int64), X, -0.5, 1)
    np.testing.assert_array_equal(out[:, 0], 0.5)  # sigma(0)
    assert np.all(out[:, 1] != 0.5)


def test_row_l2_option():
    rng = np.random.default_rng(3)
    row_ptr, col = oracle.build_csr(rng.integers(0, 20, 60), rng.integers(0, 20, 60), 20)
    X = rng.standard_normal((20, 8))
    a = oracle.ffp(row_ptr, col, X, -0.5, 3)
    b = oracle.ffp(row_ptr, col, X, -0.5, 3, out_row_l2=True)
    np.testing.assert_allclose(np.linalg.norm(b, axis=1), 1.0, atol=1e-14)
    np.testing.assert_allclose(b * np.linalg.norm(a, axis=1, keepdims=True), a, atol=1e-14)


def _brute_force_ffp(src, dst, N, X, tau, L, alpha=1.0, theta=0.1, eps=1e-3):
    """Pure-Python loops: adjacency sets, math.tanh, statistics.fmean/stdev, math.exp."""
    adj = [set() for _ in range(N)]
    for a, b in zip(src, dst):
        if a != b:
            adj[a].add(b)
            adj[b].add(a)
    dt = []
    for i in range(N):
        k = len(adj[i])
        if tau < 0:
            dt.append(k - min(abs(tau), k - eps))
        else:
            dt.append(k + tau)
    w = [0.0 if v == 0 else v ** -0.5 for v in dt]
    Z = [list(map(float, row)) for row in X]
    d = len(Z[0])
    for _ in range(L):
        T = [[math.tanh(theta * Z[i][c] + alpha * sum(w[i] * w[j] * Z[j][c] for j in adj[i]))
              for c in range(d)] for i in range(N)]
        Z = [[0.0] * d for _ in range(N)]
        for c in range(d):
            colv = [T[i][c] for i in range(N)]
            m = statistics.fmean(colv)
            s = statistics.stdev(colv)
            for i in range(N):
                Z[i][c] = 0.0 if s == 0 else (T[i][c] - m) / s
    return [[1.0 / (1.0 + math.exp(-Z[i][c])) for c in range(d)] for i in range(N)]


@pytest.mark.parametrize("seed,tau,L", [(0, -0.5, 3), (1, -1.5, 4), (2, 0.0, 2), (3, 2.0, 2), (4, -6.0, 5)])
def test_ffp_equals_brute_force(seed, tau, L):
    rng = np.random.default_rng(seed)
    N = 25
    src = rng.integers(0, N, 70).tolist()
    dst = rng.integers(0, N, 70).tolist()
    X = rng.standard_normal((N, 8)) / math.sqrt(8)
    ref = np.array(_brute_force_ffp(src, dst, N, X, tau, L))
    got = oracle.ffp_from_edges(src, dst, N, X, tau, L)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-13)


def test_ffp_permutation_equivariant():
    rng = np.random.default_rng(5)
    N = 60
    src = rng.integers(0, N, 300)
    dst = rng.integers(0, N, 300)
    X = rng.standard_normal((N, 16))
    base = oracle.ffp_from_edges(src, dst, N, X, -0.5, 6)
    p = rng.permutation(N)  # node i -> p[i]
    Xp = np.empty_like(X)
    Xp[p] = X
    perm = oracle.ffp_from_edges(p[src], p[dst], N, Xp, -0.5, 6)
    np.testing.assert_allclose(perm[p], base, rtol=1e-12, atol=1e-13)


def test_ddof_option_changes_scale():
    rng = np.random.default_rng(6)
    T = rng.standard_normal((5, 8))
    z1, _, s1 = oracle.znorm(T, 1)
    z0, _, s0 = oracle.znorm(T, 0)
    np.testing.assert_allclose(s1, T.std(0, ddof=1))
    np.testing.assert_allclose(s0, T.std(0, ddof=0))
    np.testing.assert_allclose(z0, z1 * math.sqrt(5 / 4))


# ---------------------------------------------------------------------------
# BF16 storage emulation: against torch's own conversion
# ---------------------------------------------------------------------------
def test_round_bf16_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(5000), [1 + 2 ** -8, 1 + 3 * 2 ** -8, -0.0, 3.0e38, 1e-40]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.round_bf16(x), ref)
    assert oracle.round_bf16(1 + 2 ** -8) == 1.0            # tie to even
    assert oracle.round_bf16(1 + 3 * 2 ** -8) == 1 + 2 ** -6


def test_bf16_storage_mode_rounds_layer_outputs():
    rng = np.random.default_rng(7)
    N = 50
    row_ptr, col = oracle.build_csr(rng.integers(0, N, 200), rng.integers(0, N, 200), N)
    X = rng.standard_normal((N, 8)) / math.sqrt(8)
    a = oracle.ffp(row_ptr, col, X, -0.5, 4)
    b = oracle.ffp(row_ptr, col, X, -0.5, 4, storage="bf16")
    err = np.max(np.linalg.norm(a - b, axis=1) / np.linalg.norm(a, axis=1))
    assert 0 < err < 2e-2


# ---------------------------------------------------------------------------
# Alg. 2 cumulative snapshots
# ---------------------------------------------------------------------------
def test_stream_snapshots_match_static_rebuild():
    rng = np.random.default_rng(8)
    incs = []
    n = 0
    all_s, all_d = [], []
    for t in range(4):
        n += 10
        s = rng.integers(0, n, 30)
        d = rng.integers(0, n, 30)
        incs.append((s, d, n))
        all_s.append(s)
        all_d.append(d)
    snaps = list(oracle.stream_snapshots(incs))
    rp, cl = oracle.build_csr(np.concatenate(all_s), np.concatenate(all_d), n)
    assert np.array_equal(snaps[-1][0], rp) and np.array_equal(snaps[-1][1], cl)
    assert [s[2] for s in snaps] == [10, 20, 30, 40]
