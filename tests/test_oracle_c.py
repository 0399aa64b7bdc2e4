"""The C version of the FP64 oracle (oracle/ffp_ref.c, all host cores) against the pure-Python
brute force and the hand-worked closed forms that pin the numpy oracle, and against the numpy
oracle itself on larger random graphs (two independent implementations of Alg. 1's steps)."""
import math

import numpy as np
import pytest

import oracle
from oracle import cffp
from tests.test_oracle_pins import _brute_force_ffp, _check_znorm_tanh_pattern


@pytest.mark.parametrize("seed,tau,L", [(0, -0.5, 3), (1, -1.5, 4), (2, 0.0, 2), (3, 2.0, 2), (4, -6.0, 5)])
def test_c_oracle_equals_brute_force(seed, tau, L):
    rng = np.random.default_rng(seed)
    N = 25
    src = rng.integers(0, N, 70).tolist()
    dst = rng.integers(0, N, 70).tolist()
    X = rng.standard_normal((N, 8)) / math.sqrt(8)
    ref = np.array(_brute_force_ffp(src, dst, N, X, tau, L))
    rp, col = oracle.build_csr(src, dst, N)
    np.testing.assert_allclose(cffp.ffp(rp, col, X, tau, L), ref, rtol=1e-12, atol=1e-13)


def test_c_oracle_path_graph_closed_form():
    """The hand-worked one-layer case of the numpy oracle's pins: path 0-1-2 at tau = -0.5, X
    chosen so that the layer's pre-activations are (0, ln 2, ln 3), i.e. T = (0, 3/5, 4/5)."""
    theta, alpha = 0.1, 1.0
    a = 2.0 / math.sqrt(3.0)
    B = np.array([[theta, alpha * a, 0.0], [alpha * a, theta, alpha * a], [0.0, alpha * a, theta]])
    x = np.linalg.solve(B, [0.0, math.log(2), math.log(3)])
    X = np.tile(x[:, None], (1, 8))
    rp, col = oracle.build_csr([0, 1], [1, 2], 3)
    _check_znorm_tanh_pattern(cffp.ffp(rp, col, X, -0.5, 1, alpha=alpha, theta=theta))


@pytest.mark.parametrize("tau,alpha,theta,ddof", [(-0.5, 1.0, 0.1, 1), (0.0, 1.0, 0.1, 0), (3.0, -0.5, 0.7, 1),
                                                  (-80.0, 1.0, 0.1, 1)])
def test_c_oracle_equals_numpy_oracle(tau, alpha, theta, ddof):
    rng = np.random.default_rng(7)
    N = 3000
    src = rng.integers(0, N, 20000)
    dst = rng.integers(0, N, 20000)
    rp, col = oracle.build_csr(src, dst, N + 5)  # five isolated nodes
    X = rng.standard_normal((N + 5, 16)) / 4
    ref = oracle.ffp(rp, col, X, tau, 6, alpha=alpha, theta=theta, ddof=ddof)
    for threads in (1, 0):
        got = cffp.ffp(rp, col, X, tau, 6, alpha=alpha, theta=theta, ddof=ddof, nthreads=threads)
        np.testing.assert_allclose(got, ref, rtol=1e-9, atol=1e-12)


def test_c_oracle_result_does_not_depend_on_the_thread_count():
    rng = np.random.default_rng(8)
    N = 20000
    rp, col = oracle.build_csr(rng.integers(0, N, 100000), rng.integers(0, N, 100000), N)
    X = rng.standard_normal((N, 8))
    a = cffp.ffp(rp, col, X, -0.5, 4, nthreads=1)
    b = cffp.ffp(rp, col, X, -0.5, 4, nthreads=max(2, cffp.threads()))
    assert np.array_equal(a, b)
