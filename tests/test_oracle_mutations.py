"""The oracle pins are not vacuous: plant a plausible mistake in the oracle (on
the CPU, by patching one of its functions) and check that some pin fails."""
import numpy as np
import pytest

import oracle
import oracle.fp64 as off
import oracle.philox as oph
from tests import test_oracle_pins as pins

# pins that take no fixtures/parameters, plus parametrised ones with fixed args
PIN_CALLS = [
    lambda: pins.test_one_layer_edgeless_graph_closed_form(),
    lambda: pins.test_one_layer_path_graph_closed_form(),
    lambda: pins.test_zero_layers_is_sigmoid_of_input(),
    lambda: pins.test_constant_column_maps_to_zero(),
    lambda: pins.test_degree_correction_closed_forms(),
    lambda: pins.test_ffp_equals_brute_force(1, -1.5, 4),
    lambda: pins.test_ffp_equals_brute_force(3, 2.0, 2),
    lambda: pins.test_eq3_spectral_equals_spatial(-1.5, 1.0, 0.1),
    lambda: pins.test_eq3_spectral_equals_spatial(3.0, -0.5, 0.7),
    lambda: pins.test_corrected_laplacian_on_sqrt_degree_vector(-1.5),
    lambda: pins.test_csr_equals_brute_force_sets(0),
    lambda: pins.test_philox_matches_numpy_bitgenerator([5, 7, 0, 0], [123, 456]),
    lambda: pins.test_uniform_map_closed_form(),
    lambda: pins.test_box_muller_closed_form(),
    lambda: pins.test_theta_is_gaussian_with_variance_one_over_d(),
]


def _some_pin_fails():
    for call in PIN_CALLS:
        try:
            call()
        except (AssertionError, ValueError, IndexError):
            return True
    return False


def _mut_dinv_same_side(row_ptr, col, dinv):
    # D^{-1} A instead of D^{-1/2} A D^{-1/2}
    import scipy.sparse as sp
    N = len(row_ptr) - 1
    A = sp.csr_matrix((np.ones(len(col)), col, row_ptr), shape=(N, N))
    return (sp.diags(np.asarray(dinv) ** 2) @ A).tocsr()


def _mut_global_znorm(T, ddof=1):
    # Eq. 4 read as one mean and one std over the whole matrix rather than per column
    T = np.asarray(T, dtype=np.float64)
    mu, sd = T.mean(), T.std(ddof=ddof)
    d = T.shape[1]
    return (T - mu) / sd, np.full(d, mu), np.full(d, sd)


def _mut_clamp_to_zero(deg, tau, eps=1e-3):
    # Eq. 1 without its eps: nodes with deg <= |tau| get D_tau = 0
    deg = np.asarray(deg, dtype=np.float64)
    return deg - np.minimum(abs(tau), deg) if tau < 0 else deg + tau


def _mut_inverse_not_sqrt(Dtau):
    # D_tau^{-1} where D_tau^{-1/2} is meant
    Dtau = np.asarray(Dtau, dtype=np.float64)
    out = np.zeros_like(Dtau)
    out[Dtau > 0] = 1.0 / Dtau[Dtau > 0]
    return out


MUTATIONS = {
    "ZNorm over all entries": ("znorm", _mut_global_znorm),
    "Eq. 1 clamped to 0": ("degree_correction", _mut_clamp_to_zero),
    "D^-1 instead of D^-1/2": ("inv_sqrt_degrees", _mut_inverse_not_sqrt),
    "alpha and theta swapped": ("conv", lambda Ahat, Z, alpha=1.0, theta=0.1: alpha * Z + theta * (Ahat @ Z)),
    "self term dropped": ("conv", lambda Ahat, Z, alpha=1.0, theta=0.1: alpha * (Ahat @ Z)),
    "alpha sign flipped": ("conv", lambda Ahat, Z, alpha=1.0, theta=0.1: theta * Z - alpha * (Ahat @ Z)),
    "tau ignored": ("degree_correction", lambda deg, tau, eps=1e-3: np.asarray(deg, dtype=float)),
    "eps clamp dropped": ("degree_correction", lambda deg, tau, eps=1e-3: np.asarray(deg, dtype=float) + tau),
    "dinv on one side": ("normalized_adjacency", _mut_dinv_same_side),
    "ddof 0": ("znorm", lambda T, ddof=1: off.__dict__["_orig_znorm"](T, 0)),
    "no centring": ("znorm", lambda T, ddof=1: (lambda z, m, s: (T / np.where(s > 0, s, 1), m * 0, s))(*off.__dict__["_orig_znorm"](T, ddof))),
    "sigmoid sign": ("sigmoid", lambda x: 1.0 / (1.0 + np.exp(np.asarray(x, dtype=float)))),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_ffp_mistake_is_caught(monkeypatch, name):
    fn, impl = MUTATIONS[name]
    monkeypatch.setitem(off.__dict__, "_orig_znorm", off.znorm)
    monkeypatch.setattr(off, fn, impl)
    monkeypatch.setattr(oracle, fn, impl, raising=False)
    assert _some_pin_fails(), f"no pin caught: {name}"


def test_planted_tanh_removal_is_caught(monkeypatch):
    class _NP:  # numpy facade whose tanh is the identity
        def __getattr__(self, k):
            return getattr(np, k)

        @staticmethod
        def tanh(x):
            return x
    monkeypatch.setattr(off, "np", _NP())
    assert _some_pin_fails()


@pytest.mark.parametrize("name", ["multiplier", "key bump", "word order", "uniform offset"])
def test_planted_generator_mistake_is_caught(monkeypatch, name):
    if name == "multiplier":
        monkeypatch.setattr(oph, "PHILOX_M0", np.uint64(0xD2E7470EE14C6C95))
    elif name == "key bump":
        monkeypatch.setattr(oph, "PHILOX_W1", np.uint64(0x9E3779B97F4A7C15))
    elif name == "word order":
        orig = oph.uniforms_from_words
        monkeypatch.setattr(oph, "uniforms_from_words", lambda x: orig(x)[..., ::-1])
    elif name == "uniform offset":
        monkeypatch.setattr(oph, "uniforms_from_words",
                            lambda x: ((np.asarray(x, dtype=np.uint64)[..., [0, 0, 1, 1, 2, 2, 3, 3]] >> np.uint64(40))).astype(float) * 2.0 ** -24)
    assert _some_pin_fails()


# ---------------------------------------------------------------------------
# the BF16-storage variants: their own pins (tests/test_oracle_bf16.py)
# ---------------------------------------------------------------------------
from tests import test_oracle_bf16 as bf16_pins  # noqa: E402

BF16_PIN_CALLS = [
    lambda: bf16_pins.test_bf16_theta_is_rounded_after_row_scaling(),
    lambda: bf16_pins.test_bf16_layer_statistics_come_from_the_unrounded_layer(),
    lambda: bf16_pins.test_bf16_equals_per_element_emulation(0, -0.5, 3, "row_scaled"),
    lambda: bf16_pins.test_bf16_equals_per_element_emulation(3, 2.0, 3, "row_scaled"),
]


def _some_bf16_pin_fails():
    for call in BF16_PIN_CALLS:
        try:
            call()
        except (AssertionError, ValueError, IndexError):
            return True
    return False


def _unrounded_first_call(orig):
    calls = []

    def store(a, dinv, layout="row_scaled"):
        calls.append(1)
        return np.asarray(a, dtype=np.float64) if len(calls) == 1 else orig(a, dinv, layout)
    return store


@pytest.mark.parametrize("name", ["rounds the unscaled value", "statistics of the rounded layer",
                                  "Theta not rounded"])
def test_planted_bf16_storage_mistake_is_caught(monkeypatch, name):
    if name == "rounds the unscaled value":
        monkeypatch.setattr(off, "bf16_store", lambda a, dinv, layout="row_scaled": off.round_bf16(a))
    elif name == "statistics of the rounded layer":
        orig = off.znorm
        monkeypatch.setattr(off, "znorm", lambda T, ddof=1: orig(off.round_bf16(T), ddof))
    else:
        # every test call makes a fresh wrapper, so Theta (the first store of an FFP) goes unrounded
        orig = off.bf16_store

        class _Fresh:
            def __call__(self, a, dinv, layout="row_scaled"):
                return self.fn(a, dinv, layout)
        fresh = _Fresh()
        real_ffp = off.ffp

        def ffp(*a, **k):
            fresh.fn = _unrounded_first_call(orig)
            return real_ffp(*a, **k)
        monkeypatch.setattr(off, "bf16_store", fresh)
        monkeypatch.setattr(off, "ffp", ffp)
        monkeypatch.setattr(oracle, "ffp", ffp)
    assert _some_bf16_pin_fails(), f"no pin caught: {name}"


def test_bf16_pins_pass_unmutated():
    assert not _some_bf16_pin_fails()
