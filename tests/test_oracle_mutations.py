"""Plant plausible mistakes in the oracle (CPU only) and check that the pins catch each one.

A pin suite that still passes with a dropped term, a flipped sign or a wrong
scale pins nothing; each mutation below must make at least one pin fail.
"""
import numpy as np
import pytest

import oracle
import tests.test_oracle_pins as pins


def _grad_no_lam2(Omega, W, lam2):
    G = 0.5 * (W.T + W)
    G[np.diag_indices_from(G)] -= 1.0 / np.diag(Omega)
    return G


def _grad_sign_flip(Omega, W, lam2):
    G = 0.5 * (W.T + W) + lam2 * Omega
    G[np.diag_indices_from(G)] += 1.0 / np.diag(Omega)
    return G


def _grad_no_half(Omega, W, lam2):
    G = (W.T + W) + lam2 * Omega
    G[np.diag_indices_from(G)] -= 1.0 / np.diag(Omega)
    return G


def _smooth_eq1_scale(Omega, W, lam2):
    d = np.diag(Omega)
    if np.any(d <= 0.0):
        return np.inf
    return -2 * np.sum(np.log(d)) + np.sum(W * Omega.T) + 0.5 * lam2 * np.sum(Omega * Omega)


def _prox_thresholds_diag(Z, alpha):
    return oracle.soft_threshold(Z, alpha)


def _gram_transposed(X):
    X = np.asarray(X, dtype=np.float64)
    return (X @ X.T)[: X.shape[1], : X.shape[1]] / X.shape[0] if X.shape[0] >= X.shape[1] else \
        np.eye(X.shape[1])


MUTATIONS = {
    "gradient_drops_lam2": ("gradient", _grad_no_lam2),
    "gradient_log_sign": ("gradient", _grad_sign_flip),
    "gradient_drops_half": ("gradient", _grad_no_half),
    "smooth_eq1_scale": ("smooth", _smooth_eq1_scale),
    "prox_thresholds_diagonal": ("prox", _prox_thresholds_diag),
    "gram_wrong_operand": ("gram", _gram_transposed),
}

PINS = [
    lambda: pins.test_gram_brute_force(),
    lambda: [pins.test_gradient_is_derivative_of_smooth(s) for s in (0, 1)],
    lambda: [pins.test_diagonal_S_closed_form(l) for l in (0.0, 0.3)],
    lambda: pins.test_first_step_closed_form(),
    lambda: pins.test_lambda_max_closed_form(),
    lambda: pins.test_matches_independent_coordinate_descent(4, 0, 0.05),
    lambda: pins.test_monotone_descent_and_symmetry(),
]


def _some_pin_fails():
    for pin in PINS:
        try:
            pin()
        except (AssertionError, FloatingPointError, ValueError, IndexError):
            return True
    return False


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(oracle, attr, fn)
    with np.errstate(all="ignore"):
        assert _some_pin_fails(), f"no pin catches mutation {name}"


def test_threshold_without_tau_is_caught(monkeypatch):
    """Thresholding at lam1 instead of tau*lam1 moves the fixed point."""
    real = oracle.prox

    def bad_iterate(S, Omega, W, lam1, lam2, tau0=1.0, shrink=0.5, max_halvings=60):
        G = oracle.gradient(Omega, W, lam2)
        g = oracle.smooth(Omega, W, lam2)
        tau = tau0
        for h in range(max_halvings + 1):
            Op = real(Omega - tau * G, lam1)
            if np.all(np.diag(Op) > 0.0):
                Wp = oracle.times_S(Op, S)
                gp = oracle.smooth(Op, Wp, lam2)
                D = Op - Omega
                if gp <= g + np.sum(D * G) + np.sum(D * D) / (2.0 * tau):
                    return oracle.Step(Op, Wp, tau, h + 1, True, G, g)
            tau *= shrink
        return oracle.Step(Omega, W, tau, max_halvings + 1, False, G, g)

    monkeypatch.setattr(oracle, "iterate", bad_iterate)
    assert _some_pin_fails()


def test_unmutated_oracle_passes_every_pin():
    assert not _some_pin_fails()
