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


# ------------------------------------------------------------- differentiation and entry helpers
# The differentiation oracle and the sampled-entry helpers (used by the full-size parity
# tests) carry their own pins; each mistake below must make one of those fail.

_real = {name: getattr(oracle, name) for name in
         ("smooth_loss_grads", "hypergrad", "hypergrad_sparse", "gram_entries", "gradient_entries")}


def _dx_without_transpose_term(X, Omega, lam2):
    dOm, _ = _real["smooth_loss_grads"](X, Omega, lam2)
    X = np.asarray(X, dtype=np.float64)
    return dOm, X @ Omega @ Omega / X.shape[0]


def _domega_without_half(X, Omega, lam2):
    dOm, dX = _real["smooth_loss_grads"](X, Omega, lam2)
    S = oracle.gram(X)
    return dOm + 0.5 * (Omega.T @ S + S @ Omega.T), dX


def _hypergrad_without_diag_hessian(S, S_val, Omega, lam1, lam2):
    p = S.shape[0]
    iu, ju = np.nonzero(np.triu(Omega != 0.0))
    d = np.diag(Omega)
    Hm = np.zeros((iu.size, iu.size))
    for t, (a, b) in enumerate(zip(iu, ju)):
        E = np.zeros((p, p))
        E[a, b] = E[b, a] = 1.0
        Hm[:, t] = (0.5 * (E @ S + S @ E) + lam2 * E)[iu, ju]
    gval = 0.5 * (Omega @ S_val + S_val @ Omega)
    gval[np.diag_indices(p)] -= 1.0 / d
    v = np.linalg.solve(Hm, gval[iu, ju])
    w = np.where(iu == ju, 1.0, 2.0)
    s = np.where(iu == ju, 0.0, np.sign(Omega[iu, ju]))
    return float(-np.sum(w * v * s)), float(-np.sum(w * v * Omega[iu, ju]))


def _hypergrad_lambda1_sign(S, S_val, Omega, lam1, lam2):
    g1, g2 = _real["hypergrad"](S, S_val, Omega, lam1, lam2)
    return -g1, g2


def _sparse_hypergrad_training_data_held_out(X, Xval, omega_csr, lam1, lam2):
    return _real["hypergrad_sparse"](X, X, omega_csr, lam1, lam2)


def _gram_entries_unbiased(X, rows, cols):
    n = X.shape[0]
    return _real["gram_entries"](X, rows, cols) * n / (n - 1)


def _gradient_entries_without_lam2(X, omega_csr, lam2, rows, cols):
    return _real["gradient_entries"](X, omega_csr, 0.0, rows, cols)


DIFF_MUTATIONS = {
    "dX_drops_transpose_term": ("smooth_loss_grads", _dx_without_transpose_term),
    "dOmega_drops_half": ("smooth_loss_grads", _domega_without_half),
    "hypergrad_drops_diag_hessian": ("hypergrad", _hypergrad_without_diag_hessian),
    "hypergrad_lambda1_sign": ("hypergrad", _hypergrad_lambda1_sign),
    "sparse_hypergrad_wrong_held_out_operand": ("hypergrad_sparse", _sparse_hypergrad_training_data_held_out),
    "gram_entries_divides_by_n_minus_1": ("gram_entries", _gram_entries_unbiased),
    "gradient_entries_drops_lam2": ("gradient_entries", _gradient_entries_without_lam2),
}

DIFF_PINS = [
    lambda: pins.test_entry_helpers_match_dense(),
    lambda: pins.test_smooth_loss_grads_by_central_differences(),
    lambda: pins.test_smooth_loss_grads_reduce_to_G_and_Y_Omega_at_symmetric_omega(),
    lambda: pins.test_hypergrad_by_central_differences_of_resolved_estimates(0),
    lambda: pins.test_sparse_hypergrad_equals_dense_hypergrad(),
]


def _some_diff_pin_fails():
    for pin in DIFF_PINS:
        try:
            pin()
        except (AssertionError, FloatingPointError, ValueError, IndexError, np.linalg.LinAlgError):
            return True
    return False


@pytest.mark.parametrize("name", sorted(DIFF_MUTATIONS))
def test_planted_differentiation_mistake_is_caught(name, monkeypatch):
    attr, fn = DIFF_MUTATIONS[name]
    monkeypatch.setattr(oracle, attr, fn)
    with np.errstate(all="ignore"):
        assert _some_diff_pin_fails(), f"no pin catches mutation {name}"


def test_unmutated_differentiation_oracle_passes_its_pins():
    assert not _some_diff_pin_fails()
