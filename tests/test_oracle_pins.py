"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics.

Each test pins a different part of the oracle, so that a plausible mistake in
it (a dropped term, a wrong sign, index or scale, a transposed operand, a
thresholded diagonal) fails at least one of them:

* eq. (2) values and its tie rule                      -> soft_threshold / prox
* Gram against a brute-force triple loop               -> gram
* central finite differences of g against <G, E>       -> gradient vs smooth (scales, signs)
* diagonal-S closed form w_ii = 1/sqrt(s_i + lam2)     -> fixed point of Alg. 1 (scale of G)
* lam_max closed form and the first pair to enter      -> off-diagonal gradient
* first step from Omega = I in closed form             -> prox step, tau handling
* KKT conditions at convergence                        -> stopping rule / fixed point
* an independent coordinate-descent solver (p <= 6)    -> whole solve
* every single support flip raises F (p <= 5)          -> optimality of the support
* monotone descent of F and bitwise symmetry           -> line-search test direction
* Cov (Alg. 2) and Obs (Alg. 3) agree                  -> the ||Y||^2/n identity
"""
import os

import numpy as np
import pytest

import oracle
from workloads import omega0_random, sample_x_cpu, small_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rand_problem(p, n, seed, degree=2.0):
    X = small_problem(p, n, degree, seed)
    return X, oracle.gram(X)


# ------------------------------------------------------------------ eq. (2)

def test_soft_threshold_eq2_golden():
    """Values of eq. (2) read off its three cases, including both ties (|z| = alpha -> 0)."""
    rows = np.loadtxt(os.path.join(GOLDEN, "soft_threshold_eq2.txt"), comments="#")
    z, alpha, expect = rows[:, 0], rows[:, 1], rows[:, 2]
    got = oracle.soft_threshold(z, alpha)
    assert np.array_equal(got, expect)


def test_prox_keeps_diagonal():
    Z = np.array([[0.1, 0.5, -0.05], [0.5, -0.2, 0.3], [-0.05, 0.3, 2.0]])
    P = oracle.prox(Z, 0.25)
    assert np.array_equal(np.diag(P), np.diag(Z))          # diagonal not thresholded
    assert P[0, 1] == pytest.approx(0.25) and P[0, 2] == 0.0 and P[1, 2] == pytest.approx(0.05)


# ------------------------------------------------------------------ Gram

def test_gram_brute_force():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((7, 5))
    S = oracle.gram(X)
    n, p = X.shape
    for i in range(p):
        for j in range(p):
            s = 0.0
            for k in range(n):
                s += X[k, i] * X[k, j]
            assert S[i, j] == pytest.approx(s / n, rel=1e-14, abs=1e-15)


# ------------------------------------------------------------------ gradient vs smooth part

@pytest.mark.parametrize("seed", [0, 1, 2])
def test_gradient_is_derivative_of_smooth(seed):
    """<G, E> equals the central difference of g along symmetric E (quadratic + log: O(h^2))."""
    X, S = _rand_problem(8, 12, seed)
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((8, 8)) * 0.1
    Om = np.eye(8) * 1.3 + (A + A.T) * 0.5
    E = rng.standard_normal((8, 8))
    E = E + E.T
    lam2 = 0.37
    G = oracle.gradient(Om, oracle.times_S(Om, S), lam2)
    h = 1e-5
    gp = oracle.smooth(Om + h * E, oracle.times_S(Om + h * E, S), lam2)
    gm = oracle.smooth(Om - h * E, oracle.times_S(Om - h * E, S), lam2)
    fd = (gp - gm) / (2 * h)
    assert np.sum(G * E) == pytest.approx(fd, rel=1e-7)


def test_gradient_symmetric_bitwise():
    X, S = _rand_problem(9, 20, 4)
    Om = oracle.solve(S, 0.1, 0.2, eps=1e-4).omega
    G = oracle.gradient(Om, oracle.times_S(Om, S), 0.2)
    assert np.array_equal(G, G.T)


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("lam1", [0.0, 0.3])
def test_diagonal_S_closed_form(lam1):
    """With S diagonal the minimiser is diag(1/sqrt(s_i + lam2)) for any lam1 >= 0.

    (Under eq. (1)'s literal scale it would be sqrt(2/(2 s_i + lam2)) instead.)
    """
    s = np.array([0.5, 1.0, 2.5, 0.2, 4.0, 1.7])
    lam2 = 0.2
    res = oracle.solve(np.diag(s), lam1, lam2, eps=1e-9, max_iter=5000)
    assert res.status in ("converged", "floor")
    expect = 1.0 / np.sqrt(s + lam2)
    # the FP64 sufficient-decrease test decides reliably down to ~1e-8 relative change
    assert np.allclose(np.diag(res.omega), expect, rtol=1e-7, atol=0)
    off = res.omega - np.diag(np.diag(res.omega))
    assert np.all(off == 0.0)


def test_lambda_max_closed_form():
    """Omega* is diagonal iff lam1 >= max_{i!=j} |S_ij| (w_ii + w_jj) / 2 with w_ii = 1/sqrt(S_ii+lam2)."""
    X, S = _rand_problem(7, 30, 11)
    lam2 = 0.1
    w = 1.0 / np.sqrt(np.diag(S) + lam2)
    M = 0.5 * np.abs(S) * (w[:, None] + w[None, :])
    np.fill_diagonal(M, 0.0)
    lam_max = M.max()
    a, b = np.unravel_index(np.argmax(M), M.shape)
    above = oracle.solve(S, lam_max * 1.001, lam2, eps=1e-9, max_iter=20000)
    assert np.count_nonzero(above.omega - np.diag(np.diag(above.omega))) == 0
    assert np.allclose(np.diag(above.omega), w, rtol=1e-7)
    below = oracle.solve(S, lam_max * 0.995, lam2, eps=1e-9, max_iter=20000)
    nz = np.argwhere(below.omega - np.diag(np.diag(below.omega)) != 0)
    assert {tuple(x) for x in nz} == {(a, b), (b, a)}


def test_first_step_closed_form():
    """From Omega = I: G = S - (1 - lam2) I and Omega^1 = prox(I - tau G, tau lam1) entrywise."""
    X, S = _rand_problem(10, 40, 5)
    lam1, lam2 = 0.15, 0.1
    res = oracle.solve(S, lam1, lam2, eps=1e-6, max_iter=1)
    tau = res.taus[0]
    Z = np.eye(10) - tau * (S - (1.0 - lam2) * np.eye(10))
    expect = np.where(np.abs(Z) > tau * lam1, Z - np.sign(Z) * tau * lam1, 0.0)
    np.fill_diagonal(expect, np.diag(Z))
    assert np.allclose(res.omega, expect, rtol=0, atol=1e-15)


# ------------------------------------------------------------------ optimality

def _kkt_residual(S, Om, lam1, lam2):
    G = oracle.gradient(Om, oracle.times_S(Om, S), lam2)
    p = S.shape[0]
    r = 0.0
    for i in range(p):
        for j in range(p):
            if i == j:
                r = max(r, abs(G[i, i]))
            elif Om[i, j] != 0.0:
                r = max(r, abs(G[i, j] + lam1 * np.sign(Om[i, j])))
            else:
                r = max(r, max(0.0, abs(G[i, j]) - lam1))
    return r


@pytest.mark.parametrize("seed", [0, 1])
def test_kkt_at_convergence(seed):
    X, S = _rand_problem(30, 60, seed, degree=3.0)
    lam1, lam2 = 0.12, 0.1
    res = oracle.solve(S, lam1, lam2, eps=1e-9, max_iter=20000)
    assert res.status in ("converged", "floor")
    assert _kkt_residual(S, res.omega, lam1, lam2) < 1e-6


def _cd_solve(S, lam1, lam2, sweeps=200000, tol=1e-15):
    """Exact coordinate descent on the same objective, derived independently of Alg. 1.

    Off-diagonal pair x = w_ij = w_ji:  (S_ii + S_jj + 2 lam2)/2 x^2 + b x + 2 lam1 |x|,
        b = sum_{l != j} S_jl w_il + sum_{l != i} S_il w_jl   ->  x = -soft(b, 2 lam1) / (S_ii + S_jj + 2 lam2)
    Diagonal x = w_ii: -log x + (S_ii + lam2)/2 x^2 + c x, c = sum_{l != i} S_il w_il
        ->  (S_ii + lam2) x^2 + c x - 1 = 0, positive root.
    """
    p = S.shape[0]
    Om = np.eye(p)
    for _ in range(sweeps):
        old = Om.copy()
        for i in range(p):
            c = sum(S[i, l] * Om[i, l] for l in range(p) if l != i)
            a = S[i, i] + lam2
            Om[i, i] = (-c + np.sqrt(c * c + 4.0 * a)) / (2.0 * a)
        for i in range(p):
            for j in range(i + 1, p):
                b = sum(S[j, l] * Om[i, l] for l in range(p) if l != j) + \
                    sum(S[i, l] * Om[j, l] for l in range(p) if l != i)
                st = np.sign(b) * max(abs(b) - 2.0 * lam1, 0.0)
                x = -st / (S[i, i] + S[j, j] + 2.0 * lam2)
                Om[i, j] = Om[j, i] = x
            c = sum(S[i, l] * Om[i, l] for l in range(p) if l != i)
            a = S[i, i] + lam2
            Om[i, i] = (-c + np.sqrt(c * c + 4.0 * a)) / (2.0 * a)
        if np.max(np.abs(Om - old)) < tol:
            break
    return Om


@pytest.mark.parametrize("p,seed,lam1", [(4, 0, 0.05), (5, 1, 0.1), (6, 2, 0.08), (6, 3, 0.0)])
def test_matches_independent_coordinate_descent(p, seed, lam1):
    X, S = _rand_problem(p, 3 * p, seed, degree=2.0)
    lam2 = 0.15
    ref = _cd_solve(S, lam1, lam2)
    res = oracle.solve(S, lam1, lam2, eps=1e-9, max_iter=100000)
    assert res.status in ("converged", "floor")
    err = np.linalg.norm(res.omega - ref) / np.linalg.norm(ref)
    assert err < 1e-7
    # same support (entries of the CD solution far from zero)
    assert np.array_equal(np.abs(ref) > 1e-7, np.abs(res.omega) > 1e-7)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_support_flips_raise_objective(seed):
    """Brute force on p = 5: moving any single pair off (or onto) the support raises F."""
    X, S = _rand_problem(5, 9, seed, degree=2.0)
    lam1, lam2 = 0.07, 0.1
    res = oracle.solve(S, lam1, lam2, eps=1e-9, max_iter=100000)
    Om = res.omega
    F0 = oracle.objective(S, Om, lam1, lam2)
    rng = np.random.default_rng(seed)
    for i in range(5):
        for j in range(i + 1, 5):
            for delta in (1e-3, -1e-3, 3e-2, -3e-2):
                T = Om.copy()
                if Om[i, j] != 0.0:
                    T[i, j] = T[j, i] = 0.0 if abs(delta) > 1e-2 else Om[i, j] + delta
                else:
                    T[i, j] = T[j, i] = delta
                assert oracle.objective(S, T, lam1, lam2) > F0
    for _ in range(20):     # random symmetric perturbations too
        E = rng.standard_normal((5, 5)) * 1e-3
        assert oracle.objective(S, Om + E + E.T, lam1, lam2) > F0


# ------------------------------------------------------------------ trajectory properties

def test_monotone_descent_and_symmetry():
    X, S = _rand_problem(40, 30, 7, degree=3.0)
    res = oracle.solve(S, 0.1, 0.05, eps=1e-8, max_iter=5000)
    F = np.array(res.F)
    assert np.all(np.diff(F) <= 1e-12 * np.abs(F[:-1]))
    assert np.array_equal(res.omega, res.omega.T)
    assert res.iterations > 3


def test_cov_and_obs_reach_the_same_estimate():
    """tr(Omega S Omega) = ||Omega X^T||^2 / n: Alg. 2 and Alg. 3 follow the same iterates."""
    X, S = _rand_problem(25, 15, 9, degree=2.0)     # p > n, as Obs is meant for
    a = oracle.solve(S, 0.1, 0.1, eps=1e-7, max_iter=5000)
    b = oracle.solve_obs(X, 0.1, 0.1, eps=1e-7, max_iter=5000)
    # above the FP64 floor of the decrease test both variants take the same steps
    assert a.taus == b.taus
    assert np.linalg.norm(a.omega - b.omega) / np.linalg.norm(a.omega) < 1e-10


# ------------------------------------------------------------------ sampled-entry helpers

def test_entry_helpers_match_dense():
    X = small_problem(30, 50, 3.0, 21).astype(np.float32)
    S = oracle.gram(X)
    res = oracle.solve(S, 0.1, 0.1, eps=1e-6)
    import scipy.sparse as sp

    om = sp.csr_matrix(res.omega)
    rng = np.random.default_rng(0)
    r = rng.integers(0, 30, 40)
    c = rng.integers(0, 30, 40)
    assert np.allclose(oracle.gram_entries(X, r, c), S[r, c], rtol=1e-12, atol=1e-15)
    G = oracle.gradient(res.omega, oracle.times_S(res.omega, S), 0.1)
    assert np.allclose(oracle.gradient_entries(X, om, 0.1, r, c), G[r, c], rtol=1e-10, atol=1e-13)
    assert oracle.smooth_sparse_from_S(S, om, 0.1) == pytest.approx(
        oracle.smooth(res.omega, oracle.times_S(res.omega, S), 0.1), rel=1e-12)


# ------------------------------------------------------------------ differentiation

def test_smooth_loss_grads_by_central_differences():
    """dL/dX is exact for central differences (L is quadratic in X); dL/dOmega to O(h^2)."""
    rng = np.random.default_rng(5)
    X = rng.standard_normal((9, 6))
    A = rng.standard_normal((6, 6)) * 0.1
    Om = np.eye(6) * 1.5 + A                      # deliberately not symmetric
    lam2 = 0.3
    dOm, dX = oracle.smooth_loss_grads(X, Om, lam2)
    h = 1e-3
    for (a, b) in [(0, 0), (1, 3), (4, 2), (5, 5)]:
        E = np.zeros_like(Om)
        E[a, b] = 1.0
        fd = (oracle.smooth_loss(X, Om + h * E, lam2) - oracle.smooth_loss(X, Om - h * E, lam2)) / (2 * h)
        assert dOm[a, b] == pytest.approx(fd, rel=1e-5, abs=1e-7)
    for (a, b) in [(0, 0), (3, 1), (8, 5)]:
        E = np.zeros_like(X)
        E[a, b] = 1.0
        fd = (oracle.smooth_loss(X + h * E, Om, lam2) - oracle.smooth_loss(X - h * E, Om, lam2)) / (2 * h)
        assert dX[a, b] == pytest.approx(fd, rel=1e-9, abs=1e-12)


def test_smooth_loss_grads_reduce_to_G_and_Y_Omega_at_symmetric_omega():
    X, S = _rand_problem(10, 14, 3)
    Om = oracle.solve(S, 0.1, 0.2, eps=1e-7).omega
    dOm, dX = oracle.smooth_loss_grads(X, Om, 0.2)
    assert np.allclose(dOm, oracle.gradient(Om, oracle.times_S(Om, S), 0.2), rtol=1e-12, atol=1e-12)
    assert np.allclose(dX, (X @ Om) @ Om / X.shape[0], rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("seed", [0, 1])
def test_hypergrad_by_central_differences_of_resolved_estimates(seed):
    """Implicit lambda-gradients against central differences (h = 1e-3) of L_val at re-solved
    estimates, on a support that stays constant over [lambda - h, lambda + h]."""
    p = 12
    Xtr = small_problem(p, 40, 3.0, 100 + seed)
    Xva = small_problem(p, 30, 3.0, 200 + seed)
    S, Sv = oracle.gram(Xtr), oracle.gram(Xva)
    lam2, h = 0.15, 1e-3
    sol = lambda l1, l2: oracle.solve(S, l1, l2, eps=1e-9, max_iter=200000).omega
    # the gradient exists where the support is locally constant: take the first such lambda1
    for lam1 in (0.12, 0.1, 0.14, 0.16, 0.09):
        Om = sol(lam1, lam2)
        ups = [sol(lam1 + h, lam2), sol(lam1 - h, lam2), sol(lam1, lam2 + h), sol(lam1, lam2 - h)]
        if all(np.array_equal(U != 0, Om != 0) for U in ups):
            break
    else:
        pytest.fail("no lambda1 with a support constant on the stencil")
    g1, g2 = oracle.hypergrad(S, Sv, Om, lam1, lam2)
    fd1 = (oracle.heldout_loss(Sv, ups[0]) - oracle.heldout_loss(Sv, ups[1])) / (2 * h)
    fd2 = (oracle.heldout_loss(Sv, ups[2]) - oracle.heldout_loss(Sv, ups[3])) / (2 * h)
    assert g1 == pytest.approx(fd1, rel=2e-3, abs=1e-5)
    assert g2 == pytest.approx(fd2, rel=2e-3, abs=1e-5)


def test_sparse_hypergrad_equals_dense_hypergrad():
    """The large-p form (sparse H from single S entries) against the dense form."""
    import scipy.sparse as sp

    p = 15
    Xtr = small_problem(p, 50, 3.0, 300)
    Xva = small_problem(p, 35, 3.0, 301)
    S, Sv = oracle.gram(Xtr), oracle.gram(Xva)
    Om = oracle.solve(S, 0.1, 0.2, eps=1e-9, max_iter=100000).omega
    a = oracle.hypergrad(S, Sv, Om, 0.1, 0.2)
    b = oracle.hypergrad_sparse(Xtr, Xva, sp.csr_matrix(Om), 0.1, 0.2)
    assert a[0] == pytest.approx(b[0], rel=1e-10) and a[1] == pytest.approx(b[1], rel=1e-10)
