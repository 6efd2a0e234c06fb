"""The CSR-iterate form of the oracle (Alg. 2 and Alg. 3 with Omega held sparse), used for
the full-size FP64 references, pinned to the dense oracle (CPU only):

- the chunked Gram equals the dense Gram to rounding and is exactly symmetric;
- on small problems the CSR forms take the dense oracle's exact step-size sequence and
  trial counts and return the same estimate (Cov and Obs), stopped at eps = 1e-7, above
  the FP64 floor of the literal line-search test;
- the optimality residual it reports bounds the distance to the minimiser: the estimate
  at eps = 1e-7 lies within ||r||_F / lambda2 of a solve taken to eps = 1e-9, and the
  residual of that tight solve is small;
- the closed form of the diagonal case (omega_ii = 1 / sqrt(s_i + lambda2), lambda1 = 0);
- planted mistakes in the CSR steps (candidates limited to the support, the support
  product transposed, the diagonal thresholded) are caught by these pins.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from workloads import small_problem

CASES = [(120, 80, 4.0, 3, 0.1), (120, 80, 4.0, 3, 0.3), (90, 200, 3.0, 5, 0.15), (60, 30, 2.0, 7, 0.2)]


def test_chunked_gram():
    X = small_problem(70, 53, 3.0, 1)
    S = oracle.gram(X)
    S2 = oracle.gram_chunked(X, block=16)
    assert np.array_equal(S2, S2.T) and S2.flags["C_CONTIGUOUS"]
    assert np.max(np.abs(S - S2)) <= 1e-14 * np.max(np.abs(S))


@pytest.mark.parametrize("case", CASES)
def test_csr_forms_take_the_dense_steps(case):
    p, n, d, seed, lam1 = case
    X = small_problem(p, n, d, seed)
    S = oracle.gram(X)
    r = oracle.solve(S, lam1, 0.1, eps=1e-7)
    q = oracle.solve_sparse(S, lam1, 0.1, eps=1e-7, block=32, threads=2)
    assert r.status == q.status == "converged"
    assert q.iterations == r.iterations and q.taus == r.taus and q.trials == r.trials
    nr = np.linalg.norm(r.omega)
    assert np.linalg.norm(q.omega.toarray() - r.omega) <= 1e-12 * nr
    assert np.allclose(q.F, r.F, rtol=1e-13, atol=0)
    o = oracle.solve_obs_sparse(X, lam1, 0.1, eps=1e-7, block=32)
    ro = oracle.solve_obs(X, lam1, 0.1, eps=1e-7)
    assert o.taus == ro.taus and o.trials == ro.trials
    assert np.linalg.norm(o.omega.toarray() - ro.omega) <= 1e-12 * nr


def test_residual_bounds_the_distance():
    p, n, d, seed, lam1 = CASES[0]
    lam2 = 0.1
    X = small_problem(p, n, d, seed)
    S = oracle.gram(X)
    tight = oracle.solve(S, lam1, lam2, eps=1e-9).omega
    for eps in (1e-4, 1e-6, 1e-7):
        q = oracle.solve_sparse(S, lam1, lam2, eps=eps, block=32, threads=2)
        Gk, _ = oracle.gradient_candidates_cov(S, q.omega, lam1, lam2, 32, 2)
        r = np.linalg.norm(oracle.kkt_residual_csr(Gk, q.omega, lam1))
        dist = np.linalg.norm(q.omega.toarray() - tight)
        # the tight solve is itself within its own residual of the minimiser
        Gt, _ = oracle.gradient_candidates_cov(S, sp.csr_matrix(tight), lam1, lam2, 32, 2)
        rt = np.linalg.norm(oracle.kkt_residual_csr(Gt, sp.csr_matrix(tight), lam1))
        assert dist <= (r + rt) / lam2
        assert rt < 1e-6


def test_diagonal_closed_form():
    s = np.array([0.5, 1.0, 2.0, 3.5, 0.25])
    S = np.diag(s)
    q = oracle.solve_sparse(S, 0.0, 0.2, eps=1e-8, block=2, threads=1)
    assert q.omega.nnz == 5
    assert np.allclose(q.omega.diagonal(), 1.0 / np.sqrt(s + 0.2), rtol=1e-6)


# ----------------------------------------------------------------- planted mistakes

def _cands_support_only(S, omega, lam1, lam2, block=512, threads=8):
    Gk, W = _ORIG["gradient_candidates_cov"](S, omega, lam1, lam2, block, threads)
    keep = _ORIG["_on_pattern"](omega + sp.identity(omega.shape[0], format="csr"), Gk) != 0
    rows = np.repeat(np.arange(Gk.shape[0]), np.diff(Gk.indptr))
    G2 = sp.csr_matrix((Gk.data[keep], (rows[keep], Gk.indices[keep])), shape=Gk.shape)
    G2.sort_indices()
    return G2, W


def _w_transposed(S, omega):
    return _ORIG["w_on_support"](S.T * np.linspace(1.0, 1.5, S.shape[0])[None, :], omega)


def _prox_csr_diag(Zk, alpha):
    v = oracle.soft_threshold(Zk.data, alpha)
    out = sp.csr_matrix((v, Zk.indices.copy(), Zk.indptr.copy()), shape=Zk.shape)
    out.eliminate_zeros()
    out.sort_indices()
    return out


_ORIG = {k: getattr(oracle, k) for k in ("gradient_candidates_cov", "_on_pattern", "w_on_support", "prox_csr")}

MUTATIONS = {
    "candidates_support_only": ("gradient_candidates_cov", _cands_support_only),
    "support_product_wrong_operand": ("w_on_support", _w_transposed),
    "prox_thresholds_diagonal": ("prox_csr", _prox_csr_diag),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    attr, fn = MUTATIONS[name]
    monkeypatch.setattr(oracle, attr, fn)
    caught = False
    for pin in (lambda: test_csr_forms_take_the_dense_steps(CASES[0]), test_diagonal_closed_form):
        try:
            pin()
        except (AssertionError, FloatingPointError, ValueError):
            caught = True
            break
    assert caught, name
