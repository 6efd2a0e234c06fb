"""The sampled optimality check (tests/kkt.py) that the full-size parity tests rely on:
it accepts the oracle's fixed point and rejects the same estimate checked at a
neighbouring lambda1 of the path grid (CPU only)."""
import numpy as np
import scipy.sparse as sp

import oracle
from tests import kkt
from workloads import small_problem


def test_kkt_helper_accepts_the_fixed_point_and_rejects_a_neighbour():
    X = small_problem(60, 90, 3.0, 7)
    S = oracle.gram(X)
    lam1, lam2 = 0.1, 0.1
    om = sp.csr_matrix(oracle.solve(S, lam1, lam2, eps=1e-9, max_iter=100000).omega)
    rng = np.random.default_rng(0)
    r, c = kkt.sample_pairs(om, rng, rows=20, hubs=5, per_row=10, random_pairs=200)
    d, s, o, nsup = kkt.residuals(X, om, lam1, lam2, r, c)
    assert nsup >= 10
    assert max(d, s, o) < 1e-6, (d, s, o)
    # one step along a 32-point log grid over [0.05, 0.8] is a factor 16^(1/31) = 1.094
    _, s2, _, _ = kkt.residuals(X, om, lam1 * 16 ** (1 / 31), lam2, r, c)
    assert s2 > 5e-3
    # a planted wrong diagonal breaks the diagonal condition
    bad = om.tolil()
    bad[3, 3] = bad[3, 3] * 1.01
    r3 = np.concatenate([r, [3]])
    c3 = np.concatenate([c, [3]])
    d3, _, _, _ = kkt.residuals(X, bad.tocsr(), lam1, lam2, r3, c3)
    assert d3 > 1e-3
