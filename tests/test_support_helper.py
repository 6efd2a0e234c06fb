"""The shared support rule (tests/support.py) on an oracle estimate: it accepts the estimate
itself and one-sided entries whose value is within the band, and rejects one-sided entries
far from the threshold (CPU only)."""
import numpy as np

import oracle
from tests.support import support_diff_ok
from workloads import small_problem


def test_support_rule_accepts_and_rejects():
    X = small_problem(60, 80, 3.0, 4)
    S = oracle.gram(X)
    lam1, lam2 = 0.15, 0.1
    R = oracle.solve(S, lam1, lam2, eps=1e-10, max_iter=20000).omega
    assert support_diff_ok(R, R, lam1, lam2, S=S) == (True, 0)
    G = oracle.gradient(R, oracle.times_S(R, S), lam2)
    off = ~np.eye(60, dtype=bool)
    # an entry off the support whose |G_ij| is far below lambda1: adding it breaks the rule
    i, j = np.argwhere(off & (R == 0) & (np.abs(G) < 0.5 * lam1))[0]
    bad = R.copy()
    bad[i, j] = bad[j, i] = 1e-3
    ok, detail = support_diff_ok(bad, R, lam1, lam2, S=S)
    assert not ok and detail[:2] in ((i, j), (j, i))
    # the same entry at a value within the band: accepted
    ok_small, _ = support_diff_ok(np.where(bad == 1e-3, 1e-7, bad), R, lam1, lam2, S=S)
    assert ok_small
    # dropping a support entry of the reference: accepted only if its value is within the band
    k, m = np.argwhere(off & (R != 0))[0]
    drop = R.copy()
    drop[k, m] = drop[m, k] = 0.0
    assert support_diff_ok(drop, R, lam1, lam2, S=S, band=abs(R[k, m]) * 1.01)[0]
    assert not support_diff_ok(drop, R, lam1, lam2, S=S, band=abs(R[k, m]) * 0.99)[0]
