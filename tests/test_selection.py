"""Support recovery (PPV / FDR / TPR over off-diagonal pairs, Section 4's Table 1 scores) on
hand-built patterns (CPU only)."""
import numpy as np
import scipy.sparse as sp

from paper_1710_10769_gb300.selection import support_recovery


def _sym(p, pairs, diag=True):
    r = [i for i, j in pairs] + [j for i, j in pairs]
    c = [j for i, j in pairs] + [i for i, j in pairs]
    a = sp.coo_matrix((np.ones(len(r)), (r, c)), shape=(p, p)).tocsr()
    return a + sp.identity(p) if diag else a


def test_counts_on_a_hand_built_case():
    truth = _sym(6, [(0, 1), (1, 2), (3, 4)])
    est = _sym(6, [(0, 1), (1, 2), (2, 5), (0, 5)])
    r = support_recovery(est, truth)
    assert (r["tp"], r["fp"], r["fn"], r["pairs"]) == (2, 2, 1, 4)
    assert r["ppv"] == 0.5 and r["fdr"] == 0.5 and abs(r["tpr"] - 2 / 3) < 1e-15


def test_diagonal_and_duplicates_do_not_count():
    truth = _sym(5, [(0, 4)])
    est = _sym(5, [(4, 0)]) * 3.0            # same pair, other orientation, any values
    r = support_recovery(est, truth)
    assert (r["tp"], r["fp"], r["fn"]) == (1, 0, 0) and r["ppv"] == 1.0 and r["fdr"] == 0.0
    empty = support_recovery(sp.identity(5), truth)
    assert empty["pairs"] == 0 and empty["ppv"] == 1.0 and empty["tpr"] == 0.0
    dense = support_recovery(est.toarray(), truth.toarray())
    assert dense == r
