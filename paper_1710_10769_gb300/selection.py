"""Model selection over a lambda1 grid and support recovery against a known pattern.

Section 2 motivates solving whole grids of tuning parameters (for cross-validation and
stability selection); Section 4 (Table 1) scores estimates by the positive predictive
value and false discovery rate of their sparsity pattern against the true Omega0.

- ``select_lambda1``: the grid solved by the library's warm-started path (hpc_solve_path),
  the held-out loss L_val = -sum log w_ii + tr(Omega S_val Omega)/2 of every point
  evaluated on the device (hpc_heldout_loss), and the point of smallest held-out loss.
- ``support_recovery``: PPV, FDR and the true-positive rate of an estimate's off-diagonal
  pattern (unordered pairs i < j) against a reference pattern.  Host-side set arithmetic
  on the two patterns; no estimator arithmetic happens here.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _upper_pairs(a) -> np.ndarray:
    """Keys i * p + j of the off-diagonal pattern's pairs i < j (a symmetric pattern)."""
    m = sp.coo_matrix(a)
    keep = (m.row < m.col) & (m.data != 0)
    return np.unique(m.row[keep].astype(np.int64) * m.shape[0] + m.col[keep])


def support_recovery(estimate, truth) -> dict:
    """PPV = TP / (TP + FP), FDR = FP / (TP + FP) and TPR = TP / |truth| over off-diagonal pairs.

    ``estimate`` and ``truth`` are square sparse (or dense) matrices with symmetric patterns;
    only entries off the diagonal count.  An empty estimate has PPV 1 and FDR 0."""
    e = _upper_pairs(estimate)
    t = _upper_pairs(truth)
    tp = int(np.intersect1d(e, t, assume_unique=True).size)
    fp = int(e.size - tp)
    fn = int(t.size - tp)
    ppv = tp / (tp + fp) if tp + fp else 1.0
    return {"tp": tp, "fp": fp, "fn": fn, "ppv": ppv, "fdr": 1.0 - ppv if tp + fp else 0.0,
            "tpr": tp / t.size if t.size else 1.0, "pairs": int(e.size)}


def select_lambda1(solver, Xval, lambda1s, lambda2, truth=None) -> dict:
    """Solve the grid (descending lambda1s recommended: sparse to dense warm starts), evaluate the
    held-out loss at every estimate and return the selection.

    Returns {"lambda1": grid, "heldout": losses, "best": index of the smallest loss,
    "points": per-point solve statistics, "recovery": per-point support_recovery against
    ``truth`` (when given)}.  The solver is left at the selected estimate and lambda."""
    lam = [float(v) for v in lambda1s]
    points, ests = solver.solve_path(lam, lambda2)
    losses = []
    for est in ests:
        solver.set_omega(est)
        losses.append(solver.heldout_loss(Xval))
    best = int(np.argmin(losses))
    solver.set_omega(ests[best])
    solver.set_lambda(lam[best], lambda2)
    out = {"lambda1": lam, "heldout": losses, "best": best, "points": points}
    if truth is not None:
        out["recovery"] = [support_recovery(e.to_scipy(solver.p), truth) for e in ests]
    return out
