"""Optimality conditions of the prox-gradient fixed point (eq. (2)) at sampled pairs of an
estimate, with the gradient formed by the oracle from X (FP64, one entry at a time), for
parity checks at sizes the oracle cannot solve.

At a fixed point Omega of Alg. 1, with G the smooth part's gradient (Alg. 1 step 4):
  G_ii = 0 on the diagonal (it is not thresholded);
  G_ij = -lambda1 sign(w_ij) on the off-diagonal support;
  |G_ij| <= lambda1 off the support.
"""
import numpy as np

import oracle


def sample_pairs(omega_csr, rng, rows=48, hubs=16, per_row=24, random_pairs=800, truth_csr=None):
    """Rows drawn at random plus the highest-degree rows. Each row contributes up to per_row
    of its support entries (always its diagonal) and, when truth_csr is given, those of the
    true pattern. Then random pairs are added. Returns (rows, cols) int64 arrays."""
    om = omega_csr.tocsr()
    om.sort_indices()
    p = om.shape[0]
    deg = np.diff(om.indptr)
    t = truth_csr.tocsr() if truth_csr is not None else None
    pick = np.unique(np.concatenate([rng.integers(0, p, rows), np.argsort(deg)[-hubs:]]))
    pr, pc = [], []
    for i in pick:
        sup = om.indices[om.indptr[i]:om.indptr[i + 1]]
        if t is not None:
            sup = np.union1d(sup, t.indices[t.indptr[i]:t.indptr[i + 1]])
        if sup.size > per_row:
            sup = np.union1d(rng.choice(sup, per_row, replace=False), [i])
        pr += [int(i)] * len(sup)
        pc += [int(j) for j in sup]
    pr += rng.integers(0, p, random_pairs).tolist()
    pc += rng.integers(0, p, random_pairs).tolist()
    return np.asarray(pr, np.int64), np.asarray(pc, np.int64)


def residuals(X, omega_csr, lam1, lam2, rows, cols):
    """(diagonal, support, off-support excess, number of off-diagonal support pairs):
    max |G_ii|, max |G_ij + lambda1 sign(w_ij)| over the off-diagonal support, and
    max(|G_ij| - lambda1, 0) off the support, over the given pairs."""
    om = omega_csr.tocsr()
    om.sort_indices()
    G = oracle.gradient_entries(X, om, lam2, rows, cols)
    wv = np.asarray(om[rows, cols]).ravel()
    on = wv != 0
    diag = rows == cols
    d = float(np.max(np.abs(G[on & diag]), initial=0.0))
    sup = on & ~diag
    s = float(np.max(np.abs(G[sup] + lam1 * np.sign(wv[sup])), initial=0.0))
    o = float(np.max(np.abs(G[~on]) - lam1, initial=0.0))
    return d, s, max(o, 0.0), int(sup.sum())
