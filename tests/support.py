"""The support rule of the parity bar, shared by every oracle comparison: the estimate's
support equals the reference's except for entries within `band` of the soft-threshold
(eq. (2)).  A soft-thresholded value is the distance of its argument past the threshold,
so an entry on one side only is within the band when
- it is in the reference only: |w_ref,ij| <= band;
- it is in the estimate only: |w_ij| <= band, or ||G_ij| - lambda1| <= band with G the
  smooth part's gradient at the reference (Alg. 1 step 4, formed by the oracle): the
  reference's own argument sits at the threshold."""
import numpy as np

import oracle

BAND = 1e-6


def support_diff_ok(om_gpu, om_ref, lam1, lam2, S=None, X=None, band=BAND):
    """(ok, detail) for dense p x p estimates; S, or X (then S = X^T X / n), gives G.
    detail is the number of differing entries, or the first entry that breaks the rule."""
    om_gpu = np.asarray(om_gpu, dtype=np.float64)
    om_ref = np.asarray(om_ref, dtype=np.float64)
    a = om_gpu != 0
    b = om_ref != 0
    diff = np.argwhere(a != b)
    if diff.size == 0:
        return True, 0
    if S is None:
        S = oracle.gram(np.asarray(X, dtype=np.float64))
    G = oracle.gradient(om_ref, oracle.times_S(om_ref, S), lam2)
    for i, j in diff:
        if b[i, j]:
            near = abs(om_ref[i, j]) <= band
        else:
            near = abs(om_gpu[i, j]) <= band or abs(abs(G[i, j]) - lam1) <= band
        if not near:
            return False, (int(i), int(j), float(om_gpu[i, j]), float(om_ref[i, j]), float(G[i, j]))
    return True, len(diff)
