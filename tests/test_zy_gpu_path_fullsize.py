"""Parity of the lambda1 path at its full size: the 32 points of path_p8192 (p = 8192,
n = 4096, lambda1 log-spaced over [0.05, 0.8], lambda2 = 0.1), built and solved the way
bench.py --row path times it (BF16X3 Gram, the whole path one graph launch).

The FP64 oracle cannot solve this problem, so the checks are:
- every point converges (status 0);
- each estimate is symmetric with a positive diagonal;
- at the sparsest, the middle and the densest points, the optimality conditions of the
  prox-gradient fixed point (eq. (2)) hold at sampled pairs, with G formed by the oracle
  from X (tests/kkt.py).

Stopping at ||dOmega||_F < eps ||Omega||_F (eps = 1e-6) leaves entrywise residuals far
below KKT_TOL. KKT_TOL is below the gap between neighbouring grid points: lambda1 changes
by 4.7e-3 or more per step. So an estimate warm-started from a neighbour but not moved to
its own lambda1 fails.
"""
import numpy as np
import pytest

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

KKT_TOL = 2e-3


def test_path_workload_full_size(lib):
    from tests import kkt
    from workloads import PATH_LAMBDA1, PATH_LAMBDA2, WORKLOADS, make_x, omega0_for

    w = WORKLOADS["path_p8192"]
    lam = sorted(PATH_LAMBDA1, reverse=True)
    X = make_x(w, device="cuda")
    with lib.Solver(X, lam[0], PATH_LAMBDA2, eps=w.eps, max_iter=100000) as s:
        pts, ests = s.solve_path(lam, PATH_LAMBDA2)
    assert [q["status"] for q in pts] == [0] * len(lam)
    Xh = X.cpu().numpy()
    truth = omega0_for(w)
    rng = np.random.default_rng(4)
    for t in (0, len(lam) // 2, len(lam) - 1):
        om = ests[t].to_scipy(w.p).tocsr()
        assert (om != om.T).nnz == 0
        assert np.all(om.diagonal() > 0)
        r, c = kkt.sample_pairs(om, rng, truth_csr=truth)
        d, sres, o, nsup = kkt.residuals(Xh, om, lam[t], PATH_LAMBDA2, r, c)
        assert max(d, sres, o) <= KKT_TOL, (t, lam[t], d, sres, o)
    assert nsup > 20            # the densest point's sample holds off-diagonal support entries
