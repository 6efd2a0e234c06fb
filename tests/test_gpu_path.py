"""Regularisation path (hpc_solve_path): every warm-started point equals the oracle's
cold solve at that lambda1 (the minimiser is unique for lambda2 > 0), on a descending
grid like the one the batched-path workload uses (log-spaced lambda1, fixed lambda2)."""
import numpy as np
import pytest

import oracle
from workloads import small_problem

pytestmark = pytest.mark.gpu


def test_path_points_match_cold_oracle_solves(lib):
    import torch

    p, n, lam2 = 320, 220, 0.1
    X = small_problem(p, n, 4.0, 31).astype(np.float32)
    S = oracle.gram(X)
    grid = np.logspace(np.log10(0.4), np.log10(0.08), 6)
    with lib.Solver(torch.as_tensor(X).cuda(), grid[0], lam2, precision=lib.PREC_FP32, eps=1e-7,
                    max_iter=20000) as s:
        pts, ests = s.solve_path(grid, lam2)
    cold_iters = 0
    for t, lam1 in enumerate(grid):
        ref = oracle.solve(S, lam1, lam2, eps=1e-9, max_iter=20000)
        cold_iters += ref.iterations
        om = ests[t].to_scipy(p).toarray()
        assert pts[t]["status"] == 0 and pts[t]["lambda1"] == lam1
        assert pts[t]["nnz"] == ests[t].col.size
        err = np.linalg.norm(om - ref.omega) / np.linalg.norm(ref.omega)
        assert err < 1e-5, (t, lam1, err)
    # the path gets denser as lambda1 decreases
    nnz = [q["nnz"] for q in pts]
    assert nnz == sorted(nnz)


def test_path_without_estimates_and_bad_arguments(lib):
    import torch

    X = small_problem(100, 80, 3.0, 2).astype(np.float32)
    with lib.Solver(torch.as_tensor(X).cuda(), 0.3, 0.1, precision=lib.PREC_FP32) as s:
        pts, none = s.solve_path([0.3, 0.2], 0.1, return_estimates=False)
        assert none is None and len(pts) == 2 and all(q["status"] == 0 for q in pts)
        with pytest.raises(lib.HpcError) as e:
            s.solve_path([0.2, -1.0], 0.1)
        assert e.value.status == lib.ERR_ARG
