"""Regularisation path (hpc_solve_path): every warm-started point equals the oracle's
cold solve at that lambda1 (the minimiser is unique for lambda2 > 0), on a descending
grid like the one the batched-path workload uses (log-spaced lambda1, fixed lambda2)."""
import numpy as np
import pytest

import oracle
from tests.support import support_diff_ok
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
        ok, detail = support_diff_ok(om, ref.omega, lam1, lam2, S=S)
        assert ok, (t, lam1, detail)
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


def _path(lib, X, grid, lam2, **opt):
    import torch

    with lib.Solver(torch.as_tensor(X).cuda(), grid[0], lam2, precision=lib.PREC_FP32, eps=1e-7, max_iter=20000,
                    **opt) as s:
        return s.solve_path(grid, lam2)


def test_path_in_one_launch_matches_the_host_driven_path(lib):
    """device_loop=1 runs the whole grid as one graph launch (an outer WHILE over the
    points); it must give the host-driven path's points and estimates bit for bit."""
    X = small_problem(260, 200, 4.0, 33).astype(np.float32)
    grid = np.logspace(np.log10(0.5), np.log10(0.06), 9)
    pd, ed = _path(lib, X, grid, 0.1, device_loop=1)
    ph, eh = _path(lib, X, grid, 0.1, device_loop=0)
    for a, b in zip(pd, ph):
        for key in ("lambda1", "iterations", "ls_trials", "nnz", "status", "F", "rel_change"):
            assert a[key] == b[key], key
        assert a["ms"] > 0
    for a, b in zip(ed, eh):
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col, b.col)
        assert np.array_equal(a.val, b.val)


@pytest.mark.parametrize("device_loop", [0, 1])
def test_path_estimate_capacity_and_iteration_limit(lib, device_loop):
    import torch

    X = small_problem(150, 120, 3.0, 5).astype(np.float32)
    grid = [0.4, 0.2, 0.1]
    with lib.Solver(torch.as_tensor(X).cuda(), 0.4, 0.1, precision=lib.PREC_FP32, device_loop=device_loop) as s:
        with pytest.raises(lib.HpcError) as e:
            s.solve_path(grid, 0.1, capacity=200)        # less than the first estimate (>= 150 diagonal entries + ...)
        assert e.value.status == lib.ERR_CAPACITY
    with lib.Solver(torch.as_tensor(X).cuda(), 0.4, 0.1, precision=lib.PREC_FP32, device_loop=device_loop,
                    eps=1e-12, max_iter=3) as s:
        pts, ests = s.solve_path(grid, 0.1)
        assert [q["status"] for q in pts] == [1, 1, 1]   # HPC_NOT_CONVERGED at every point, the path goes on
        assert [q["iterations"] for q in pts] == [3, 3, 3]
