"""Batched solves of independent problems (hpc_solve_batch): every problem against the oracle,
and the batch bitwise equal to solving the same problems one after another (the kernels are
deterministic and the problems share nothing)."""
import numpy as np
import pytest

import oracle
from tests.support import support_diff_ok
from workloads import BATCH_PROBLEMS, omega0_banded, make_x, sample_x_cpu

pytestmark = pytest.mark.gpu


def _problem(p, n, seed):
    return sample_x_cpu(omega0_banded(p, 3, seed), n, seed).astype(np.float32)


@pytest.mark.parametrize("device_loop", [1, 0])
def test_batch_of_uneven_problems_matches_oracle_and_sequential(lib, device_loop):
    """device_loop=1: the whole batch is one graph launch; 0: a host thread pool."""
    import torch

    shapes = [(120, 60), (200, 100), (257, 128), (300, 150), (384, 192), (500, 250)]
    Xs = [_problem(p, n, 10 + t) for t, (p, n) in enumerate(shapes)]
    lam1, lam2 = 0.15, 0.1
    streams = [torch.cuda.Stream() for _ in shapes]
    solvers = [lib.Solver(torch.as_tensor(X).cuda(), lam1, lam2, stream=st, precision=lib.PREC_FP32, eps=1e-7,
                          max_iter=20000, device_loop=device_loop) for X, st in zip(Xs, streams)]
    stats = lib.solve_batch(solvers)
    batch = [s.get_omega() for s in solvers]
    for s in solvers:
        s.close()
    assert all(st["status"] == 0 for st in stats)
    for (p, n), X, est in zip(shapes, Xs, batch):
        S = oracle.gram(X)
        ref = oracle.solve(S, lam1, lam2, eps=1e-9, max_iter=20000)
        om = est.to_scipy(p).toarray()
        assert np.linalg.norm(om - ref.omega) / np.linalg.norm(ref.omega) < 1e-5
        ok, detail = support_diff_ok(om, ref.omega, lam1, lam2, S=S)
        assert ok, (p, detail)
    # sequential, default stream
    for X, est in zip(Xs, batch):
        with lib.Solver(torch.as_tensor(X).cuda(), lam1, lam2, precision=lib.PREC_FP32, eps=1e-7,
                        max_iter=20000) as s:
            s.solve()
            seq = s.get_omega()
        assert np.array_equal(seq.row_ptr, est.row_ptr) and np.array_equal(seq.col, est.col)
        assert np.array_equal(seq.val, est.val)


def test_batch_thread_limit_and_errors(lib):
    import torch

    Xs = [_problem(100, 50, 20 + t) for t in range(3)]
    solvers = [lib.Solver(torch.as_tensor(X).cuda(), 0.15, 0.1, stream=torch.cuda.Stream(),
                          precision=lib.PREC_FP32, device_loop=0) for X in Xs]
    stats = lib.solve_batch(solvers, threads=2)
    assert len(stats) == 3 and all(st["iterations"] > 0 for st in stats)
    for s in solvers:
        s.close()


def test_batch_launch_with_overflow_and_shared_stream(lib):
    """One graph launch: a handle with a tiny candidate capacity overflows, grows and
    finishes alone; two handles on one stream; a handle with max_iter = 0.  Every
    result equals the same handle's plain solve."""
    import torch

    Xs = [_problem(180, 90, 30 + t) for t in range(4)]
    st_shared = torch.cuda.Stream()
    opts = [dict(capacity=200), dict(), dict(), dict(max_iter=0)]
    streams = [torch.cuda.Stream(), st_shared, st_shared, torch.cuda.Stream()]
    solvers = [lib.Solver(torch.as_tensor(X).cuda(), 0.08, 0.1, stream=st, precision=lib.PREC_FP32, eps=1e-7, **o)
               for X, st, o in zip(Xs, streams, opts)]
    stats = lib.solve_batch(solvers)
    ests = [s.get_omega() for s in solvers]
    for s in solvers:
        s.close()
    assert stats[0]["capacity_regrows"] >= 1
    assert stats[3]["status"] == 1 and stats[3]["iterations"] == 0
    for X, o, est, st in list(zip(Xs, opts, ests, stats))[:3]:
        with lib.Solver(torch.as_tensor(X).cuda(), 0.08, 0.1, precision=lib.PREC_FP32, eps=1e-7, **o) as s:
            ref = s.solve().as_dict()
            seq = s.get_omega()
        assert st["iterations"] == ref["iterations"] and st["ls_trials"] == ref["ls_trials"]
        assert np.array_equal(seq.col, est.col) and np.array_equal(seq.val, est.val)


@pytest.mark.slow
def test_sixteen_problem_workload(lib):
    """p = 1024 k, k = 1..16, n = p/2, banded: the batch equals sequential solves bitwise and
    the two smallest problems match the oracle."""
    import torch

    Xs = [make_x(w, device="cuda") for w in BATCH_PROBLEMS]
    streams = [torch.cuda.Stream() for _ in BATCH_PROBLEMS]
    solvers = [lib.Solver(X, w.lambda1, w.lambda2, stream=st, precision=lib.PREC_BF16X3, eps=w.eps,
                          max_iter=20000) for X, w, st in zip(Xs, BATCH_PROBLEMS, streams)]
    torch.cuda.synchronize()
    stats = lib.solve_batch(solvers)
    ests = [s.get_omega() for s in solvers]
    for s in solvers:
        s.close()
    assert all(st["status"] == 0 for st in stats)
    for X, w, est in list(zip(Xs, BATCH_PROBLEMS, ests))[:2]:
        S = oracle.gram(X.cpu().numpy())
        ref = oracle.solve(S, w.lambda1, w.lambda2, eps=1e-9, max_iter=20000)
        om = est.to_scipy(w.p).toarray()
        assert np.linalg.norm(om - ref.omega) / np.linalg.norm(ref.omega) < 1e-5
        ok, detail = support_diff_ok(om, ref.omega, w.lambda1, w.lambda2, S=S)
        assert ok, (w.p, detail)
    for X, w, est in list(zip(Xs, BATCH_PROBLEMS, ests))[::5]:
        with lib.Solver(X, w.lambda1, w.lambda2, precision=lib.PREC_BF16X3, eps=w.eps, max_iter=20000) as s:
            s.solve()
            seq = s.get_omega()
        assert np.array_equal(seq.col, est.col) and np.array_equal(seq.val, est.val)
