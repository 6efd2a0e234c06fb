"""The device loop (one CUDA-graph launch per solve, conditional WHILE nodes for
the iterations and the line-search windows) against the host-driven loop.

Both run the same kernels on the same data in the same order; the device loop
only copies the accepted iterate where the host loop swaps buffers.  So the
iterates, iteration counts and step sizes must agree bit for bit, and the
device loop must also match the FP64 oracle like the host loop does.
"""
import numpy as np
import pytest

import oracle
from workloads import small_problem

pytestmark = pytest.mark.gpu


def _torch():
    import torch

    assert torch.cuda.is_available()
    return torch


def _run(lib, X, lam1, lam2, k=None, variant=None, **opt):
    torch = _torch()
    Xt = torch.as_tensor(X).cuda()
    kw = {} if variant is None else {"variant": variant}
    with lib.Solver(Xt, lam1, lam2, **kw, **opt) as s:
        st = s.solve() if k is None else s.iterate(k)
        return s.omega_dense(), st.as_dict()


def _same(a, b):
    om_a, st_a = a
    om_b, st_b = b
    assert np.array_equal(om_a, om_b)
    for key in ("iterations", "ls_trials", "nnz", "status", "accepted_halvings"):
        assert st_a[key] == st_b[key], key
    assert st_a["F"] == st_b["F"]
    assert st_a["rel_change"] == st_b["rel_change"]


@pytest.mark.parametrize("p,n,dtype", [(300, 200, np.float32), (129, 90, np.float32), (200, 150, np.float64)])
def test_device_loop_matches_host_loop(lib, p, n, dtype):
    X = small_problem(p, n, 4.0, seed=p + 11).astype(dtype)
    f64 = dtype == np.float64
    opt = dict(value_dtype=lib.F64 if f64 else lib.F32, precision=lib.PREC_FP64 if f64 else lib.PREC_FP32,
               eps=1e-10 if f64 else 1e-7, max_iter=20000)
    dev = _run(lib, X, 0.15, 0.1, device_loop=1, **opt)
    host = _run(lib, X, 0.15, 0.1, device_loop=0, **opt)
    _same(dev, host)
    assert dev[1]["status"] == 0
    ref = oracle.solve(oracle.gram(X), 0.15, 0.1, eps=1e-9, max_iter=20000)
    rel = np.linalg.norm(dev[0] - ref.omega) / np.linalg.norm(ref.omega)
    assert rel < (1e-7 if dtype == np.float64 else 1e-5)


def test_device_loop_iterate_k(lib):
    """hpc_iterate(k): exactly k iterations, no stopping rule, same as the host loop."""
    X = small_problem(260, 180, 5.0, seed=3).astype(np.float32)
    dev = _run(lib, X, 0.1, 0.1, k=5, device_loop=1)
    host = _run(lib, X, 0.1, 0.1, k=5, device_loop=0)
    _same(dev, host)
    assert dev[1]["iterations"] == 5


def test_device_loop_capacity_regrow(lib):
    """Overflowing candidate buffers end the graph launch; the host grows them,
    rebuilds the graph and the repeated iteration gives the host loop's result."""
    X = small_problem(300, 120, 6.0, seed=5).astype(np.float32)
    dev = _run(lib, X, 0.05, 0.1, eps=1e-6, capacity=300, device_loop=1)
    host = _run(lib, X, 0.05, 0.1, eps=1e-6, capacity=300, device_loop=0)
    _same(dev, host)
    assert dev[1]["capacity_regrows"] >= 1


def test_device_loop_max_iter_and_timing(lib):
    X = small_problem(256, 200, 4.0, seed=9).astype(np.float32)
    om, st = _run(lib, X, 0.1, 0.1, eps=1e-12, max_iter=4, device_loop=1, timing=1)
    assert st["status"] == 1 and st["iterations"] == 4      # HPC_NOT_CONVERGED at max_iter
    assert st["grad_pass_launches"] == 4
    assert st["ms_grad_pass"] > 0.0 and st["ms_total"] >= st["ms_grad_pass"]
    assert st["kernel_launches"] > 4 * 10


def test_device_loop_set_lambda_reuses_graph(lib):
    """lambda lives in the device control block: a new lambda needs no new graph
    and gives the same result as a fresh host-loop solve at that lambda."""
    torch = _torch()
    X = small_problem(200, 160, 4.0, seed=21).astype(np.float32)
    Xt = torch.as_tensor(X).cuda()
    with lib.Solver(Xt, 0.3, 0.1, device_loop=1, eps=1e-7) as s:
        s.solve()
        s.set_lambda(0.12, 0.1)
        st = s.solve().as_dict()
        om = s.omega_dense()
    with lib.Solver(Xt, 0.3, 0.1, device_loop=0, eps=1e-7) as s:
        s.solve()
        s.set_lambda(0.12, 0.1)
        st_h = s.solve().as_dict()
        om_h = s.omega_dense()
    _same((om, st), (om_h, st_h))


def test_device_loop_obs(lib):
    X = small_problem(256, 192, 4.0, seed=31).astype(np.float32)
    dev = _run(lib, X, 0.2, 0.1, variant=lib.OBS, eps=3e-7, device_loop=1)
    host = _run(lib, X, 0.2, 0.1, variant=lib.OBS, eps=3e-7, device_loop=0)
    _same(dev, host)
