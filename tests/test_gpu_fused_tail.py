"""The fused iteration tail (tuning fused_tail = 1) against the chain of separate
kernels it replaces (fused_tail = 0, the default).

The tail builds the candidate structure, forms G on it (Alg. 2 steps 5-6),
evaluates the line-search windows with the prox of eq. (2) and takes the
sufficient-decrease decision of Alg. 1 step 9, then compacts the accepted iterate
and applies the stopping rule.  fused_tail = 1 runs all of it as one cooperative
kernel, with grid-wide barriers where the chain has kernel boundaries.  Each step
runs the same device code, so with the same line-search grid (ls_blocks_per_sm
fixed for both) the windows' partial sums are grouped the same way and iterates,
step sizes and iteration counts must agree bit for bit.  The objective value F
comes from partials grouped by the grid of the gradient step, which differs
between the two, so it agrees to rounding only.
"""
import numpy as np
import pytest

import oracle
from tests.support import support_diff_ok
from workloads import small_problem

pytestmark = pytest.mark.gpu


def _solve(lib, X, lam1, lam2, tuning, k=None, **opt):
    import torch

    with lib.Solver(torch.as_tensor(X).cuda(), lam1, lam2, **opt) as s:
        s.set_tuning(**tuning)
        st = s.solve() if k is None else s.iterate(k)
        return s.omega_dense(), st.as_dict()


def _same(a, b):
    om_a, st_a = a
    om_b, st_b = b
    assert np.array_equal(om_a, om_b)
    for key in ("iterations", "ls_trials", "nnz", "status", "accepted_halvings"):
        assert st_a[key] == st_b[key], key
    assert st_a["F"] == pytest.approx(st_b["F"], rel=1e-12)


def _opt(lib, dtype, loop, **kw):
    f64 = dtype == np.float64
    return dict(value_dtype=lib.F64 if f64 else lib.F32, precision=lib.PREC_FP64 if f64 else lib.PREC_FP32,
                eps=1e-10 if f64 else 1e-7, max_iter=20000, device_loop=loop, **kw)


@pytest.mark.parametrize("p,n,dtype,loop,window", [
    (300, 200, np.float32, 1, 8),
    (300, 200, np.float32, 0, 8),
    (129, 90, np.float32, 1, 1),       # one tau per window: many windows per iteration
    (260, 180, np.float32, 1, 4),
    (200, 150, np.float64, 1, 8),
    (200, 150, np.float64, 0, 16),
])
def test_fused_tail_matches_chain_and_oracle(lib, p, n, dtype, loop, window):
    X = small_problem(p, n, 4.0, seed=p + 5).astype(dtype)
    opt = _opt(lib, dtype, loop)
    fused = _solve(lib, X, 0.15, 0.1, dict(fused_tail=1, ls_blocks_per_sm=2, ls_window=window), **opt)
    chain = _solve(lib, X, 0.15, 0.1, dict(fused_tail=0, ls_blocks_per_sm=2, ls_window=window), **opt)
    _same(fused, chain)
    assert fused[1]["status"] == 0
    # one launch instead of the chain's candidate, window and accept kernels
    assert fused[1]["kernel_launches"] < chain[1]["kernel_launches"]
    ref = oracle.solve(oracle.gram(X.astype(np.float64)), 0.15, 0.1, eps=1e-9, max_iter=20000)
    rel = np.linalg.norm(fused[0] - ref.omega) / np.linalg.norm(ref.omega)
    assert rel < (1e-7 if dtype == np.float64 else 1e-5)
    ok, detail = support_diff_ok(fused[0], ref.omega, 0.15, 0.1, X=X)
    assert ok, detail


def test_fused_tail_multi_tile_scans(lib):
    """p = 9000 rows: three tiles of the row-count scans inside the fused launch
    (iid normal X: a fast draw; the comparison needs no oracle)."""
    X = np.random.default_rng(21).standard_normal((2500, 9000)).astype(np.float32)
    opt = _opt(lib, np.float32, 1)
    fused = _solve(lib, X, 0.2, 0.1, dict(fused_tail=1, ls_blocks_per_sm=2), k=12, **opt)
    chain = _solve(lib, X, 0.2, 0.1, dict(fused_tail=0, ls_blocks_per_sm=2), k=12, **opt)
    _same(fused, chain)
    assert fused[1]["iterations"] == 12


def test_fused_tail_capacity_regrow(lib):
    """Overflowing candidate buffers raise a flag inside the fused launch; every
    later step of it is skipped, the host grows the buffers and the repeated
    iteration gives the chain's result."""
    X = small_problem(300, 120, 6.0, seed=5).astype(np.float32)
    opt = _opt(lib, np.float32, 1, capacity=300)
    opt["eps"] = 1e-6
    fused = _solve(lib, X, 0.05, 0.1, dict(fused_tail=1, ls_blocks_per_sm=2), **opt)
    chain = _solve(lib, X, 0.05, 0.1, dict(fused_tail=0, ls_blocks_per_sm=2), **opt)
    _same(fused, chain)
    assert fused[1]["capacity_regrows"] >= 1


def test_fused_tail_obs_matches_oracle(lib):
    """The Obs form of the window evaluation (Alg. 3) inside the fused launch."""
    X = small_problem(300, 200, 4.0, seed=17).astype(np.float32)
    opt = _opt(lib, np.float32, 1, variant=lib.OBS)
    fused = _solve(lib, X, 0.15, 0.1, dict(fused_tail=1), **opt)
    chain = _solve(lib, X, 0.15, 0.1, dict(fused_tail=0), **opt)
    assert fused[1]["status"] == 0
    ref = oracle.solve(oracle.gram(X.astype(np.float64)), 0.15, 0.1, eps=1e-9, max_iter=20000)
    for om in (fused[0], chain[0]):
        rel = np.linalg.norm(om - ref.omega) / np.linalg.norm(ref.omega)
        assert rel < 1e-5
        ok, detail = support_diff_ok(om, ref.omega, 0.15, 0.1, X=X)
        assert ok, detail
    assert fused[1]["kernel_launches"] < chain[1]["kernel_launches"]


def test_fused_tail_path_matches_chain(lib):
    """The lambda1 path in one graph launch (each point's iteration loop with the fused
    tail in its body) gives the chain's points: same iterations, trials and estimates."""
    import torch

    p, n, lam2 = 320, 220, 0.1
    X = small_problem(p, n, 4.0, 31).astype(np.float32)
    grid = np.logspace(np.log10(0.4), np.log10(0.08), 6)
    out = []
    for form in (1, 0):
        with lib.Solver(torch.as_tensor(X).cuda(), grid[0], lam2, precision=lib.PREC_FP32, eps=1e-7,
                        max_iter=20000) as s:
            s.set_tuning(fused_tail=form, ls_blocks_per_sm=2)
            out.append(s.solve_path(grid, lam2))
    (pf, ef), (pc, ec) = out
    for t in range(len(grid)):
        for key in ("status", "iterations", "ls_trials", "nnz"):
            assert pf[t][key] == pc[t][key], (t, key)
        assert np.array_equal(ef[t].row_ptr, ec[t].row_ptr) and np.array_equal(ef[t].col, ec[t].col)
        assert np.array_equal(ef[t].val, ec[t].val)
