"""GPU solver vs the FP64 oracle, through the C ABI, on seeded small problems.

Sizes are chosen so the oracle finishes in seconds while the GPU path still
spans several 128-column screening blocks, several line-search blocks and a
ragged tail (p not a multiple of 128).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from tests.support import support_diff_ok
from workloads import WORKLOADS, make_x, small_problem

pytestmark = pytest.mark.gpu

FP32_REL = 1e-5          # ||Omega - Omega_ref||_F / ||Omega_ref||_F, FP32 path
FP64_REL = 1e-7          # FP64 path (the FP64 oracle itself is decided to ~1e-8)
THRESH_BAND = 1e-6       # support may differ only within this band of the threshold


def _torch():
    import torch

    assert torch.cuda.is_available()
    return torch


def _support_diff_ok(om_gpu, om_ref, S, lam1, lam2):
    """Support identical except entries of the reference within THRESH_BAND of the threshold."""
    return support_diff_ok(om_gpu, om_ref, lam1, lam2, S=S, band=THRESH_BAND)


def _solve_gpu(lib, X, lam1, lam2, **opt):
    torch = _torch()
    Xt = torch.as_tensor(X).cuda()
    with lib.Solver(Xt, lam1, lam2, **opt) as s:
        st = s.solve()
        om = s.omega_dense()
        stats = st.as_dict()
    return om, stats


# ------------------------------------------------------------------ Gram

@pytest.mark.parametrize("n,p", [(257, 300), (64, 129), (1, 5), (1000, 1)])
def test_gram_fp32_elementwise(lib, n, p):
    torch = _torch()
    rng = np.random.default_rng(n * 7 + p)
    X = rng.standard_normal((n, p)).astype(np.float32)
    S = torch.full((p, p + 3), float("nan"), dtype=torch.float32, device="cuda")
    lib.gram(torch.as_tensor(X).cuda(), S, precision=lib.PREC_FP32)
    torch.cuda.synchronize()
    got = S[:, :p].double().cpu().numpy()
    ref = oracle.gram(X)
    d = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    # rigorous FP32 bound |dS_ij| <= n u sqrt(S_ii S_jj) with u = 2^-24, plus the division
    bound = (n + 2) * 2.0 ** -24 * d + 1e-30
    assert np.all(np.abs(got - ref) <= bound)
    assert np.array_equal(got, got.T)
    assert torch.isnan(S[:, p:]).all()          # padding columns untouched


def test_gram_fp64_elementwise(lib):
    torch = _torch()
    rng = np.random.default_rng(1)
    X = rng.standard_normal((250, 500))
    S = torch.empty((500, 500), dtype=torch.float64, device="cuda")
    lib.gram(torch.as_tensor(X).cuda(), S, precision=lib.PREC_FP64)
    torch.cuda.synchronize()
    got = S.cpu().numpy()
    ref = oracle.gram(X)
    assert np.allclose(got, ref, rtol=1e-13, atol=1e-14)
    assert np.array_equal(got, got.T)


# ------------------------------------------------------------------ solves

def test_fp64_tridiagonal_p500(lib):
    """The FP64 workload (p=500, n=250, tridiagonal Omega0, lambda = (0.3, 0.2))."""
    w = WORKLOADS["fp64_p500"]
    X = make_x(w)
    S = oracle.gram(X)
    ref = oracle.solve(S, w.lambda1, w.lambda2, eps=1e-9, max_iter=20000)
    assert ref.status in ("converged", "floor")
    om, st = _solve_gpu(lib, X, w.lambda1, w.lambda2, value_dtype=lib.F64, precision=lib.PREC_FP64,
                        eps=1e-10, max_iter=20000)
    assert st["status"] == 0
    err = np.linalg.norm(om - ref.omega) / np.linalg.norm(ref.omega)
    assert err < FP64_REL, err
    ok, info = _support_diff_ok(om, ref.omega, S, w.lambda1, w.lambda2)
    assert ok, info
    assert np.array_equal(om, om.T)


def test_fp64_eps_1e6_matches_oracle_trajectory(lib):
    """At the workload's eps = 1e-6 both stop after the same number of iterations."""
    w = WORKLOADS["fp64_p500"]
    X = make_x(w)
    S = oracle.gram(X)
    ref = oracle.solve(S, w.lambda1, w.lambda2, eps=w.eps)
    om, st = _solve_gpu(lib, X, w.lambda1, w.lambda2, value_dtype=lib.F64, precision=lib.PREC_FP64, eps=w.eps)
    assert st["iterations"] == ref.iterations
    assert st["ls_trials"] == sum(ref.trials)
    assert np.linalg.norm(om - ref.omega) / np.linalg.norm(ref.omega) < 1e-10
    assert st["F"] == pytest.approx(ref.F[-2], rel=1e-12)      # F at the last gradient pass


@pytest.mark.parametrize("p,n,seed,degree,lam1,lam2", [
    (1000, 700, 0, 5.0, 0.2, 0.1),
    (333, 150, 1, 3.0, 0.12, 0.1),     # p > n
    (700, 2000, 2, 8.0, 0.15, 0.05),
])
def test_fp32_solve_matches_oracle(lib, p, n, seed, degree, lam1, lam2):
    X = small_problem(p, n, degree, seed).astype(np.float32)
    S = oracle.gram(X)
    ref = oracle.solve(S, lam1, lam2, eps=1e-9, max_iter=20000)
    assert ref.status in ("converged", "floor")
    om, st = _solve_gpu(lib, X, lam1, lam2, precision=lib.PREC_FP32, eps=1e-7, max_iter=20000)
    assert st["status"] == 0, st
    err = np.linalg.norm(om - ref.omega) / np.linalg.norm(ref.omega)
    assert err < FP32_REL, err
    ok, info = _support_diff_ok(om, ref.omega, S, lam1, lam2)
    assert ok, info
    assert np.array_equal(om, om.T)          # bitwise symmetric iterates


def test_fp32_first_iterations_follow_oracle(lib):
    """Iterate by iterate, the GPU takes the oracle's steps (same tau) for the first iterations."""
    torch = _torch()
    p, n = 400, 300
    X = small_problem(p, n, 4.0, 5).astype(np.float32)
    S = oracle.gram(X)
    lam1, lam2 = 0.1, 0.1
    with lib.Solver(torch.as_tensor(X).cuda(), lam1, lam2, precision=lib.PREC_FP32) as s:
        Om = np.eye(p)
        W = oracle.times_S(Om, S)
        for k in range(6):
            step = oracle.iterate(S, Om, W, lam1, lam2)
            st = s.iterate(1)
            assert st.accepted_halvings == round(-np.log2(step.tau))
            got = s.omega_dense()
            err = np.linalg.norm(got - step.omega) / np.linalg.norm(step.omega)
            assert err < 1e-5, (k, err)
            Om, W = step.omega, step.W


@pytest.mark.parametrize("p,n,f64", [
    (600, 400, False),      # 5 column blocks: the per-block mask and selection
    (1024, 500, False),     # 8 blocks of 128: the 16-byte (8-block) vector forms
    (512, 300, True),       # FP64, 8 blocks of 64: the vector forms in double
])
def test_screened_gradient_matches_oracle(lib, p, n, f64):
    """After a few iterations: G on every reported candidate equals the oracle's G, and every
    entry outside the candidate set has w_ij = 0 and |G_ij| <= lambda1 (the bound screening
    skipped no block that can emit)."""
    torch = _torch()
    X = small_problem(p, n, 5.0, 8).astype(np.float64 if f64 else np.float32)
    S = oracle.gram(X)
    lam1, lam2 = 0.08, 0.1
    opt = dict(value_dtype=lib.F64, precision=lib.PREC_FP64) if f64 else dict(precision=lib.PREC_FP32)
    with lib.Solver(torch.as_tensor(X).cuda(), lam1, lam2, **opt) as s:
        s.iterate(4)
        om_before = None
        # candidates belong to the gradient pass at the iterate *before* the last accept
        s2 = lib.Solver(torch.as_tensor(X).cuda(), lam1, lam2, **opt)
        s2.iterate(3)
        om_before = s2.omega_dense()
        s2.close()
        r, c, o, g = s.candidates()
    G = oracle.gradient(om_before, oracle.times_S(om_before, S), lam2)
    scale = np.abs(G).max()
    assert np.allclose(o, om_before[r, c], rtol=1e-6, atol=1e-7)
    assert np.max(np.abs(g - G[r, c])) < 2e-5 * scale
    mask = np.zeros((p, p), bool)
    mask[r, c] = True
    assert np.array_equal(mask, mask.T)
    outside = ~mask
    assert np.all(om_before[outside] == 0)
    assert np.all(np.abs(G[outside]) <= lam1 + 2e-5 * scale)
    assert np.all(np.diag(mask))


# ------------------------------------------------------------------ edge cases

def test_p1_closed_form(lib):
    torch = _torch()
    X = np.array([[1.0], [2.0], [-1.0], [0.5]], np.float32)
    s = float(np.mean(X[:, 0].astype(np.float64) ** 2))
    om, st = _solve_gpu(lib, X, 0.3, 0.2, precision=lib.PREC_FP32, eps=1e-7)
    assert om.shape == (1, 1)
    assert om[0, 0] == pytest.approx(1 / np.sqrt(s + 0.2), rel=1e-5)


def test_diagonal_solution_above_lambda_max(lib):
    X = small_problem(150, 80, 3.0, 3).astype(np.float32)
    S = oracle.gram(X)
    lam2 = 0.1
    w = 1 / np.sqrt(np.diag(S) + lam2)
    M = 0.5 * np.abs(S) * (w[:, None] + w[None, :])
    np.fill_diagonal(M, 0)
    om, st = _solve_gpu(lib, X, M.max() * 1.01, lam2, precision=lib.PREC_FP32, eps=1e-7)
    assert np.count_nonzero(om - np.diag(np.diag(om))) == 0
    assert np.allclose(np.diag(om), w, rtol=2e-5)


def test_lambda1_zero_dense_solution_grows_capacity(lib):
    """lambda1 = 0 makes every entry a candidate: the buffers must grow past the default."""
    p, n = 200, 400
    X = small_problem(p, n, 3.0, 4).astype(np.float32)
    S = oracle.gram(X)
    ref = oracle.solve(S, 0.0, 0.3, eps=1e-9, max_iter=20000)
    om, st = _solve_gpu(lib, X, 0.0, 0.3, precision=lib.PREC_FP32, eps=1e-7, capacity=2 * p)
    assert st["capacity_regrows"] >= 1
    assert np.linalg.norm(om - ref.omega) / np.linalg.norm(ref.omega) < FP32_REL


def test_warm_start_and_set_lambda(lib):
    """set_lambda + a warm start reach the same fixed point as a cold solve (unique minimiser)."""
    torch = _torch()
    X = small_problem(300, 200, 4.0, 6).astype(np.float32)
    Xt = torch.as_tensor(X).cuda()
    with lib.Solver(Xt, 0.3, 0.1, precision=lib.PREC_FP32, eps=1e-7) as s:
        s.solve()
        s.set_lambda(0.15, 0.1)
        s.solve()
        warm = s.omega_dense()
    cold, _ = _solve_gpu(lib, X, 0.15, 0.1, precision=lib.PREC_FP32, eps=1e-7)
    assert np.linalg.norm(warm - cold) / np.linalg.norm(cold) < 2 * FP32_REL


def test_set_and_get_omega_roundtrip_and_checks(lib):
    torch = _torch()
    X = small_problem(50, 40, 2.0, 1).astype(np.float32)
    with lib.Solver(torch.as_tensor(X).cuda(), 0.2, 0.1, precision=lib.PREC_FP32) as s:
        s.solve()
        csr = s.get_omega()
        s.set_omega(csr)
        again = s.get_omega()
        assert np.array_equal(csr.row_ptr, again.row_ptr) and np.array_equal(csr.col, again.col)
        assert np.allclose(csr.val, again.val, rtol=0, atol=0)
        bad = lib.Csr(csr.row_ptr.copy(), csr.col.copy(), csr.val.copy())
        bad.val[csr.row_ptr[3] + list(csr.col[csr.row_ptr[3]:csr.row_ptr[4]]).index(3)] = -1.0
        with pytest.raises(lib.HpcError) as e:
            s.set_omega(bad)
        assert e.value.status == lib.ERR_NONPOS_DIAG
        # device-side export
        rp = torch.empty(51, dtype=torch.int64, device="cuda")
        ci = torch.empty(csr.col.size, dtype=torch.int32, device="cuda")
        v = torch.empty(csr.col.size, dtype=torch.float32, device="cuda")
        m = s.get_omega_device(rp, ci, v)
        assert m == csr.col.size
        assert np.array_equal(rp.cpu().numpy(), csr.row_ptr)


def test_invalid_arguments(lib):
    torch = _torch()
    X = torch.zeros((4, 3), device="cuda")
    for kw in ({"eps": 0.0}, {"ls_window": 3}, {"max_halvings": -1}):
        with pytest.raises(lib.HpcError) as e:
            lib.Solver(X, 0.1, 0.1, **kw)
        assert e.value.status == lib.ERR_ARG
    with pytest.raises(lib.HpcError):
        lib.Solver(X, -0.1, 0.1)
    with pytest.raises(lib.HpcError):
        lib.Solver(X, 0.1, float("nan"))


def test_nan_input_reports_nan(lib):
    torch = _torch()
    X = small_problem(40, 30, 2.0, 2).astype(np.float32)
    X[3, 5] = np.nan
    with lib.Solver(torch.as_tensor(X).cuda(), 0.1, 0.1, precision=lib.PREC_FP32) as s:
        with pytest.raises(lib.HpcError) as e:
            s.solve()
        assert e.value.status == lib.ERR_NAN
