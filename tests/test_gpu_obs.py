"""Obs variant (Alg. 3) through the C ABI: Y^T = Omega X^T, Z = Y X / n on tensor cores with
the paired-tile screening epilogue, and the line search on ||X D||^2 / n.  Its fixed point
is the Cov one (tr(Omega S Omega) = ||Omega X^T||^2 / n), so it is checked against the
oracle's estimate and against the GPU's own Cov solve.

Obs recomputes Z from a freshly rounded Y^T every iteration, and BF16X3 products carry
~2^-17 relative error, so the map has a noise floor: measured relative steps bottom out
near 1.6e-7 (p = 257, n = 100) while the estimate is within 1.3e-6 of the oracle's.  The
solves here therefore stop at eps = 3e-7 and a stop at max_iter is accepted when the
last step is below 1e-6."""
import numpy as np
import pytest

import oracle
from tests.support import support_diff_ok
from workloads import WORKLOADS, make_x, small_problem

pytestmark = pytest.mark.gpu


def _solve(lib, X, lam1, lam2, variant, **kw):
    import torch

    with lib.Solver(torch.as_tensor(X).cuda(), lam1, lam2, variant=variant, eps=3e-7, max_iter=3000, **kw) as s:
        st = s.solve().as_dict()
        return s.omega_dense(), st


def _stopped_ok(st):
    return st["status"] == 0 or (st["status"] == 1 and st["rel_change"] < 1e-6)


@pytest.mark.parametrize("p,n,seed,lam1", [(300, 150, 0, 0.12), (257, 100, 1, 0.1), (400, 500, 2, 0.15)])
def test_obs_matches_oracle(lib, p, n, seed, lam1):
    lam2 = 0.1
    X = small_problem(p, n, 4.0, 60 + seed).astype(np.float32)
    ref = oracle.solve(oracle.gram(X), lam1, lam2, eps=1e-9, max_iter=20000)
    om, st = _solve(lib, X, lam1, lam2, lib.OBS, precision=lib.PREC_BF16X3)
    assert _stopped_ok(st), st
    err = np.linalg.norm(om - ref.omega) / np.linalg.norm(ref.omega)
    assert err < 1e-5, err
    ok, detail = support_diff_ok(om, ref.omega, lam1, lam2, X=X)
    assert ok, detail
    assert np.array_equal(om, om.T)


def test_obs_and_cov_reach_the_same_estimate(lib):
    X = small_problem(350, 200, 4.0, 70).astype(np.float32)
    a, sa = _solve(lib, X, 0.12, 0.1, lib.COV, precision=lib.PREC_BF16X3)
    b, sb = _solve(lib, X, 0.12, 0.1, lib.OBS, precision=lib.PREC_BF16X3)
    assert _stopped_ok(sa) and _stopped_ok(sb)
    assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-5
    assert np.array_equal(a != 0, b != 0)


def test_obs_tf32_runs_and_is_close(lib):
    """TF32 keeps 10 mantissa bits per input: reported, not held to the FP32 tolerance."""
    X = small_problem(200, 120, 3.0, 71).astype(np.float32)
    ref = oracle.solve(oracle.gram(X), 0.12, 0.1, eps=1e-9, max_iter=20000)
    om, st = _solve(lib, X, 0.12, 0.1, lib.OBS, precision=lib.PREC_TF32)
    assert st["status"] in (0, 1)
    assert np.linalg.norm(om - ref.omega) / np.linalg.norm(ref.omega) < 1e-2


def test_obs_modes(lib):
    """PREC_FP32 selects the chunked BF16X3 Z product (FP32-class); FP64 values are Cov only."""
    import torch

    X = torch.zeros((8, 16), device="cuda")
    with lib.Solver(X, 0.1, 0.1, variant=lib.OBS, precision=lib.PREC_FP32) as s:
        assert s.precision_used() == lib.PREC_BF16X3
    with pytest.raises(lib.HpcError) as e:
        lib.Solver(X.double(), 0.1, 0.1, variant=lib.OBS, precision=lib.PREC_FP64, value_dtype=lib.F64)
    assert e.value.status == lib.ERR_NOT_IMPLEMENTED


@pytest.mark.slow
def test_obs_equals_cov_on_the_fp32_workload(lib):
    """p = 16384, n = 8192 (the FP32 Cov/Obs workload): both variants, same estimate."""
    w = WORKLOADS["fp32_p16384"]
    X = make_x(w, device="cuda")
    ests = []
    for v in (lib.COV, lib.OBS):
        with lib.Solver(X, w.lambda1, w.lambda2, variant=v, precision=lib.PREC_BF16X3, eps=1e-6, max_iter=5000) as s:
            s.solve()
            ests.append(s.get_omega().to_scipy(w.p))
    a, b = ests
    d = a - b
    assert np.sqrt(d.multiply(d).sum()) / np.sqrt(a.multiply(a).sum()) < 1e-5


@pytest.mark.parametrize("n,p", [(200, 150), (40, 300)])
def test_auto_variant_matches_oracle(lib, n, p):
    """variant = AUTO resolves by Lemma 3.1 (hpc_choose_variant) and reaches the oracle's estimate."""
    import torch

    X = small_problem(p, n, 3.0, 80 + n).astype(np.float32)
    want, _, _ = lib.choose_variant(n, p)
    with lib.Solver(torch.as_tensor(X).cuda(), 0.15, 0.1, variant=lib.AUTO, precision=lib.PREC_FP32, eps=3e-7,
                    max_iter=5000) as s:
        assert s.info().variant == want
        st = s.solve().as_dict()
        om = s.omega_dense()
    assert _stopped_ok(st), st
    ref = oracle.solve(oracle.gram(X), 0.15, 0.1, eps=1e-9, max_iter=20000)
    assert np.linalg.norm(om - ref.omega) / np.linalg.norm(ref.omega) < 1e-5
    ok, detail = support_diff_ok(om, ref.omega, 0.15, 0.1, X=X)
    assert ok, detail
