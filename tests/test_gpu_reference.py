"""Full-size parity against cached FP64 references (tests/golden/ref_<name>.npz, written by
tests/golden/make_fullsize_refs.py from the CSR form of the oracle, each with a certified
bound ||r||_F / lambda2 on its own distance to the minimiser).

- p = 16384, n = 8192, FP32 X, lambda = (0.2, 0.1): the Cov solve with the plain FP32 Gram,
  the Cov solve with the BF16X3 tensor-core Gram and the Obs solve, each within
  ||Omega - Omega_ref||_F / ||Omega_ref||_F <= 1e-5 with the support identical except for
  entries within 1e-6 of the threshold.  The minimiser is unique (lambda2 > 0), so one
  reference serves both variants.
- p = 65536, n = 32768, BF16 X, lambda = (0.15, 0.05), the headline solve: its error
  against the FP64 reference computed on the same BF16 X, for the estimate and for the
  objective F (FP64, from X).

Before comparing, each test checks that the X it drew on the device is the reference's X
(column sums and sampled rows against the CPU draw).
"""
import os

import numpy as np
import pytest

import oracle
from tests.refcheck import check_x, compare, load_ref, ref_path, report
from workloads import WORKLOADS, make_x, omega0_for

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-5


def _stopped_ok(st, floor=1e-6):
    return st["status"] == 0 or (st["status"] == 1 and st["rel_change"] < floor)


@pytest.fixture(scope="module")
def fp32_case(lib):
    w = WORKLOADS["fp32_p16384"]
    ref = load_ref(w.name)
    X = make_x(w, device="cuda")
    xinfo = check_x(X, ref, omega0_for(w), w.seed)
    return dict(w=w, ref=ref, X=X, Xh=X.cpu().numpy(), xinfo=xinfo)


@pytest.mark.parametrize("variant,precision,eps", [("cov", "fp32", 1e-7), ("cov", "bf16x3", 1e-7),
                                                   ("obs", "fp32", 3e-7)])
def test_fp32_workload_against_fp64_reference(lib, fp32_case, variant, precision, eps):
    w, ref = fp32_case["w"], fp32_case["ref"]
    v = lib.COV if variant == "cov" else lib.OBS
    prec = {"fp32": lib.PREC_FP32, "bf16x3": lib.PREC_BF16X3}[precision]
    with lib.Solver(fp32_case["X"], w.lambda1, w.lambda2, variant=v, precision=prec, eps=eps,
                    max_iter=3000) as s:
        st = s.solve().as_dict()
        est = s.get_omega().to_scipy(w.p)
    assert _stopped_ok(st), st
    c = compare(est, ref, fp32_case["Xh"], w.lambda1, w.lambda2)
    report({"workload": w.name, "variant": variant, "precision": precision, "eps": eps,
            "iterations": st["iterations"], "ref_bound": float(ref["distance_bound_rel"]), **c,
            **fp32_case["xinfo"]})
    assert c["rel_fro"] <= TOL, c
    assert c["support_ok"], c


@pytest.mark.skipif(not os.path.exists(ref_path("bf16_p65536")), reason="FP64 reference not cached")
def test_headline_against_fp64_reference(lib):
    import torch

    w = WORKLOADS["bf16_p65536"]
    ref = load_ref(w.name)
    X = make_x(w, device="cuda")
    xinfo = check_x(X, ref, omega0_for(w), w.seed)
    with lib.Solver(X, w.lambda1, w.lambda2, precision=lib.PREC_AUTO, eps=1e-7, max_iter=5000) as s:
        st = s.solve().as_dict()
        est = s.get_omega().to_scipy(w.p)
        rng = np.random.default_rng(5)
        r = np.concatenate([rng.integers(0, w.p, 300), np.arange(0, w.p, 2048)])
        c_ = np.concatenate([rng.integers(0, w.p, 300), np.arange(0, w.p, 2048)])
        s_gpu = s.s_entries(r, c_)
    assert _stopped_ok(st), st
    Xh = X.float().cpu().numpy()
    del X
    torch.cuda.empty_cache()
    c = compare(est, ref, Xh, w.lambda1, w.lambda2)
    s_ref = oracle.gram_entries(Xh, r, c_)
    d_ref = np.sqrt(oracle.gram_entries(Xh, r, r) * oracle.gram_entries(Xh, c_, c_))
    s_err = float(np.max(np.abs(s_gpu - s_ref) / d_ref))
    F_gpu = oracle.objective_from_x(Xh, est, w.lambda1, w.lambda2)
    F_ref = float(ref["F"][-1])
    rec = {"workload": w.name, "variant": "cov", "precision": "bf16 (mixed)", "eps": 1e-7,
           "iterations": st["iterations"], "ref_bound": float(ref["distance_bound_rel"]), **c, **xinfo,
           "S_max_err_rel_to_sqrt_diag": s_err, "F_at_estimate": F_gpu, "F_ref": F_ref,
           "F_rel_err": abs(F_gpu - F_ref) / abs(F_ref)}
    report(rec)
    assert c["rel_fro"] <= TOL, rec
    assert c["support_ok"], rec
