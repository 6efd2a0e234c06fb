"""Differentiation through the C ABI against the FP64 oracle.

* hpc_backward: dL/dOmega (dense) and dL/dX of the smooth loss at the estimate, against
  oracle.smooth_loss_grads (itself pinned by central differences), and dL/dOmega against
  the solver's own G on its candidates, bitwise.
* ConcordSmoothLoss (torch.autograd.Function) gives the same gradients through autograd.
* hpc_hypergrad: the implicit lambda-gradient of the held-out loss, against oracle.hypergrad
  (dense, pinned by central differences of re-solved estimates) at small p and against the
  sparse FP64 form at the differentiation workload's size.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from workloads import WORKLOADS, make_x, omega0_for, sample_x_cpu, small_problem

pytestmark = pytest.mark.gpu

REL = 1e-4     # gradient tolerance against the FP64 reference


def _solved(lib, X, lam1, lam2, eps=1e-7):
    import torch

    Xt = torch.as_tensor(X).cuda()
    s = lib.Solver(Xt, lam1, lam2, precision=lib.PREC_FP32, eps=eps, max_iter=20000)
    s.solve()
    return s, Xt


def test_backward_matches_oracle_gradients(lib):
    X = small_problem(260, 180, 4.0, 41).astype(np.float32)
    lam1, lam2 = 0.12, 0.1
    s, Xt = _solved(lib, X, lam1, lam2)
    Om = s.omega_dense()
    dO, dX = s.backward(Xt, grad_loss=1.0)
    rO, rX = oracle.smooth_loss_grads(X.astype(np.float64), Om, lam2)
    dO, dX = dO.double().cpu().numpy(), dX.double().cpu().numpy()
    assert np.max(np.abs(dO - rO)) <= REL * np.max(np.abs(rO))
    assert np.max(np.abs(dX - rX)) <= REL * np.max(np.abs(rX))
    assert np.array_equal(dO, dO.T)
    # scaling by the upstream derivative
    dO2, dX2 = s.backward(Xt, grad_loss=-2.5)
    assert np.allclose(dO2.double().cpu().numpy(), -2.5 * dO, rtol=1e-6, atol=1e-7)
    assert np.allclose(dX2.double().cpu().numpy(), -2.5 * dX, rtol=1e-6, atol=1e-9)
    s.close()


def test_backward_fp64_handle_keeps_fp64(lib):
    """An FP64 handle: dL/dOmega and dL/dX (its transposes included) carry FP64 through,
    so both agree with the FP64 oracle far below FP32 rounding."""
    import torch

    X = small_problem(120, 90, 3.0, 43)
    lam1, lam2 = 0.12, 0.1
    Xt = torch.as_tensor(X).cuda()
    s = lib.Solver(Xt, lam1, lam2, value_dtype=lib.F64, precision=lib.PREC_FP64, eps=1e-10, max_iter=100000)
    s.solve()
    Om = s.omega_dense()
    dO, dX = s.backward(Xt, grad_loss=-1.5)
    assert dO.dtype == torch.float64 and dX.dtype == torch.float64
    rO, rX = oracle.smooth_loss_grads(X, Om, lam2)
    dO, dX = dO.cpu().numpy(), dX.cpu().numpy()
    assert np.max(np.abs(dO + 1.5 * rO)) <= 1e-12 * np.max(np.abs(rO))
    assert np.max(np.abs(dX + 1.5 * rX)) <= 1e-12 * np.max(np.abs(rX))
    s.close()


def test_backward_domega_is_the_solvers_gradient_bitwise(lib):
    X = small_problem(300, 200, 4.0, 42).astype(np.float32)
    s, Xt = _solved(lib, X, 0.15, 0.1, eps=1e-4)
    dO, _ = s.backward(Xt, dx=False)
    s.iterate(1)                       # its gradient pass runs at the estimate backward used
    r, c, _, g = s.candidates()
    assert np.array_equal(dO.cpu().numpy()[r, c].astype(np.float64), g)
    s.close()


@pytest.mark.parametrize("f64", [False, True])
def test_backward_domega_several_tile_pairs_per_cta(lib, f64):
    """p = 2600: more tile pairs than resident CTAs, so each CTA takes several and loads
    the next pair's S tile while it finishes the current one; the last tile is ragged
    (2600 = 40 x 64 + 40).  dL/dOmega against the FP64 oracle, and bitwise against the
    solver's own G on its candidates."""
    import torch

    rng = np.random.default_rng(47)
    X = rng.standard_normal((1200, 2600))
    if not f64:
        X = X.astype(np.float32)
    lam1, lam2 = 0.15, 0.1
    Xt = torch.as_tensor(X).cuda()
    opt = dict(value_dtype=lib.F64, precision=lib.PREC_FP64) if f64 else dict(precision=lib.PREC_FP32)
    s = lib.Solver(Xt, lam1, lam2, eps=1e-4, max_iter=20000, **opt)
    s.solve()
    Om = s.omega_dense()
    dO, _ = s.backward(Xt, dx=False)
    dO = dO.double().cpu().numpy()
    rO, _ = oracle.smooth_loss_grads(X.astype(np.float64), Om, lam2)
    assert np.max(np.abs(dO - rO)) <= (1e-12 if f64 else REL) * np.max(np.abs(rO))
    assert np.array_equal(dO, dO.T)
    s.iterate(1)                       # its gradient pass runs at the estimate backward used
    r, c, _, g = s.candidates()
    assert np.array_equal(dO[r, c], g)
    s.close()


def test_smooth_value_matches_oracle(lib):
    X = small_problem(200, 150, 3.0, 43).astype(np.float32)
    s, Xt = _solved(lib, X, 0.1, 0.1)
    f = s.smooth_value()
    ref = oracle.smooth_loss(X.astype(np.float64), s.omega_dense(), 0.1)
    assert f == pytest.approx(ref, rel=1e-6)
    s.close()


@pytest.mark.parametrize("form", ["values", "dense"])
def test_autograd_function(lib, form):
    import torch

    X = small_problem(180, 120, 3.0, 44).astype(np.float32)
    lam2 = 0.1
    s, Xt = _solved(lib, X, 0.12, lam2)
    Om = s.omega_dense()
    rO, rX = oracle.smooth_loss_grads(X.astype(np.float64), Om, lam2)
    Xg = Xt.clone().requires_grad_(True)
    if form == "values":
        rp, ci, v = s.omega_values()
        om = v.clone().requires_grad_(True)
    else:
        om = torch.as_tensor(Om, dtype=torch.float32, device="cuda").requires_grad_(True)
    loss = lib.concord_smooth_loss(Xg, om, s)
    assert float(loss) == pytest.approx(oracle.smooth_loss(X.astype(np.float64), Om, lam2), rel=1e-6)
    (3.0 * loss).backward()
    gx = Xg.grad.double().cpu().numpy()
    assert np.max(np.abs(gx - 3.0 * rX)) <= REL * 3.0 * np.max(np.abs(rX))
    go = om.grad.double().cpu().numpy()
    if form == "values":
        rows = np.repeat(np.arange(180), np.diff(rp.cpu().numpy()))
        ref = 3.0 * rO[rows, ci.cpu().numpy()]
    else:
        ref = 3.0 * rO
    assert np.max(np.abs(go - ref)) <= REL * np.max(np.abs(ref))
    s.close()


@pytest.mark.parametrize("form", ["values", "dense"])
def test_autograd_evaluates_at_the_given_omega(lib, form):
    """A perturbed omega (symmetric, on the estimate's pattern) changes the loss and its
    gradients to the oracle's at that omega: forward loads omega into the solver."""
    import torch

    X = small_problem(150, 100, 3.0, 47).astype(np.float32)
    lam2 = 0.1
    s, Xt = _solved(lib, X, 0.12, lam2)
    Om = s.omega_dense()
    f0 = s.smooth_value()
    rng = np.random.default_rng(3)
    P = np.where(Om != 0, rng.uniform(-0.05, 0.05, Om.shape), 0.0)
    Om2 = (Om + (P + P.T) / 2).astype(np.float32).astype(np.float64)
    Xg = Xt.clone().requires_grad_(True)
    rp, ci, _ = s.omega_values()
    rows = np.repeat(np.arange(150), np.diff(rp.cpu().numpy()))
    cols = ci.cpu().numpy()
    if form == "values":
        om = torch.as_tensor(Om2[rows, cols], dtype=torch.float32, device="cuda").requires_grad_(True)
    else:
        om = torch.as_tensor(Om2, dtype=torch.float32, device="cuda").requires_grad_(True)
    loss = lib.concord_smooth_loss(Xg, om, s)
    X64 = X.astype(np.float64)
    ref = oracle.smooth_loss(X64, Om2, lam2)
    assert float(loss.detach()) == pytest.approx(ref, rel=1e-6)
    assert abs(float(loss.detach()) - f0) > 1e-3 * abs(f0)
    loss.backward()
    rO, rX = oracle.smooth_loss_grads(X64, Om2, lam2)
    go = om.grad.double().cpu().numpy()
    refo = rO[rows, cols] if form == "values" else rO
    assert np.max(np.abs(go - refo)) <= REL * np.max(np.abs(refo))
    gx = Xg.grad.double().cpu().numpy()
    assert np.max(np.abs(gx - rX)) <= REL * np.max(np.abs(rX))
    with pytest.raises(ValueError):
        A = torch.as_tensor(Om2, dtype=torch.float32, device="cuda")
        A[0, 1] += 0.5
        lib.concord_smooth_loss(Xt, A, s)
    s.close()


def test_support_gradient_of_the_obs_variant(lib):
    """hpc_backward_support on an Obs handle (no S): dL/dOmega on the support from
    Y^T = Omega X^T and the resident X^T, against the oracle's dense gradient."""
    import torch

    X = small_problem(140, 90, 3.0, 48).astype(np.float32)
    lam2 = 0.1
    with lib.Solver(torch.as_tensor(X).cuda(), 0.12, lam2, variant=lib.OBS, precision=lib.PREC_FP32, eps=3e-7,
                    max_iter=3000) as s:
        s.solve()
        Om = s.omega_dense()
        dv, _ = s.backward_support(None, 2.0)
        rp, ci, _ = s.omega_values()
    rows = np.repeat(np.arange(140), np.diff(rp.cpu().numpy()))
    rO, _ = oracle.smooth_loss_grads(X.astype(np.float64), Om, lam2)
    ref = 2.0 * rO[rows, ci.cpu().numpy()]
    assert np.max(np.abs(dv.cpu().numpy() - ref)) <= REL * max(np.max(np.abs(ref)), 1.0)


def test_hypergrad_matches_dense_oracle(lib):
    import torch

    p = 60
    Xtr = small_problem(p, 90, 3.0, 45).astype(np.float32)
    Xva = small_problem(p, 50, 3.0, 46).astype(np.float32)
    lam1, lam2 = 0.1, 0.15
    s, Xt = _solved(lib, Xtr, lam1, lam2)
    d1, d2, info = s.hypergrad(torch.as_tensor(Xva).cuda(), tol=1e-10)
    assert info["converged"] == 1
    Om = s.omega_dense()
    r1, r2 = oracle.hypergrad(oracle.gram(Xtr), oracle.gram(Xva), Om, lam1, lam2)
    assert d1 == pytest.approx(r1, rel=REL)
    assert d2 == pytest.approx(r2, rel=REL)
    # and at the oracle's own estimate: the end-to-end value
    ref_om = oracle.solve(oracle.gram(Xtr), lam1, lam2, eps=1e-9, max_iter=100000).omega
    assert np.array_equal(ref_om != 0, Om != 0)
    e1, e2 = oracle.hypergrad(oracle.gram(Xtr), oracle.gram(Xva), ref_om, lam1, lam2)
    assert d1 == pytest.approx(e1, rel=1e-3) and d2 == pytest.approx(e2, rel=1e-3)
    s.close()


@pytest.mark.parametrize("handle,xdt", [("f64", "f64"), ("f64", "f32"), ("f64", "bf16"), ("f32", "bf16")])
def test_hypergrad_handle_and_xval_dtypes(lib, handle, xdt):
    """The held-out term (Omega S_val on the support) from X_val of each dtype. The
    held-out values are BF16-representable, so every dtype carries the same numbers; an
    FP64 handle (FP64 values, FP64 products) must then agree with the dense FP64 oracle
    to CG accuracy, an FP32 handle to the FP32 tolerance."""
    import torch

    p = 60
    Xtr = small_problem(p, 90, 3.0, 45)
    Xva = torch.as_tensor(small_problem(p, 50, 3.0, 46)).to(torch.bfloat16).double()
    lam1, lam2 = 0.1, 0.15
    if handle == "f64":
        Xt = torch.as_tensor(Xtr).cuda()
        s = lib.Solver(Xt, lam1, lam2, value_dtype=lib.F64, precision=lib.PREC_FP64, eps=1e-10, max_iter=100000)
        s.solve()
        rel, tol = 1e-8, 1e-13
    else:
        s, Xt = _solved(lib, Xtr.astype(np.float32), lam1, lam2)
        rel, tol = REL, 1e-10
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[xdt]
    d1, d2, info = s.hypergrad(Xva.to(tdt).cuda(), tol=tol)
    assert info["converged"] == 1
    Om = s.omega_dense()
    Xtr_used = Xtr if handle == "f64" else Xtr.astype(np.float32).astype(np.float64)
    r1, r2 = oracle.hypergrad(oracle.gram(Xtr_used), oracle.gram(Xva.numpy()), Om, lam1, lam2)
    assert d1 == pytest.approx(r1, rel=rel)
    assert d2 == pytest.approx(r2, rel=rel)
    s.close()


def test_hypergrad_iteration_cap(lib):
    """CG runs in captured chunks of eight iterations plus a directly launched tail:
    the cap is honoured exactly below, at and above one chunk, a capped run reports
    NOT_CONVERGED, repeats bitwise, and more iterations approach the converged value."""
    import torch

    p = 60
    Xtr = small_problem(p, 90, 3.0, 45).astype(np.float32)
    Xva = torch.as_tensor(small_problem(p, 50, 3.0, 46).astype(np.float32)).cuda()
    s, _ = _solved(lib, Xtr, 0.1, 0.15)
    ref1, ref2, info = s.hypergrad(Xva, tol=1e-12)
    assert info["converged"] == 1
    errs = []
    for cap in (5, 8, 13):
        d1, d2, info = s.hypergrad(Xva, tol=1e-30, max_iter=cap)
        assert info["converged"] == 0 and info["cg_iterations"] == cap
        e1, e2, _ = s.hypergrad(Xva, tol=1e-30, max_iter=cap)
        assert (d1, d2) == (e1, e2)
        errs.append(abs(d1 - ref1) + abs(d2 - ref2))
    assert errs[2] <= errs[0]
    s.close()


@pytest.mark.slow
def test_differentiation_workload_full_size(lib):
    """p = 16384, n = 4096 train + 2048 held-out (same Omega0 law): backward at sampled
    entries and the hypergradient against the sparse FP64 reference on the GPU's support."""
    import torch

    w = WORKLOADS["adjoint_p16384"]
    om0 = omega0_for(w)
    from workloads import HELDOUT_STREAM, cast_x, sample_x_cuda

    Xtr = cast_x(sample_x_cuda(om0, w.n, w.seed), "f32")
    Xva = cast_x(sample_x_cuda(om0, 2048, w.seed, stream=HELDOUT_STREAM), "f32")
    s = lib.Solver(Xtr, w.lambda1, w.lambda2, precision=lib.PREC_FP32, eps=1e-6, max_iter=20000)
    s.solve()
    d1, d2, info = s.hypergrad(Xva, tol=1e-10)
    assert info["converged"] == 1
    csr = s.get_omega().to_scipy(w.p)
    Xh, Xvh = Xtr.cpu().numpy(), Xva.cpu().numpy()
    r1, r2 = oracle.hypergrad_sparse(Xh, Xvh, csr, w.lambda1, w.lambda2)
    assert d1 == pytest.approx(r1, rel=REL) and d2 == pytest.approx(r2, rel=REL)
    # backward: dL/dX and dL/dOmega at sampled entries against FP64 formulas from X
    dO, dX = s.backward(Xtr)
    rng = np.random.default_rng(0)
    ri = rng.integers(0, w.p, 300)
    rj = rng.integers(0, w.p, 300)
    gref = oracle.gradient_entries(Xh, csr, w.lambda2, ri, rj)
    got = dO[torch.as_tensor(ri).cuda(), torch.as_tensor(rj).cuda()].double().cpu().numpy()
    assert np.max(np.abs(got - gref)) <= REL * max(np.max(np.abs(gref)), 1.0)
    rr = rng.integers(0, w.n, 20)
    Y = Xh[rr].astype(np.float64) @ csr          # rows of X Omega
    dx_ref = (Y @ csr) / w.n
    dx_got = dX[torch.as_tensor(rr).cuda()].double().cpu().numpy()
    assert np.max(np.abs(dx_got - dx_ref)) <= REL * np.max(np.abs(dx_ref))
    s.close()


@pytest.mark.slow
def test_hypergrad_central_differences_full_size(lib):
    """p = 16384, n = 4096 train + 2048 held-out: the FP32 handle's hpc_hypergrad against
    central differences of the held-out loss (evaluated by the oracle from X_val) at re-solves
    with lambda1 +- h and lambda2 +- h.  The implicit-function gradient holds while the support
    stays fixed, and with h = 1e-3 entries near the threshold enter or leave; so the
    differences are taken on an FP64 handle (SIMT FP64 Gram, FP64 iterates, eps = 1e-11) with
    h = 1e-3, 1e-5 and 1e-6, warm-started from the estimate, and checked with the smallest h
    whose four re-solves keep the support (relative error <= 1e-4).  dL/dX (exactly quadratic
    in X) is checked against central differences of the oracle's loss at three entries."""
    import json
    import os

    from workloads import HELDOUT_STREAM, cast_x, sample_x_cuda

    w = WORKLOADS["adjoint_p16384"]
    om0 = omega0_for(w)
    Xtr = cast_x(sample_x_cuda(om0, w.n, w.seed), "f32")
    Xva = cast_x(sample_x_cuda(om0, 2048, w.seed, stream=HELDOUT_STREAM), "f32")
    Xvh = Xva.cpu().numpy()
    s = lib.Solver(Xtr, w.lambda1, w.lambda2, precision=lib.PREC_FP32, eps=1e-8, max_iter=20000)
    s.solve()
    d1, d2, info = s.hypergrad(Xva, tol=1e-12)
    s64 = lib.Solver(Xtr.double(), w.lambda1, w.lambda2, precision=lib.PREC_FP64, value_dtype=lib.F64, eps=1e-11,
                     max_iter=50000)
    s64.solve()
    e1, e2, _ = s64.hypergrad(Xva.double(), tol=1e-13)
    base = s64.get_omega()
    pattern = base.to_scipy(w.p) != 0
    rec = {"workload": w.name, "hypergrad_fp32": [d1, d2], "hypergrad_fp64": [e1, e2], "steps": {}}
    chosen = {}
    for h in (1e-3, 1e-5, 1e-6):
        vals, same = {}, {}
        for name, (l1, l2) in {"l1+": (w.lambda1 + h, w.lambda2), "l1-": (w.lambda1 - h, w.lambda2),
                               "l2+": (w.lambda1, w.lambda2 + h), "l2-": (w.lambda1, w.lambda2 - h)}.items():
            s64.set_omega(base)
            s64.set_lambda(l1, l2)
            s64.solve()
            est = s64.get_omega().to_scipy(w.p)
            same[name] = int(((est != 0) != pattern).nnz)
            vals[name] = oracle.heldout_loss_from_x(Xvh, est)
        g1 = (vals["l1+"] - vals["l1-"]) / (2 * h)
        g2 = (vals["l2+"] - vals["l2-"]) / (2 * h)
        rec["steps"][str(h)] = {"central_differences": [g1, g2], "support_changes": same}
        if "l1" not in chosen and same["l1+"] == 0 and same["l1-"] == 0:
            chosen["l1"] = (h, g1)
        if "l2" not in chosen and same["l2+"] == 0 and same["l2-"] == 0:
            chosen["l2"] = (h, g2)
    rec["chosen"] = chosen
    if os.environ.get("HPC_REPORT_DIR"):
        with open(os.path.join(os.environ["HPC_REPORT_DIR"], "hypergrad_fd.json"), "w") as fh:
            json.dump(rec, fh, default=float)
    assert chosen, rec
    if "l1" in chosen:
        assert d1 == pytest.approx(chosen["l1"][1], rel=1e-4), rec
    if "l2" in chosen:
        assert d2 == pytest.approx(chosen["l2"][1], rel=1e-4), rec
    # dL/dX at the FP32 estimate against central differences of the oracle's loss (lambda1 = 0
    # in objective_from_x leaves the smooth part)
    est32 = s.get_omega().to_scipy(w.p)
    _, dX = s.backward(Xtr, domega=False)
    Xh = Xtr.cpu().numpy().astype(np.float64)
    h = 1e-3
    for (k, j) in [(0, 0), (17, 9001), (4095, 16383)]:
        vals = []
        for sgn in (1, -1):
            Xp = Xh.copy()
            Xp[k, j] += sgn * h
            vals.append(oracle.objective_from_x(Xp, est32, 0.0, w.lambda2))
        fdx = (vals[0] - vals[1]) / (2 * h)
        got = float(dX[k, j])
        assert got == pytest.approx(fdx, rel=1e-4, abs=1e-6), (k, j, got, fdx)
    s.close()
    s64.close()
