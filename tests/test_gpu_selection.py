"""Model selection over a lambda1 grid (Section 2's grids; Section 4's support scores):
the device's held-out loss against the oracle's, and the selected grid point against the
oracle's own selection (a cold FP64 solve and held-out loss per point)."""
import numpy as np
import pytest
import scipy.sparse as sp

import oracle
from paper_1710_10769_gb300.selection import select_lambda1, support_recovery
from workloads import HELDOUT_STREAM, omega0_random, sample_x_cpu

pytestmark = pytest.mark.gpu


def _problem(p, n, nval, d, seed):
    om0 = omega0_random(p, d, seed)
    X = sample_x_cpu(om0, n, seed, x_dtype="f32")
    Xv = sample_x_cpu(om0, nval, seed, stream=HELDOUT_STREAM, x_dtype="f32")
    return om0, X, Xv


@pytest.mark.parametrize("variant", ["cov", "obs"])
def test_heldout_loss_matches_oracle(lib, variant):
    import torch

    om0, X, Xv = _problem(220, 160, 90, 4.0, 7)
    v = lib.COV if variant == "cov" else lib.OBS
    with lib.Solver(torch.as_tensor(X).cuda(), 0.12, 0.1, variant=v, precision=lib.PREC_FP32, eps=3e-7,
                    max_iter=3000) as s:
        s.solve()
        got = s.heldout_loss(torch.as_tensor(Xv).cuda())
        est = s.get_omega().to_scipy(220)
    ref = oracle.heldout_loss_from_x(Xv.astype(np.float64), est)
    assert got == pytest.approx(ref, rel=1e-6)


def test_selection_matches_the_oracles(lib):
    import torch

    p, lam2 = 180, 0.1
    om0, X, Xv = _problem(p, 120, 80, 4.0, 11)
    grid = list(np.logspace(np.log10(0.4), np.log10(0.05), 8))
    with lib.Solver(torch.as_tensor(X).cuda(), grid[0], lam2, precision=lib.PREC_FP32, eps=1e-7,
                    max_iter=20000) as s:
        sel = select_lambda1(s, torch.as_tensor(Xv).cuda(), grid, lam2, truth=om0)
        chosen = s.get_omega().to_scipy(p)
    S = oracle.gram(X.astype(np.float64))
    ref_losses, ref_ests = [], []
    for l1 in grid:
        r = oracle.solve(S, l1, lam2, eps=1e-9, max_iter=20000)
        ref_ests.append(r.omega)
        ref_losses.append(oracle.heldout_loss_from_x(Xv.astype(np.float64), sp.csr_matrix(r.omega)))
    assert np.allclose(sel["heldout"], ref_losses, rtol=1e-5, atol=0)
    assert sel["best"] == int(np.argmin(ref_losses))
    # the solver is left at the selected estimate
    assert np.linalg.norm(chosen.toarray() - ref_ests[sel["best"]]) <= 1e-5 * np.linalg.norm(ref_ests[sel["best"]])
    # support scores are those of the oracle's estimates (identical patterns at this tolerance)
    for rec, ref in zip(sel["recovery"], ref_ests):
        want = support_recovery(sp.csr_matrix(ref), om0)
        assert abs(rec["ppv"] - want["ppv"]) <= 0.02 and abs(rec["tpr"] - want["tpr"]) <= 0.02
