"""Candidate rows far longer than one block's shared-memory sort (the hub row of a one-factor
X: about 2p entries before de-dup in Cov, p in Obs, at p = 9000).  They are sorted in chunks
and merged by ranks; the first iterations, where the hub row is longest, must take the
oracle's steps (same step sizes) and reach its iterate (CSR form of Alg. 2 and Alg. 3)."""
import numpy as np
import pytest

import oracle
from tests.support import support_diff_ok
from workloads import hub_factor_problem

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

P, N, LAM1, LAM2, ITERS = 9000, 1000, 0.4, 0.1, 3


@pytest.fixture(scope="module")
def hub():
    X = hub_factor_problem(P, N, 3).astype(np.float32)
    return X, oracle.gram_chunked(X.astype(np.float64))


@pytest.mark.parametrize("variant", ["cov", "obs"])
def test_hub_row_iterations_follow_the_oracle(lib, hub, variant):
    import torch

    X, S = hub
    if variant == "cov":
        ref = oracle.solve_sparse(S, LAM1, LAM2, eps=1e-12, max_iter=ITERS, block=512, threads=8)
    else:
        ref = oracle.solve_obs_sparse(X, LAM1, LAM2, eps=1e-12, max_iter=ITERS, block=512)
    v = lib.COV if variant == "cov" else lib.OBS
    with lib.Solver(torch.as_tensor(X).cuda(), LAM1, LAM2, variant=v, precision=lib.PREC_FP32, eps=1e-12,
                    max_iter=ITERS, device_loop=0) as s:
        halvings, cands = [], []
        for _ in range(ITERS):
            st = s.iterate(1).as_dict()
            halvings.append(st["accepted_halvings"])
            cands.append(st["candidates"])
        om = s.omega_dense()
    # the hub row alone holds p candidates at the first iteration
    assert cands[0] >= P, cands
    assert halvings == [round(-np.log2(t)) for t in ref.taus], (halvings, ref.taus)
    R = ref.omega.toarray()
    err = np.linalg.norm(om - R) / np.linalg.norm(R)
    assert err < 1e-5, err
    ok, detail = support_diff_ok(om, R, LAM1, LAM2, S=S)
    assert ok, detail
    assert np.array_equal(om, om.T)
