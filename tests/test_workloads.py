"""The seeded input generator follows the stated recipe (CPU only):

- random graphs: round(p d / 2) distinct pairs, values +-U(0.2, 0.5) with both signs, a
  diagonal of 1.5 x the row's absolute off-diagonal sum (1 for an empty row);
- banded graphs: every pair with 0 < |i - j| <= b; tridiagonal: 1.0 and -0.4;
- the same seed gives the same matrix, another seed another one;
- BF16 rounding is round-to-nearest-even, the conversion torch does;
- the normals come from Philox4x32-10, which reproduces its published known-answer
  vectors, and the numpy and torch forms of the draw give the same integers;
- Omega0 = B^T B for the sparse factor the sampler builds, and the rows of X follow
  N(0, Omega0^-1);
- a row of X depends on its index only (not on how the rows are chunked), and the
  torch form of the draw agrees with the numpy form to FP64 rounding;
- the workload table holds the shapes the benchmark and the tests name.
"""
import math

import numpy as np
import pytest

import os

from workloads import (BATCH_PROBLEMS, PATH_LAMBDA1, PATH_LAMBDA2, WORKLOADS, normal_pairs, omega0_banded,
                       omega0_random, omega0_tridiagonal, philox4x32, round_to_bf16, sample_factor, sample_rows_cpu,
                       sample_x_cpu, sample_x_cuda)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _check_dominant(om, lo, hi):
    A = om.toarray()
    assert np.array_equal(A, A.T)
    off = A - np.diag(np.diag(A))
    nz = off[off != 0]
    assert np.all((np.abs(nz) >= lo) & (np.abs(nz) <= hi))
    rowsum = np.abs(off).sum(axis=1)
    want = np.where(rowsum > 0, 1.5 * rowsum, 1.0)
    assert np.allclose(np.diag(A), want, rtol=1e-15, atol=0)
    np.linalg.cholesky(A)                      # strictly diagonally dominant: positive definite
    return off


@pytest.mark.parametrize("p,d,seed", [(200, 5.0, 0), (97, 8.0, 3), (50, 0.5, 1)])
def test_random_graph_recipe(p, d, seed):
    om = omega0_random(p, d, seed)
    off = _check_dominant(om, 0.2, 0.5)
    iu, ju = np.nonzero(np.triu(off))
    assert iu.size == int(round(p * d / 2))
    signs = np.sign(off[iu, ju])
    if iu.size >= 20:
        assert 0.25 < np.mean(signs > 0) < 0.75
    assert (omega0_random(p, d, seed) != om).nnz == 0
    assert (omega0_random(p, d, seed + 1) != om).nnz > 0


def test_banded_and_tridiagonal_recipes():
    p, b = 60, 3
    om = omega0_banded(p, b, 7)
    off = _check_dominant(om, 0.2, 0.5)
    i, j = np.nonzero(off)
    assert np.all((np.abs(i - j) > 0) & (np.abs(i - j) <= b))
    assert i.size == 2 * sum(p - k for k in range(1, b + 1))
    T = omega0_tridiagonal(10).toarray()
    assert np.all(np.diag(T) == 1.0) and np.all(np.diag(T, 1) == -0.4) and np.all(np.diag(T, -1) == -0.4)
    assert np.count_nonzero(T) == 10 + 2 * 9


def test_bf16_rounding_is_nearest_even():
    import torch

    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)                # BF16 spacing at 1
    cases = np.array([one + ulp / 2,           # halfway, 1.0 is even: down
                      one + 3 * ulp / 2,       # halfway, 1 + 2 ulp is even: up
                      one + ulp / 2 + np.float32(2.0 ** -20),   # above halfway: up
                      -(one + ulp / 2), np.inf, -np.inf, 0.0, -0.0], dtype=np.float32)
    got = round_to_bf16(cases)
    assert got[0] == 1.0 and got[1] == one + 2 * ulp and got[2] == one + ulp and got[3] == -1.0
    assert np.isinf(got[4]) and np.isinf(got[5]) and got[6] == 0.0
    x = np.random.default_rng(0).standard_normal(100000).astype(np.float32) * 10.0 ** np.random.default_rng(
        1).integers(-6, 6, 100000)
    ref = torch.from_numpy(x).to(torch.bfloat16).float().numpy()
    assert np.array_equal(round_to_bf16(x), ref)


def test_philox_known_answers():
    rows = []
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as fh:
        for ln in fh:
            if ln.strip() and not ln.startswith("#"):
                rows.append([int(t, 16) for t in ln.split()])
    assert len(rows) == 3
    for r in rows:
        c = [np.array([v], dtype=np.int64) for v in r[:4]]
        out = philox4x32(*c, r[4], r[5])
        assert [int(o[0]) for o in out] == r[6:10]


def test_numpy_and_torch_draws_agree():
    import torch

    z_np = normal_pairs(np, 11, 0, np.arange(7), 300)
    z_t = normal_pairs(torch, 11, 0, np.arange(7), 300, device="cpu").numpy()
    # the same Philox integers; Box-Muller's log and cos may differ in the last bit
    assert np.max(np.abs(z_np - z_t)) <= 4 * np.finfo(np.float64).eps * np.max(np.abs(z_np))
    assert 0.3 < np.mean(np.abs(z_np)) < 1.3 and abs(np.mean(z_np)) < 0.1
    om = omega0_random(300, 5.0, 3)
    X = sample_x_cpu(om, 200, 3)
    Xt = sample_x_cuda(om, 200, 3, device="cpu", chunk=64).numpy()
    assert np.max(np.abs(X - Xt)) <= 1e-13 * np.max(np.abs(X))


def test_sparse_factor_and_rows():
    for om in (omega0_random(150, 6.0, 2), omega0_banded(90, 3, 4), omega0_tridiagonal(40)):
        f = sample_factor(om)
        assert f.m == om.shape[0] + (om.nnz - om.shape[0]) // 2
        assert abs(f.Bt @ f.Bt.T - om).max() <= 1e-14
    om = omega0_random(150, 6.0, 2)
    X = sample_x_cpu(om, 70, 9, chunk=64)
    assert np.array_equal(X, sample_x_cpu(om, 70, 9, chunk=16))
    assert np.array_equal(X[[3, 69, 40]], sample_rows_cpu(om, [3, 69, 40], 9))
    assert not np.array_equal(X, sample_x_cpu(om, 70, 10))
    assert not np.array_equal(X, sample_x_cpu(om, 70, 9, stream=1))


@pytest.mark.parametrize("graph", ["random", "tridiagonal"])
def test_samples_follow_the_stated_law(graph):
    """Rows of X follow N(0, Omega0^-1): the sample covariance of many draws is within
    five standard errors of Omega0^-1 in every entry."""
    p, n = 12, 200000
    om = omega0_random(p, 3.0, 5) if graph == "random" else omega0_tridiagonal(p)
    X = sample_x_cpu(om, n, 5, chunk=20000)
    S = X.T @ X / n
    Sigma = np.linalg.inv(om.toarray())
    # each entry's sampling error is about sqrt((Sigma_ii Sigma_jj + Sigma_ij^2) / n)
    sd = np.sqrt((np.outer(np.diag(Sigma), np.diag(Sigma)) + Sigma ** 2) / n)
    assert np.all(np.abs(S - Sigma) <= 5 * sd)
    # and not the law of X = Z L^-T with Omega0 = L L^T, (L^T L)^-1
    if graph == "random":
        L = np.linalg.cholesky(om.toarray())
        assert np.max(np.abs(S - np.linalg.inv(L.T @ L)) / sd) > 20


def test_workload_table():
    assert (WORKLOADS["bf16_p65536"].p, WORKLOADS["bf16_p65536"].n) == (65536, 32768)
    assert (WORKLOADS["fp32_p16384"].p, WORKLOADS["fp32_p16384"].n) == (16384, 8192)
    assert (WORKLOADS["fp64_p500"].p, WORKLOADS["fp64_p500"].n) == (500, 250)
    assert (WORKLOADS["path_p8192"].p, WORKLOADS["path_p8192"].n) == (8192, 4096)
    assert (WORKLOADS["adjoint_p16384"].p, WORKLOADS["adjoint_p16384"].n) == (16384, 4096)
    assert len(PATH_LAMBDA1) == 32 and PATH_LAMBDA2 == 0.1
    assert PATH_LAMBDA1[0] == pytest.approx(0.05) and PATH_LAMBDA1[-1] == pytest.approx(0.8)
    r = np.diff(np.log(PATH_LAMBDA1))
    assert np.allclose(r, math.log(16) / 31)
    assert [(w.p, w.n) for w in BATCH_PROBLEMS] == [(1024 * k, 512 * k) for k in range(1, 17)]
