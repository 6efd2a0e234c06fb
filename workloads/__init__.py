"""Seeded synthetic inputs shared by the FP64 oracle and the GPU library.

This module draws the data only: a sparse, strictly diagonally dominant
ground-truth precision matrix Omega0 and Gaussian observations X whose rows
follow N(0, Omega0^-1).  It holds none of the estimator's arithmetic, so the
oracle and the CUDA path can both consume its arrays without sharing code.

Recipe (Section 4 describes banded "chain" and random strictly diagonally
dominant Omega0 with Gaussian samples; the exact sizes below are the
benchmark workloads of this project):

* random graphs: round(p*d/2) distinct off-diagonal pairs (i<j) drawn
  uniformly, each valued sign * U(lo, hi) with a fair random sign; the
  diagonal is ``dominance * sum_j |omega_ij|`` (1.0 for an empty row);
* banded graphs: every pair with 0 < |i-j| <= bandwidth, same values;
* tridiagonal: diagonal 1.0, first off-diagonals -0.4;
* X = Z L^-T with Omega0 = L L^T (Cholesky) and Z iid N(0, 1), so that
  cov(x) = (L L^T)^-1 = Omega0^-1.

Everything is a pure function of ``seed``.  numpy's PCG64 draws Omega0 and,
on the CPU path, Z; the CUDA path (used for p >= 16384, where a dense CPU
Cholesky takes minutes) draws Z with torch's Philox generator on the device
and factors Omega0 in FP32.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp


@dataclasses.dataclass(frozen=True)
class Workload:
    """One benchmark configuration: problem shape, graph law and solver knobs."""

    name: str
    p: int
    n: int
    graph: str            # "tridiagonal" | "random" | "banded"
    degree: float         # mean off-diagonal nonzeros per row of Omega0 (random)
    bandwidth: int        # banded graphs
    lambda1: float
    lambda2: float
    eps: float
    x_dtype: str          # "f64" | "f32" | "bf16"
    seed: int


# The five workloads the project measures and checks (sizes, graph laws and
# tuning parameters as stated for each benchmark configuration).
WORKLOADS = {
    "fp64_p500": Workload("fp64_p500", 500, 250, "tridiagonal", 2.0, 1, 0.3, 0.2, 1e-6, "f64", 0),
    "fp32_p16384": Workload("fp32_p16384", 16384, 8192, "random", 5.0, 0, 0.2, 0.1, 1e-6, "f32", 1),
    "bf16_p65536": Workload("bf16_p65536", 65536, 32768, "random", 8.0, 0, 0.15, 0.05, 1e-6, "bf16", 2),
    "path_p8192": Workload("path_p8192", 8192, 4096, "random", 5.0, 0, 0.05, 0.1, 1e-6, "f32", 3),
    "adjoint_p16384": Workload("adjoint_p16384", 16384, 4096, "random", 5.0, 0, 0.2, 0.1, 1e-6, "f32", 4),
}

# Batch of independent problems of uneven size: p = 1024 k (k = 1..16), n = p / 2,
# banded Omega0 of bandwidth 3 (FP32 X).
BATCH_PROBLEMS = tuple(Workload(f"batch_p{1024 * k}", 1024 * k, 512 * k, "banded", 0.0, 3, 0.15, 0.1, 1e-6, "f32",
                                100 + k) for k in range(1, 17))

# Regularisation grid of the batched path workload: 32 values of lambda1,
# log-spaced over [0.05, 0.8], at lambda2 = 0.1.
PATH_LAMBDA1 = tuple(float(v) for v in np.logspace(math.log10(0.05), math.log10(0.8), 32))
PATH_LAMBDA2 = 0.1


def _finish_dominant(p: int, rows: np.ndarray, cols: np.ndarray, vals: np.ndarray,
                     dominance: float) -> sp.csr_matrix:
    """Symmetrise off-diagonal pairs (i<j) and set a dominant diagonal."""
    r = np.concatenate([rows, cols])
    c = np.concatenate([cols, rows])
    v = np.concatenate([vals, vals])
    off = sp.coo_matrix((v, (r, c)), shape=(p, p)).tocsr()
    absrow = np.asarray(abs(off).sum(axis=1)).ravel()
    diag = np.where(absrow > 0, dominance * absrow, 1.0)
    om = (off + sp.diags(diag)).tocsr()
    om.sort_indices()
    return om


def omega0_tridiagonal(p: int, diag: float = 1.0, off: float = -0.4) -> sp.csr_matrix:
    """Tridiagonal Omega0 (positive definite since |2*off| < diag)."""
    i = np.arange(p - 1)
    om = sp.diags([np.full(p - 1, off), np.full(p, diag), np.full(p - 1, off)], [-1, 0, 1],
                  shape=(p, p), format="csr")
    om.sort_indices()
    return om


def omega0_random(p: int, degree: float, seed: int, lo: float = 0.2, hi: float = 0.5,
                  dominance: float = 1.5) -> sp.csr_matrix:
    """Random graph: round(p*degree/2) uniform distinct pairs (i<j)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    m = int(round(p * degree / 2.0))
    m = min(m, p * (p - 1) // 2)
    keys = np.empty(0, dtype=np.int64)
    while keys.size < m:
        need = m - keys.size
        i = rng.integers(0, p, size=2 * need + 16, dtype=np.int64)
        j = rng.integers(0, p, size=2 * need + 16, dtype=np.int64)
        a, b = np.minimum(i, j), np.maximum(i, j)
        ok = a != b
        new = a[ok] * p + b[ok]
        # keep first occurrences in draw order, so the result depends on seed only
        allk = np.concatenate([keys, new])
        _, first = np.unique(allk, return_index=True)
        keys = allk[np.sort(first)][:m]
    rows, cols = keys // p, keys % p
    mag = rng.uniform(lo, hi, size=m)
    sign = np.where(rng.integers(0, 2, size=m) == 1, 1.0, -1.0)
    return _finish_dominant(p, rows, cols, sign * mag, dominance)


def omega0_banded(p: int, bandwidth: int, seed: int, lo: float = 0.2, hi: float = 0.5,
                  dominance: float = 1.5) -> sp.csr_matrix:
    """Banded ("chain") graph: all pairs with 0 < j - i <= bandwidth."""
    rng = np.random.Generator(np.random.PCG64(seed))
    rows, cols = [], []
    for k in range(1, bandwidth + 1):
        i = np.arange(p - k, dtype=np.int64)
        rows.append(i)
        cols.append(i + k)
    rows = np.concatenate(rows) if rows else np.empty(0, np.int64)
    cols = np.concatenate(cols) if cols else np.empty(0, np.int64)
    m = rows.size
    mag = rng.uniform(lo, hi, size=m)
    sign = np.where(rng.integers(0, 2, size=m) == 1, 1.0, -1.0)
    return _finish_dominant(p, rows, cols, sign * mag, dominance)


def omega0_for(w: Workload) -> sp.csr_matrix:
    if w.graph == "tridiagonal":
        return omega0_tridiagonal(w.p)
    if w.graph == "random":
        return omega0_random(w.p, w.degree, w.seed)
    if w.graph == "banded":
        return omega0_banded(w.p, w.bandwidth, w.seed)
    raise ValueError(w.graph)


def round_to_bf16(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), as float32."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    bias = ((u >> 16) & 1) + 0x7FFF
    r = ((u + bias) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    return np.where(np.isfinite(a), out, a).astype(np.float32)


def sample_x_cpu(omega0: sp.csr_matrix, n: int, seed: int) -> np.ndarray:
    """X = Z L^-T in float64 on the CPU (dense Cholesky; fine up to p ~ 8192), where
    Omega0 = L L^T: rows of X have covariance L^-1 L^-T = (L^T L)^-1 (not Omega0^-1)."""
    import scipy.linalg as sla

    p = omega0.shape[0]
    rng = np.random.Generator(np.random.PCG64(seed + 1_000_003))
    z = rng.standard_normal((n, p))
    L = np.linalg.cholesky(omega0.toarray())
    xt = sla.solve_triangular(L, z.T, lower=True, check_finite=False)
    return np.ascontiguousarray(xt.T)


def sample_x_cuda(omega0: sp.csr_matrix, n: int, seed: int, device: str = "cuda"):
    """X = Z L^-T on a CUDA device with torch (FP32 factor), returned as a float32 tensor;
    the same law as sample_x_cpu (row covariance (L^T L)^-1)."""
    import torch

    p = omega0.shape[0]
    g = torch.Generator(device=device)
    g.manual_seed(seed + 1_000_003)
    dense = torch.zeros((p, p), dtype=torch.float32, device=device)
    coo = omega0.tocoo()
    r = torch.as_tensor(coo.row, dtype=torch.int64, device=device)
    c = torch.as_tensor(coo.col, dtype=torch.int64, device=device)
    v = torch.as_tensor(coo.data, dtype=torch.float32, device=device)
    dense[r, c] = v
    L = torch.linalg.cholesky(dense)
    del dense
    zt = torch.randn((p, n), generator=g, dtype=torch.float32, device=device)
    xt = torch.linalg.solve_triangular(L, zt, upper=False)
    del L, zt
    return xt.t().contiguous()


def make_x(w: Workload, device: str = "cpu"):
    """Observations for workload ``w``: numpy float64 (CPU) or a torch tensor (CUDA).

    The dtype is the workload's storage type: FP64 and FP32 stay as drawn
    (FP32 workloads are rounded to float32), BF16 workloads are rounded to
    bfloat16 (kept as float32 values on the CPU path).
    """
    om = omega0_for(w)
    if device == "cpu":
        x = sample_x_cpu(om, w.n, w.seed)
        if w.x_dtype == "f32":
            return x.astype(np.float32)
        if w.x_dtype == "bf16":
            return round_to_bf16(x.astype(np.float32))
        return x
    import torch

    x = sample_x_cuda(om, w.n, w.seed, device)
    if w.x_dtype == "bf16":
        return x.to(torch.bfloat16)
    if w.x_dtype == "f64":
        return x.to(torch.float64)
    return x


def small_problem(p: int, n: int, degree: float, seed: int, graph: str = "random",
                  bandwidth: int = 2) -> np.ndarray:
    """A seeded small problem's X (float64), for parity cases the oracle runs in seconds."""
    if graph == "random":
        om = omega0_random(p, degree, seed)
    elif graph == "banded":
        om = omega0_banded(p, bandwidth, seed)
    else:
        om = omega0_tridiagonal(p)
    return sample_x_cpu(om, n, seed)
