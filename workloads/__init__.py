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
* samples: rows of X follow N(0, Omega0^-1).  Omega0 = B^T B with a sparse B
  (one row per off-diagonal pair and one per vertex, which diagonal dominance
  allows); x = Omega0^-1 B^T z with z iid N(0, 1), solved by FP64 conjugate
  gradients.

Everything is a pure function of ``seed``.  numpy's PCG64 draws Omega0.  The
normals z come from the counter-based Philox4x32-10 generator, keyed by the
seed and indexed by (sample row, normal index), so that the CPU draw (numpy)
and the device draw (torch, used at large p) give the same numbers; the two
then differ only by the rounding of the FP64 solve.
"""
from __future__ import annotations

import dataclasses
import math
import warnings

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


# ----------------------------------------------------------------- counter-based normals
#
# Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy
# as 1, 2, 3", SC 2011): ten rounds of two 32 x 32 -> 64-bit multiplications with
# the round keys bumped by two Weyl constants.  It is a pure function of
# (counter, key), written here once over array operators that numpy int64 arrays
# and torch int64 tensors both provide, so the CPU draw and the device draw are
# the same integers.  Every intermediate stays below 2^50: the multiplier is split
# into 16-bit halves, so no signed 64-bit product overflows.

PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57      # round multipliers
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85      # key increments
_MASK32 = 0xFFFFFFFF


def _mulhilo32(m: int, b):
    """(hi, lo) 32-bit words of m * b for a constant m < 2^32 and words b < 2^32."""
    p_lo = b * (m & 0xFFFF)                     # < 2^48
    p_hi = b * (m >> 16)                        # < 2^48
    mid = p_lo + ((p_hi & 0xFFFF) << 16)        # < 2^49
    return (p_hi >> 16) + (mid >> 32), mid & _MASK32


def philox4x32(c0, c1, c2, c3, k0: int, k1: int, rounds: int = 10):
    """The four 32-bit output words of Philox4x32 for counters (c0..c3) and key (k0, k1).

    Counters are int64 arrays (numpy or torch) of 32-bit words, broadcastable to one
    shape; the key is two Python ints."""
    for r in range(rounds):
        h0, l0 = _mulhilo32(PHILOX_M0, c0)
        h1, l1 = _mulhilo32(PHILOX_M1, c2)
        rk0 = (k0 + r * PHILOX_W0) & _MASK32
        rk1 = (k1 + r * PHILOX_W1) & _MASK32
        c0, c1, c2, c3 = h1 ^ c1 ^ rk0, l1, h0 ^ c3 ^ rk1, l0
    return c0, c1, c2, c3


def _key(seed: int, stream: int):
    return seed & _MASK32, (0x5EED0000 + stream) & _MASK32


def normal_pairs(xp, seed: int, stream: int, rows, npairs: int, device=None):
    """Standard normals z[s, k] (k < 2 npairs) for the sample rows ``rows`` (an int array).

    Pair k // 2 of row s comes from one Philox call with counter (k // 2, row, 0, 0) and
    key (seed, stream): two 52-bit uniforms u = (2a + 1) / 2^53 in (0, 1) from its four
    words, then Box-Muller: sqrt(-2 log u1) (cos 2 pi u2, sin 2 pi u2), in FP64.
    ``xp`` is numpy or torch; ``device`` places the torch arrays."""
    if xp is np:
        j = np.arange(npairs, dtype=np.int64)[None, :]
        r = np.asarray(rows, dtype=np.int64)[:, None]
        zero = np.zeros((1, 1), dtype=np.int64)
    else:
        j = xp.arange(npairs, dtype=xp.int64, device=device)[None, :]
        r = xp.as_tensor(np.asarray(rows, dtype=np.int64), device=device)[:, None]
        zero = xp.zeros((1, 1), dtype=xp.int64, device=device)
    k0, k1 = _key(seed, stream)
    w0, w1, w2, w3 = philox4x32(j, r, zero, zero, k0, k1)
    a1 = ((w0 >> 6) << 26) | (w1 >> 6)          # < 2^52
    a2 = ((w2 >> 6) << 26) | (w3 >> 6)
    del w0, w1, w2, w3
    scale = 2.0 ** -53
    if xp is np:
        u1 = (2.0 * a1.astype(np.float64) + 1.0) * scale
        u2 = (2.0 * a2.astype(np.float64) + 1.0) * scale
    else:
        u1 = (2.0 * a1.to(xp.float64) + 1.0) * scale
        u2 = (2.0 * a2.to(xp.float64) + 1.0) * scale
    del a1, a2
    rad = xp.sqrt(-2.0 * xp.log(u1))
    ang = (2.0 * math.pi) * u2
    z = xp.stack([rad * xp.cos(ang), rad * xp.sin(ang)], -1)     # rows x npairs x 2
    return z.reshape(z.shape[0], 2 * npairs)


# ----------------------------------------------------------------- samples of N(0, Omega0^-1)
#
# Omega0 is symmetric with omega_ii >= sum_j |omega_ij| (every generator above), so
# it has an exact sparse factor Omega0 = B^T B: one row sqrt|v| (e_i + sign(v) e_j)
# per off-diagonal pair (i < j, value v) and one row sqrt(r_i) e_i per vertex, with
# r_i = omega_ii - sum_j |omega_ij| >= 0.  With z ~ N(0, I_m) (m = pairs + p),
# b = B^T z has covariance Omega0 and x = Omega0^-1 b has covariance
# Omega0^-1 Omega0 Omega0^-1 = Omega0^-1: rows of X follow N(0, Omega0^-1) without a
# dense factorisation.  The solve is Jacobi-preconditioned conjugate gradients in
# FP64 for a fixed number of iterations set by the Gershgorin bound of the scaled
# matrix, enough to reach FP64 rounding.

@dataclasses.dataclass
class SampleFactor:
    p: int
    m: int                       # normals per sample: off-diagonal pairs + p
    Bt: sp.csr_matrix            # B^T, p x m
    omega: sp.csr_matrix         # Omega0, p x p
    diag: np.ndarray             # diagonal of Omega0
    cg_iters: int


def sample_factor(omega0: sp.csr_matrix) -> SampleFactor:
    """B^T of Omega0 = B^T B (columns: the pairs i < j in row-major order, then the
    vertices) and the CG iteration count."""
    om = sp.csr_matrix(omega0, dtype=np.float64)
    om.sort_indices()
    p = om.shape[0]
    up = sp.triu(om, k=1).tocsr()
    up.sort_indices()
    iu = np.repeat(np.arange(p, dtype=np.int64), np.diff(up.indptr))
    ju = up.indices.astype(np.int64)
    v = up.data
    E = v.size
    diag = om.diagonal().copy()
    absoff = np.asarray(abs(om).sum(axis=1)).ravel() - np.abs(diag)
    rem = diag - absoff
    if np.any(rem < -1e-12 * np.maximum(diag, 1.0)):
        raise ValueError("Omega0 is not diagonally dominant; the sparse factor does not exist")
    rem = np.maximum(rem, 0.0)
    s = np.sqrt(np.abs(v))
    rows = np.concatenate([iu, ju, np.arange(p, dtype=np.int64)])
    cols = np.concatenate([np.arange(E), np.arange(E), E + np.arange(p)])
    vals = np.concatenate([s, np.sign(v) * s, np.sqrt(rem)])
    Bt = sp.csr_matrix((vals, (rows, cols)), shape=(p, E + p))
    Bt.sort_indices()
    # D^-1/2 Omega0 D^-1/2 has the eigenvalues of D^-1 Omega0, inside the Gershgorin discs
    # centred at 1 of radius sum_j |omega_ij| / omega_ii <= rho < 1; CG error then falls by
    # (sqrt(k) - 1) / (sqrt(k) + 1) per iteration with k = (1 + rho) / (1 - rho)
    rho = float(np.max(absoff / diag))
    kappa = (1.0 + rho) / (1.0 - rho)
    rate = (math.sqrt(kappa) - 1.0) / (math.sqrt(kappa) + 1.0)
    iters = 4 if rate <= 0 else int(math.ceil(math.log(0.5e-17) / math.log(rate))) + 2
    return SampleFactor(p, E + p, Bt, om, diag, min(iters, 500))


def _cg_numpy(f: SampleFactor, b: np.ndarray) -> np.ndarray:
    """Omega0^-1 b for the columns of b (p x c), Jacobi-preconditioned CG, FP64."""
    d = f.diag[:, None]
    x = b / d
    r = b - f.omega @ x
    z = r / d
    q = z.copy()
    rz = np.sum(r * z, axis=0)
    for _ in range(f.cg_iters):
        Aq = f.omega @ q
        qAq = np.sum(q * Aq, axis=0)
        alpha = np.where(qAq > 0.0, rz / np.where(qAq > 0.0, qAq, 1.0), 0.0)
        x += alpha * q
        r -= alpha * Aq
        z = r / d
        rz_new = np.sum(r * z, axis=0)
        beta = np.where(rz > 0.0, rz_new / np.where(rz > 0.0, rz, 1.0), 0.0)
        q = z + beta * q
        rz = rz_new
    return x


def _rows_numpy(f: SampleFactor, seed: int, rows: np.ndarray, stream: int) -> np.ndarray:
    z = normal_pairs(np, seed, stream, rows, (f.m + 1) // 2)[:, : f.m]
    b = f.Bt @ z.T                                  # p x c
    del z
    return np.ascontiguousarray(_cg_numpy(f, b).T)


def _rows_worker(args):
    om, seed, r0, r1, stream, x_dtype = args
    f = sample_factor(om)
    return r0, cast_x(_rows_numpy(f, seed, np.arange(r0, r1, dtype=np.int64), stream), x_dtype)


def sample_x_cpu(omega0: sp.csr_matrix, n: int, seed: int, stream: int = 0, workers: int = 1,
                 chunk: int = 64, x_dtype: str = "f64") -> np.ndarray:
    """n samples of N(0, Omega0^-1) as the rows of an n x p array, on the CPU.

    Row s is a pure function of (Omega0, seed, stream, s), computed in FP64 and stored in
    the storage type ``x_dtype`` (cast_x).  ``workers`` > 1 spreads the rows over
    processes started with spawn; the result does not depend on it."""
    f = sample_factor(omega0)
    out = np.empty((n, f.p), dtype=np.float64 if x_dtype == "f64" else np.float32)
    if workers <= 1 or n <= chunk:
        for r0 in range(0, n, chunk):
            r1 = min(n, r0 + chunk)
            out[r0:r1] = cast_x(_rows_numpy(f, seed, np.arange(r0, r1, dtype=np.int64), stream), x_dtype)
        return out
    import multiprocessing as mp

    jobs = [(f.omega, seed, r0, min(n, r0 + chunk), stream, x_dtype) for r0 in range(0, n, chunk)]
    with mp.get_context("spawn").Pool(workers) as pool:
        for r0, rows in pool.imap_unordered(_rows_worker, jobs):
            out[r0:r0 + rows.shape[0]] = rows
    return out


def sample_rows_cpu(omega0: sp.csr_matrix, rows, seed: int, stream: int = 0) -> np.ndarray:
    """Selected rows (float64) of the sample matrix that sample_x_cpu / sample_x_cuda draw."""
    f = sample_factor(omega0)
    return _rows_numpy(f, seed, np.asarray(rows, dtype=np.int64), stream)


def sample_x_cuda(omega0: sp.csr_matrix, n: int, seed: int, stream: int = 0, device: str = "cuda",
                  chunk: int = 2048):
    """The samples of sample_x_cpu drawn with torch on ``device`` (float64 n x p tensor).

    The same normals (Philox integers, FP64 Box-Muller) and the same FP64 CG: the two
    agree to rounding (the order of the CG's sums, and the last bit of log and cos)."""
    import torch

    f = sample_factor(omega0)

    def csr_t(a):
        a = sp.csr_matrix(a)
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")       # torch flags sparse CSR support as beta
            return torch.sparse_csr_tensor(torch.as_tensor(a.indptr, dtype=torch.int64),
                                           torch.as_tensor(a.indices, dtype=torch.int64),
                                           torch.as_tensor(a.data, dtype=torch.float64), size=a.shape,
                                           check_invariants=False).to(device)

    Bt = csr_t(f.Bt)
    Om = csr_t(f.omega)
    d = torch.as_tensor(f.diag, dtype=torch.float64, device=device)[:, None]
    out = torch.empty((n, f.p), dtype=torch.float64, device=device)
    for r0 in range(0, n, chunk):
        r1 = min(n, r0 + chunk)
        z = normal_pairs(torch, seed, stream, np.arange(r0, r1), (f.m + 1) // 2, device=device)[:, : f.m]
        b = Bt @ z.t().contiguous()
        del z
        x = b / d
        r = b - Om @ x
        del b
        zz = r / d
        q = zz.clone()
        rz = (r * zz).sum(0)
        for _ in range(f.cg_iters):
            Aq = Om @ q
            qAq = (q * Aq).sum(0)
            alpha = torch.where(qAq > 0, rz / torch.where(qAq > 0, qAq, torch.ones_like(qAq)),
                                torch.zeros_like(qAq))
            x += alpha * q
            r -= alpha * Aq
            zz = r / d
            rz_new = (r * zz).sum(0)
            beta = torch.where(rz > 0, rz_new / torch.where(rz > 0, rz, torch.ones_like(rz)),
                               torch.zeros_like(rz))
            q = zz + beta * q
            rz = rz_new
        out[r0:r1] = x.t()
        del x, r, zz, q, Aq
    return out


def cast_x(x, x_dtype: str):
    """The workload's storage type: FP64 kept, FP32 rounded once, BF16 rounded to FP32 and
    then to BF16 (nearest, ties to even) -- on numpy float64 arrays (BF16 values returned
    as float32) or torch float64 tensors."""
    if isinstance(x, np.ndarray):
        if x_dtype == "f32":
            return x.astype(np.float32)
        if x_dtype == "bf16":
            return round_to_bf16(x.astype(np.float32))
        return x
    import torch

    if x_dtype == "f32":
        return x.to(torch.float32)
    if x_dtype == "bf16":
        return x.to(torch.float32).to(torch.bfloat16)
    return x


def make_x(w: Workload, device: str = "cpu", workers: int = 1, stream: int = 0):
    """Observations for workload ``w`` in its storage type: a numpy array (CPU; BF16
    values as float32) or a torch tensor on a CUDA device."""
    om = omega0_for(w)
    if device == "cpu":
        return sample_x_cpu(om, w.n, w.seed, stream=stream, workers=workers, x_dtype=w.x_dtype)
    x = sample_x_cuda(om, w.n, w.seed, stream=stream, device=device)
    out = cast_x(x, w.x_dtype)
    del x
    return out


# The held-out draw of a workload: the same Omega0 and seed, Philox key stream 1.
HELDOUT_STREAM = 1


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


def hub_factor_problem(p: int, n: int, seed: int, loading: float = 0.5) -> np.ndarray:
    """A one-factor X (float64, n x p) with a hub column: x_0 = z and x_j = loading z + e_j
    (z, e_j iid N(0, 1)), so that S_0j is near loading for every j while the other
    off-diagonal entries of S stay near loading^2.  Its precision matrix is a star centred
    on column 0; at lambda1 between loading^2 and loading the hub row's candidate list
    holds about p entries at every iteration (an edge case of the candidate sort)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    z = rng.standard_normal(n)
    X = rng.standard_normal((n, p))
    X[:, 0] = z
    X[:, 1:] += loading * z[:, None]
    return X
