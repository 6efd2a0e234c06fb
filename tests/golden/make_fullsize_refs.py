"""Write the FP64 reference estimate of a full-size workload to tests/golden/ref_<name>[_obs].npz.

It calls the oracle (the CSR-iterate form of Alg. 2, or of Alg. 3 with --variant obs) on
the workload's X drawn on the CPU, and nothing else:

    python tests/golden/make_fullsize_refs.py fp32_p16384 [--variant cov|obs] [--eps 1e-9]
                                             [--workers 8] [--threads 8]

Stored with the estimate (CSR, FP64): the oracle's iteration and trial counts, step sizes
and objective values F; the optimality residual r of the returned estimate and the bound
||Omega - Omega*||_F <= ||r||_F / lambda2 it gives on the distance to the minimiser; and
the column sums and a SHA-256 digest of X as drawn here, so that a user of the file can
check that their X is this one.
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from workloads import WORKLOADS, make_x  # noqa: E402


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=sorted(WORKLOADS))
    ap.add_argument("--variant", default="cov", choices=["cov", "obs"])
    ap.add_argument("--eps", type=float, default=1e-9)
    ap.add_argument("--workers", type=int, default=8)
    ap.add_argument("--threads", type=int, default=8)
    ap.add_argument("--block", type=int, default=512)
    ap.add_argument("--max-iter", type=int, default=2000)
    args = ap.parse_args(argv)
    w = WORKLOADS[args.workload]
    t0 = time.time()

    def log(msg):
        print(f"[{time.time() - t0:8.1f} s] {msg}", flush=True)

    X = make_x(w, device="cpu", workers=args.workers)          # FP32 array (BF16 values for bf16)
    log(f"X {X.shape} {X.dtype} drawn")
    digest = hashlib.sha256(np.ascontiguousarray(X).tobytes()).hexdigest()
    colsum = np.asarray(X, dtype=np.float64).sum(axis=0) if X.shape[1] <= 16384 else \
        sum(np.asarray(X[r:r + 4096], dtype=np.float64).sum(axis=0) for r in range(0, X.shape[0], 4096))
    if args.variant == "cov":
        S = oracle.gram_chunked(X)
        log("S formed")
        del X
        res = oracle.solve_sparse(S, w.lambda1, w.lambda2, eps=args.eps, max_iter=args.max_iter,
                                  block=args.block, threads=args.threads, log=log)
        Gk, _ = oracle.gradient_candidates_cov(S, res.omega, w.lambda1, w.lambda2, args.block, args.threads)
    else:
        res = oracle.solve_obs_sparse(X, w.lambda1, w.lambda2, eps=args.eps, max_iter=args.max_iter,
                                      block=args.block, log=log)
        Xd = np.asarray(X, dtype=np.float64)
        Y = np.asarray(res.omega @ Xd.T)
        Gk = oracle.gradient_candidates_obs(Xd, Y, res.omega, w.lambda1, w.lambda2, args.block)
    r = oracle.kkt_residual_csr(Gk, res.omega, w.lambda1)
    om = res.omega.tocsr()
    om.sort_indices()
    fro = float(np.sqrt(np.sum(om.data ** 2)))
    rn = float(np.linalg.norm(r))
    log(f"{res.status} after {res.iterations} iterations; nnz {om.nnz}; residual {rn:.3e}; "
        f"bound on relative distance {rn / w.lambda2 / fro:.3e}")
    name = f"ref_{w.name}" + ("_obs" if args.variant == "obs" else "")
    np.savez_compressed(
        os.path.join(HERE, name + ".npz"),
        indptr=om.indptr.astype(np.int64), indices=om.indices.astype(np.int32), data=om.data,
        p=w.p, n=w.n, lambda1=w.lambda1, lambda2=w.lambda2, eps=args.eps, variant=args.variant,
        iterations=res.iterations, trials=np.asarray(res.trials), taus=np.asarray(res.taus),
        F=np.asarray(res.F), rel_change=res.rel_change, status=res.status,
        residual_fro=rn, omega_fro=fro, distance_bound_rel=rn / w.lambda2 / fro,
        x_sha256=digest, x_colsum=colsum, x_dtype=w.x_dtype, seconds=time.time() - t0)
    log(f"wrote {name}.npz")


if __name__ == "__main__":
    main()
