"""Comparison of a GPU estimate with a cached FP64 reference of a full-size workload
(tests/golden/ref_<name>.npz, written by tests/golden/make_fullsize_refs.py from the oracle).

- the relative Frobenius error ||Omega - Omega_ref||_F / ||Omega_ref||_F;
- the support rule: an entry in the reference's support only needs |omega_ref,ij| <= 1e-6;
  one in the estimate's support only needs |omega_ij| <= 1e-6 or ||G_ref,ij| - lambda1| <=
  1e-6, with G_ref formed by the oracle from X at the reference estimate (one entry at a
  time);
- that the X a test drew on the device is the X the reference was computed from: FP64 column
  sums against the stored ones, and sampled rows against the CPU draw.
"""
from __future__ import annotations

import json
import os

import numpy as np
import scipy.sparse as sp

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
BAND = 1e-6


def ref_path(name, variant="cov"):
    return os.path.join(GOLDEN, f"ref_{name}" + ("_obs" if variant == "obs" else "") + ".npz")


def load_ref(name, variant="cov"):
    z = np.load(ref_path(name, variant), allow_pickle=False)
    p = int(z["p"])
    om = sp.csr_matrix((z["data"], z["indices"], z["indptr"]), shape=(p, p))
    out = {k: z[k] for k in z.files}
    out["omega"] = om
    return out


def fro(a):
    return float(np.sqrt(a.multiply(a).sum())) if sp.issparse(a) else float(np.linalg.norm(a))


def compare(est: sp.csr_matrix, ref: dict, X_host, lam1, lam2, band=BAND):
    """Relative Frobenius error and the support rule; X_host is the n x p data (for G_ref)."""
    R = ref["omega"].tocsr()
    E = sp.csr_matrix(est).tocsr()
    rel = fro(E - R) / fro(R)
    pe = E.copy()
    pe.data[:] = 1.0
    pr = R.copy()
    pr.data[:] = 1.0
    diff = (pe - pr).tocoo()
    rows, cols = diff.row[diff.data != 0], diff.col[diff.data != 0]
    ok = True
    worst = 0.0
    if rows.size:
        wref = np.asarray(R[rows, cols]).ravel()
        west = np.asarray(E[rows, cols]).ravel()
        g = oracle.gradient_entries(X_host, R, lam2, rows, cols)
        # in the reference only: its value; in the estimate only: its value, or the
        # reference's gradient at the threshold
        dist = np.where(wref != 0, np.abs(wref), np.minimum(np.abs(west), np.abs(np.abs(g) - lam1)))
        worst = float(np.max(dist))
        ok = bool(np.all(dist <= band))
    return {"rel_fro": rel, "support_differences": int(rows.size), "support_worst_band": worst,
            "support_ok": ok, "nnz": int(E.nnz), "nnz_ref": int(R.nnz)}


def check_x(X_dev, ref: dict, omega0, seed, rows=(0, 1, 777), stream=0):
    """The device X against the reference's: column sums (FP64) and sampled rows drawn on the
    CPU, in the workload's storage type.  Returns a dict; raises AssertionError on a mismatch
    beyond the last-bit differences the two draws may have."""
    import torch

    from workloads import cast_x, sample_rows_cpu

    cs = X_dev.double().sum(0).cpu().numpy()
    cref = ref["x_colsum"]
    scale = max(1.0, float(np.max(np.abs(cref))))
    col_err = float(np.max(np.abs(cs - cref))) / scale
    assert col_err <= 1e-6, col_err
    dt = str(ref["x_dtype"])
    cpu = cast_x(sample_rows_cpu(omega0, list(rows), seed, stream), dt).astype(np.float32)
    dev = X_dev[torch.as_tensor(list(rows), device=X_dev.device)].float().cpu().numpy()
    mism = int(np.sum(cpu != dev))
    # a last-bit difference of the FP64 draw can move a value across a rounding boundary
    rel = np.abs(cpu - dev) / np.maximum(np.abs(cpu), 1e-30)
    assert mism <= 4 and (mism == 0 or float(np.max(rel)) <= (2.0 ** -7 if dt == "bf16" else 2.0 ** -23)), mism
    return {"colsum_rel_err": col_err, "sampled_row_mismatches": mism}


def report(record: dict):
    """Append a record to $HPC_REPORT_DIR/refcheck.jsonl when that variable is set."""
    d = os.environ.get("HPC_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, "refcheck.jsonl"), "a") as fh:
            fh.write(json.dumps(record, default=float) + "\n")
