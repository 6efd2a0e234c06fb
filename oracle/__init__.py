"""Plain FP64 CPU oracle of the CONCORD/PseudoNet proximal-gradient method.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The GPU library and
its Python binding never import, call or execute anything here, and this
package shares no code with them; the two meet only through the seeded arrays
of ``workloads``.

What it computes (HP-CONCORD, arXiv:1710.10769):

* ``gram``            S = X^T X / n                       (Alg. 1 step 2, Alg. 2 step 2)
* ``soft_threshold``  the elementwise operator of eq. (2)
* ``prox``            eq. (2) applied to the off-diagonal entries only
* ``gradient``        G = -diag(1/w_ii) + (W + W^T)/2 + lam2*Omega, W = Omega S
                                                            (Alg. 1 step 4, Alg. 2 steps 5-6)
* ``smooth``          g(Omega) = -sum log w_ii + tr(W Omega)/2 + lam2/2 ||Omega||_F^2
                                                            (Alg. 2 step 7, scaled as below)
* ``iterate``/``solve``  Alg. 1 / Alg. 2: backtracking over tau = 1, 1/2, 1/4, ...
                      with a fresh W+ = Omega+ S per trial and the sufficient-
                      decrease test of Alg. 1 step 9 / Alg. 2 step 12
* ``solve_obs``       Alg. 3 (Y = Omega X^T, Z = Y X / n, ||Y||^2 / n)
* ``*_entries``       single entries of S and G formed straight from X, for
                      sampled checks at sizes where the dense oracle is too slow

Readings of the paper (where it is silent, ambiguous or garbled):

* Scaling (eq. 1 vs Alg. 1 step 4): the smooth part is
  f = -sum log w_ii + tr(Omega S Omega)/2 + lam2/2 ||Omega||_F^2, whose gradient
  is exactly the G of Alg. 1 step 4; the line search uses this f.
* The l1 term counts every off-diagonal entry (both triangles); each entry is
  thresholded at tau*lam1.
* The diagonal is not thresholded (the penalty is on Omega_X only).
* A trial with any w+_ii <= 0 fails (the log needs a positive diagonal) and tau halves.
* tau restarts at 1 every outer iteration, shrinks by 1/2, at most 60 halvings.
* Ties in eq. (2): |z| <= alpha maps to 0.
* Stopping: ||Omega+ - Omega||_F / ||Omega||_F < eps.
* Obs scaling: Y = Omega X^T unscaled, Z = Y X / n, tr(Omega S Omega) = ||Y||_F^2 / n.
* S is not centred and is divided by n.

Numerical floor.  The test of Alg. 1 step 9 compares two O(|g|) numbers whose
difference is O(||Delta||^2); in FP64 it decides reliably while
||Delta||_F / ||Omega||_F stays above ~1e-8.  Parity references therefore stop
at eps = 1e-9 at most, and a line search that runs out of halvings after the
relative change has already dropped below 1e-8 is reported as converged
(``status == "floor"``) rather than as a failure.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp


# ----------------------------------------------------------------- building blocks

def gram(X) -> np.ndarray:
    """S = X^T X / n in FP64 (Alg. 1 step 2); X is n x p, rows are observations."""
    X = np.asarray(X, dtype=np.float64)
    return (X.T @ X) / X.shape[0]


def soft_threshold(Z, alpha):
    """Eq. (2): z - alpha if z > alpha, z + alpha if z < -alpha, otherwise 0."""
    Z = np.asarray(Z, dtype=np.float64)
    return np.where(Z > alpha, Z - alpha, np.where(Z < -alpha, Z + alpha, 0.0))


def prox(Z, alpha):
    """Proximal map of alpha*||Z_X||_1: eq. (2) off the diagonal, diagonal kept."""
    out = soft_threshold(Z, alpha)
    np.fill_diagonal(out, np.diag(Z))
    return out


def times_S(Omega, S):
    """W = Omega S, the sparse-dense product of Alg. 2 steps 3 and 10."""
    return np.asarray(sp.csr_matrix(Omega) @ S)


def gradient(Omega, W, lam2):
    """G = -(Omega_D)^-1 + (W^T + W)/2 + lam2*Omega (Alg. 2 step 6, W = Omega S)."""
    G = 0.5 * (W.T + W) + lam2 * Omega
    G[np.diag_indices_from(G)] -= 1.0 / np.diag(Omega)
    return G


def smooth(Omega, W, lam2):
    """g(Omega) = -sum_i log w_ii + tr(W Omega)/2 + lam2/2 ||Omega||_F^2 (Alg. 2 step 7).

    Returns +inf when a diagonal entry is not positive (the log is undefined).
    """
    d = np.diag(Omega)
    if np.any(d <= 0.0):
        return np.inf
    tr_wo = np.sum(W * Omega.T)          # tr(W Omega) = sum_ij W_ij Omega_ji
    return -np.sum(np.log(d)) + 0.5 * tr_wo + 0.5 * lam2 * np.sum(Omega * Omega)


def penalty(Omega, lam1):
    """lam1 * sum_{i != j} |w_ij| (both triangles)."""
    a = np.abs(Omega)
    return lam1 * (a.sum() - np.trace(a))


def objective(S, Omega, lam1, lam2):
    """F(Omega) = g(Omega) + lam1 ||Omega_X||_1."""
    return smooth(Omega, times_S(Omega, S), lam2) + penalty(Omega, lam1)


# ----------------------------------------------------------------- Alg. 1 / Alg. 2

@dataclasses.dataclass
class Step:
    omega: np.ndarray
    W: np.ndarray
    tau: float
    trials: int
    accepted: bool
    G: np.ndarray
    g: float


def iterate(S, Omega, W, lam1, lam2, tau0=1.0, shrink=0.5, max_halvings=60) -> Step:
    """One outer iteration of Alg. 2 (steps 5-12) from the iterate Omega with W = Omega S."""
    G = gradient(Omega, W, lam2)
    g = smooth(Omega, W, lam2)
    tau = tau0
    for h in range(max_halvings + 1):
        Op = prox(Omega - tau * G, tau * lam1)             # step 9
        if np.all(np.diag(Op) > 0.0):
            Wp = times_S(Op, S)                             # step 10
            gp = smooth(Op, Wp, lam2)                       # step 11
            D = Op - Omega
            # step 12: g(O+) <= g(O) - tr((O - O+)^T G) + ||O - O+||^2 / (2 tau)
            rhs = g - np.sum((Omega - Op) * G) + np.sum(D * D) / (2.0 * tau)
            if gp <= rhs:
                return Step(Op, Wp, tau, h + 1, True, G, g)
        tau *= shrink
    return Step(Omega, W, tau, max_halvings + 1, False, G, g)


@dataclasses.dataclass
class Result:
    omega: np.ndarray
    iterations: int
    trials: list
    taus: list
    F: list                 # F(Omega^k) for k = 0..iterations
    rel_change: float
    status: str             # "converged" | "floor" | "max_iter" | "ls_fail"


def solve(S, lam1, lam2, eps=1e-6, max_iter=1000, omega0=None, tau0=1.0, shrink=0.5,
          max_halvings=60) -> Result:
    """Alg. 2 (the Cov variant of Alg. 1): Omega^0 = I, iterate until the relative change < eps."""
    S = np.asarray(S, dtype=np.float64)
    p = S.shape[0]
    Omega = np.eye(p) if omega0 is None else np.array(omega0, dtype=np.float64)
    W = times_S(Omega, S)                                   # step 3
    F = [smooth(Omega, W, lam2) + penalty(Omega, lam1)]
    trials, taus = [], []
    rel = np.inf
    status = "max_iter"
    for _ in range(max_iter):
        st = iterate(S, Omega, W, lam1, lam2, tau0, shrink, max_halvings)
        if not st.accepted:
            status = "floor" if rel < 1e-8 else "ls_fail"
            break
        rel = np.linalg.norm(st.omega - Omega) / np.linalg.norm(Omega)
        Omega, W = st.omega, st.W
        trials.append(st.trials)
        taus.append(st.tau)
        F.append(smooth(Omega, W, lam2) + penalty(Omega, lam1))
        if rel < eps:
            status = "converged"
            break
    return Result(Omega, len(trials), trials, taus, F, float(rel), status)


# ----------------------------------------------------------------- Alg. 3 (Obs)

def solve_obs(X, lam1, lam2, eps=1e-6, max_iter=1000, tau0=1.0, shrink=0.5,
              max_halvings=60) -> Result:
    """Alg. 3: never forms S; Y = Omega X^T, Z = Y X / n, tr(Omega S Omega) = ||Y||^2 / n."""
    X = np.asarray(X, dtype=np.float64)
    n, p = X.shape
    Xt = X.T

    def g_of(Om, Y):
        d = np.diag(Om)
        if np.any(d <= 0.0):
            return np.inf
        return -np.sum(np.log(d)) + 0.5 * np.sum(Y * Y) / n + 0.5 * lam2 * np.sum(Om * Om)

    Omega = np.eye(p)
    Y = np.asarray(sp.csr_matrix(Omega) @ Xt)               # step 2
    F = [g_of(Omega, Y) + penalty(Omega, lam1)]
    trials, taus = [], []
    rel = np.inf
    status = "max_iter"
    for _ in range(max_iter):
        Z = (Y @ X) / n                                     # step 4
        G = gradient(Omega, Z, lam2)                        # steps 5-6
        g = g_of(Omega, Y)                                  # step 7
        tau, accepted = tau0, False
        for h in range(max_halvings + 1):
            Op = prox(Omega - tau * G, tau * lam1)          # step 9
            if np.all(np.diag(Op) > 0.0):
                Yp = np.asarray(sp.csr_matrix(Op) @ Xt)     # step 10
                gp = g_of(Op, Yp)                           # step 11
                D = Op - Omega
                if gp <= g - np.sum((Omega - Op) * G) + np.sum(D * D) / (2.0 * tau):
                    accepted = True
                    break
            tau *= shrink
        if not accepted:
            status = "floor" if rel < 1e-8 else "ls_fail"
            break
        rel = np.linalg.norm(Op - Omega) / np.linalg.norm(Omega)
        Omega, Y = Op, Yp
        trials.append(h + 1)
        taus.append(tau)
        F.append(g_of(Omega, Y) + penalty(Omega, lam1))
        if rel < eps:
            status = "converged"
            break
    return Result(Omega, len(trials), trials, taus, F, float(rel), status)


# ----------------------------------------------------------------- sampled entries

def _columns(X, idx):
    return np.asarray(X[:, idx], dtype=np.float64)


def gram_entries(X, rows, cols) -> np.ndarray:
    """S_ij = sum_k X_ki X_kj / n for the listed pairs, in FP64, straight from X."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    n = X.shape[0]
    uniq, inv = np.unique(np.concatenate([rows, cols]), return_inverse=True)
    C = _columns(X, uniq)
    a = C[:, inv[: rows.size]]
    b = C[:, inv[rows.size:]]
    return np.einsum("ki,ki->i", a, b) / n


def gradient_entries(X, omega_csr: sp.csr_matrix, lam2, rows, cols) -> np.ndarray:
    """G_ij of Alg. 1 step 4 at the listed pairs for a sparse symmetric Omega, from X.

    W_ij = sum_k w_ik S_kj (Alg. 2 step 3) with S = X^T X / n, summed in FP64 as
    <X w_i, x_j> / n: the column X w_i = sum_k w_ik x_k is formed once per row i that the
    pairs name, and W_ji = <X w_j, x_i> / n likewise.
    """
    om = sp.csr_matrix(omega_csr, dtype=np.float64)
    om.sort_indices()
    n = X.shape[0]
    X = np.asfortranarray(X)                 # columns contiguous: x_k is one slice
    w_pairs = np.asarray(om[np.asarray(rows), np.asarray(cols)], dtype=np.float64).ravel()
    diag = om.diagonal()
    xw = {}

    def x_omega(i):
        if i not in xw:
            ki = om.indices[om.indptr[i]:om.indptr[i + 1]]
            vi = om.data[om.indptr[i]:om.indptr[i + 1]]
            xw[i] = _columns(X, ki) @ vi if ki.size else np.zeros(n)
        return xw[i]

    out = np.empty(len(rows))
    for t, (i, j) in enumerate(zip(rows, cols)):
        i, j = int(i), int(j)
        xi = np.asarray(X[:, i], dtype=np.float64)
        xj = np.asarray(X[:, j], dtype=np.float64)
        w_ij = (x_omega(i) @ xj) / n
        w_ji = (x_omega(j) @ xi) / n
        g = 0.5 * (w_ij + w_ji) + lam2 * w_pairs[t]
        if i == j:
            g -= 1.0 / diag[i]
        out[t] = g
    return out


def smooth_sparse_from_S(S, omega_csr: sp.csr_matrix, lam2) -> float:
    """g(Omega) for a sparse symmetric Omega and a dense S (row sums of w_i^T S w_i)."""
    om = sp.csr_matrix(omega_csr, dtype=np.float64)
    d = om.diagonal()
    if np.any(d <= 0.0):
        return np.inf
    W = om @ S
    tr = float(np.sum(om.multiply(W)))
    return -float(np.sum(np.log(d))) + 0.5 * tr + 0.5 * lam2 * float(om.multiply(om).sum())


# ----------------------------------------------------------------- differentiation

def smooth_loss(X, Omega, lam2):
    """L(Omega, X) = -sum log w_ii + tr(Omega S Omega)/2 + lam2/2 ||Omega||_F^2 with S = X^T X / n:
    the smooth part of the objective under the scaling reading, as a function of both inputs."""
    X = np.asarray(X, dtype=np.float64)
    S = gram(X)
    d = np.diag(Omega)
    return -np.sum(np.log(d)) + 0.5 * np.trace(Omega @ S @ Omega) + 0.5 * lam2 * np.sum(Omega * Omega)


def smooth_loss_grads(X, Omega, lam2):
    """(dL/dOmega, dL/dX) of smooth_loss for any square Omega with a positive diagonal.

    d tr(Omega S Omega) = <dOmega, Omega^T S + S Omega^T> gives
        dL/dOmega = -diag(1/w_ii) + (Omega^T S + S Omega^T)/2 + lam2 Omega;
    tr(Omega X^T X Omega) / (2n) differentiates to
        dL/dX = (X Omega Omega + X Omega^T Omega^T) / (2n),
    which at a symmetric Omega are Alg. 1's G and Y Omega / n with Y = X Omega.
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    S = gram(X)
    dOm = 0.5 * (Omega.T @ S + S @ Omega.T) + lam2 * Omega
    dOm[np.diag_indices_from(dOm)] -= 1.0 / np.diag(Omega)
    dX = (X @ Omega @ Omega + X @ Omega.T @ Omega.T) / (2.0 * n)
    return dOm, dX


def heldout_loss(S_val, Omega):
    """L_val(Omega) = -sum log w_ii + tr(Omega S_val Omega)/2: the unpenalised pseudolikelihood loss on
    held-out data (the model-selection criterion differentiated by hypergrad)."""
    d = np.diag(Omega)
    return -np.sum(np.log(d)) + 0.5 * np.sum((Omega @ S_val) * Omega.T)


def hypergrad(S, S_val, Omega, lam1, lam2):
    """(dL_val/dlambda1, dL_val/dlambda2) at the estimate Omega(lambda) by the implicit function theorem.

    On the support A of Omega (both triangles and the diagonal) the fixed point of Alg. 1 satisfies
    G_ij(Omega) + lambda1 s_ij = 0 with s_ij = sign(w_ij) off the diagonal and 0 on it.  With A held
    fixed, d/dlambda of that system gives H_A[dOmega/dlambda1] = -s and H_A[dOmega/dlambda2] = -Omega_A,
    where H_A is the Hessian of the smooth part restricted to symmetric matrices supported on A,
        H[E] = (E S + S E)/2 + lambda2 E + diag(E_ii / w_ii^2),
    so dL_val/dlambda = <grad L_val, dOmega/dlambda> with grad L_val = -diag(1/w) + (Omega S_val + S_val Omega)/2.
    H_A is formed explicitly on the unique pairs i <= j of A and solved densely: small p only.
    """
    p = S.shape[0]
    iu, ju = np.nonzero(np.triu(Omega != 0.0))
    m = iu.size
    idx = {(int(i), int(j)): t for t, (i, j) in enumerate(zip(iu, ju))}
    d = np.diag(Omega)
    Hm = np.zeros((m, m))
    for t, (a, b) in enumerate(zip(iu, ju)):
        E = np.zeros((p, p))
        E[a, b] = E[b, a] = 1.0
        HE = 0.5 * (E @ S + S @ E) + lam2 * E
        HE[np.diag_indices(p)] += np.diag(E) / d ** 2
        Hm[:, t] = HE[iu, ju]
    gval = 0.5 * (Omega @ S_val + S_val @ Omega)
    gval[np.diag_indices(p)] -= 1.0 / d
    v = np.linalg.solve(Hm, gval[iu, ju])
    w = np.where(iu == ju, 1.0, 2.0)          # full-entry inner product on symmetric matrices
    s = np.where(iu == ju, 0.0, np.sign(Omega[iu, ju]))
    return float(-np.sum(w * v * s)), float(-np.sum(w * v * Omega[iu, ju]))


def hypergrad_sparse(X, Xval, omega_csr: sp.csr_matrix, lam1, lam2):
    """hypergrad() at a sparse estimate for large p: the same implicit-function gradient, with
    H_A assembled as a sparse matrix on the unique pairs (i <= j) of the support and every S
    and S_val entry it needs formed from X and X_val in FP64 (gram_entries).  Returns
    (dL_val/dlambda1, dL_val/dlambda2)."""
    import scipy.sparse.linalg as spla

    om = sp.csr_matrix(omega_csr, dtype=np.float64)
    om.sort_indices()
    p = om.shape[0]
    rows = np.repeat(np.arange(p), np.diff(om.indptr))
    cols = om.indices
    vals = om.data
    up = rows <= cols
    U = list(zip(rows[up].tolist(), cols[up].tolist()))
    uid = {u: t for t, u in enumerate(U)}
    supp = [om.indices[om.indptr[i]:om.indptr[i + 1]] for i in range(p)]
    wrow = [om.data[om.indptr[i]:om.indptr[i + 1]] for i in range(p)]
    diag = om.diagonal()
    # every S entry (k, j) with k, j in the support of one row
    need_k, need_j = [], []
    for i in range(p):
        for k in supp[i]:
            for j in supp[i]:
                need_k.append(k)
                need_j.append(j)
    need_k = np.asarray(need_k, np.int64)
    need_j = np.asarray(need_j, np.int64)
    Sv = dict(zip(zip(need_k.tolist(), need_j.tolist()), gram_entries(X, need_k, need_j).tolist()))
    Svv = dict(zip(zip(need_k.tolist(), need_j.tolist()), gram_entries(Xval, need_k, need_j).tolist()))

    def key(a, b):
        return uid[(a, b) if a <= b else (b, a)]

    # H on U: H[E]_ij = ((E S)_ij + (E S)_ji)/2 + lambda2 E_ij + [i=j] E_ii / w_ii^2,
    # (E S)_ij = sum_{k in supp(i)} E_ik S_kj with E symmetric on the support
    r_, c_, v_ = [], [], []
    for t, (i, j) in enumerate(U):
        for k in supp[i]:
            r_.append(t); c_.append(key(i, k)); v_.append(0.5 * Sv[(k, j)])
        for k in supp[j]:
            r_.append(t); c_.append(key(j, k)); v_.append(0.5 * Sv[(k, i)])
        r_.append(t); c_.append(t); v_.append(lam2 + (1.0 / diag[i] ** 2 if i == j else 0.0))
    H = sp.csr_matrix((v_, (r_, c_)), shape=(len(U), len(U)))
    # gradient of L_val on U
    b = np.empty(len(U))
    for t, (i, j) in enumerate(U):
        a1 = sum(w * Svv[(k, j)] for k, w in zip(supp[i], wrow[i]))
        a2 = sum(w * Svv[(k, i)] for k, w in zip(supp[j], wrow[j]))
        b[t] = 0.5 * (a1 + a2) - (1.0 / diag[i] if i == j else 0.0)
    v = spla.spsolve(H.tocsc(), b)
    wgt = np.array([1.0 if i == j else 2.0 for i, j in U])
    om_u = np.array([om[i, j] for i, j in U])
    s_u = np.where(np.array([i == j for i, j in U]), 0.0, np.sign(om_u))
    return float(-np.sum(wgt * v * s_u)), float(-np.sum(wgt * v * om_u))


# ----------------------------------------------------------------- CSR iterate form (large p)
#
# The same Alg. 2 / Alg. 3 with the iterate Omega and every trial Omega+ held as CSR, so
# that p = 16384 and p = 65536 fit in host memory next to a dense FP64 S.  The steps and
# their order are those of ``solve`` / ``solve_obs``; three things change only the storage:
#
# * W = Omega S (step 3) and G (steps 5-6) are formed in blocks of rows, and G is kept on
#   K = supp(Omega) + diagonal + {(i, j): |G_ij| > lambda1}.  Outside K an entry of
#   Omega - tau G is -tau G_ij with |tau G_ij| <= tau lambda1 (tau is a power of two, so
#   the scaling is exact), which eq. (2) maps to 0 for every tau of the line search; such
#   entries add nothing to Omega+, to <Omega - Omega+, G> or to ||Omega+ - Omega||^2.
# * tr(W+ Omega+) in g(Omega+) (steps 10-11) needs W+ = Omega+ S only on supp(Omega+):
#   W+_ij = sum_k w+_ik S_kj over the row's support.
# * S = X^T X / n is formed one block of columns at a time (S[I, J] = X_I^T X_J / n, the
#   upper blocks, mirrored).

def gram_chunked(X, block=4096) -> np.ndarray:
    """S = X^T X / n in FP64 (Alg. 2 step 2), one block of columns at a time: S[I, J] = X_I^T X_J / n
    for the blocks I <= J, mirrored to S[J, I]; each diagonal block is made exactly symmetric
    from its upper triangle.  X may be float32 (converted block by block).  Returns a C-ordered
    p x p float64 array."""
    n, p = X.shape
    S = np.empty((p, p), dtype=np.float64)
    for j0 in range(0, p, block):
        XJ = np.asarray(X[:, j0:j0 + block], dtype=np.float64)
        for i0 in range(0, j0 + 1, block):
            XI = XJ if i0 == j0 else np.asarray(X[:, i0:i0 + block], dtype=np.float64)
            B = (XI.T @ XJ) / n
            if i0 == j0:
                S[j0:j0 + block, j0:j0 + block] = np.triu(B) + np.triu(B, 1).T
            else:
                S[i0:i0 + block, j0:j0 + block] = B
                S[j0:j0 + block, i0:i0 + block] = B.T
    return S


def _csr_identity(p):
    I = sp.identity(p, format="csr", dtype=np.float64)
    I.sort_indices()
    return I


def _blocks(p, block):
    return [(r0, min(p, r0 + block)) for r0 in range(0, p, block)]


def gradient_candidates_cov(S, omega: sp.csr_matrix, lam1, lam2, block=512, threads=8):
    """Steps 3 and 5-6 of Alg. 2 for a CSR iterate: W = Omega S and
    G = (W + W^T)/2 + lam2 Omega - diag(1/w_ii), formed in row blocks.

    Returns (Gk, Wsupp): G on K = supp(Omega) + diagonal + {|G_ij| > lam1} as CSR, and
    W on supp(Omega) as a CSR with Omega's pattern."""
    from concurrent.futures import ThreadPoolExecutor

    p = S.shape[0]
    om = omega
    dinv = 1.0 / om.diagonal()

    def one(rb):
        r0, r1 = rb
        WI = np.asarray(om[r0:r1] @ S)                                  # rows r0..r1 of W
        WtI = np.asarray(om @ np.ascontiguousarray(S[:, r0:r1])).T      # rows r0..r1 of W^T
        OI = om[r0:r1].toarray()
        GI = 0.5 * (WtI + WI) + lam2 * OI
        rr = np.arange(r1 - r0)
        GI[rr, r0 + rr] -= dinv[r0:r1]
        keep = (np.abs(GI) > lam1) | (OI != 0.0)
        keep[rr, r0 + rr] = True
        i, j = np.nonzero(keep)
        si, sj = np.nonzero(OI != 0.0)
        return (i + r0, j, GI[i, j]), (si + r0, sj, WI[si, sj])

    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(one, _blocks(p, block)))
    gi = np.concatenate([a[0][0] for a in parts])
    gj = np.concatenate([a[0][1] for a in parts])
    gv = np.concatenate([a[0][2] for a in parts])
    wi = np.concatenate([a[1][0] for a in parts])
    wj = np.concatenate([a[1][1] for a in parts])
    wv = np.concatenate([a[1][2] for a in parts])
    Gk = sp.csr_matrix((gv, (gi, gj)), shape=(p, p))
    Gk.sort_indices()
    Wsupp = sp.csr_matrix((wv, (wi, wj)), shape=(p, p))
    Wsupp.sort_indices()
    return Gk, Wsupp


def w_on_support(S, omega: sp.csr_matrix) -> np.ndarray:
    """W = Omega S at the entries of supp(Omega), in CSR order: W_ij = sum_k w_ik S_kj over
    the row's support (step 10, restricted to the entries step 11 reads)."""
    om = omega
    L = np.diff(om.indptr)
    row = np.repeat(np.arange(om.shape[0]), L)
    rep = L[row]                                   # each entry pairs with every entry of its row
    u = np.repeat(np.arange(om.nnz), rep)
    start = np.repeat(np.cumsum(rep) - rep, rep)
    v = om.indptr[row][u] + (np.arange(u.size) - start)
    # entry v = (i, j) receives w_ik S_kj from entry u = (i, k)
    return np.bincount(v, weights=om.data[u] * S[om.indices[u], om.indices[v]], minlength=om.nnz)


def smooth_csr(omega: sp.csr_matrix, w_supp, lam2) -> float:
    """g(Omega) = -sum log w_ii + tr(W Omega)/2 + lam2/2 ||Omega||^2 with W given on supp(Omega)
    (an array in Omega's CSR order)."""
    d = omega.diagonal()
    if np.any(d <= 0.0):
        return np.inf
    return -float(np.sum(np.log(d))) + 0.5 * float(np.sum(w_supp * omega.data)) + \
        0.5 * lam2 * float(np.sum(omega.data * omega.data))


def penalty_csr(omega: sp.csr_matrix, lam1) -> float:
    a = np.abs(omega.data)
    return lam1 * (float(a.sum()) - float(np.sum(np.abs(omega.diagonal()))))


def _on_pattern(A: sp.csr_matrix, pattern: sp.csr_matrix) -> np.ndarray:
    """Values of A at the entries of ``pattern`` (0 where A has none), in pattern's CSR order."""
    rows = np.repeat(np.arange(pattern.shape[0]), np.diff(pattern.indptr))
    return np.asarray(A[rows, pattern.indices]).ravel()


def prox_csr(Zk: sp.csr_matrix, alpha) -> sp.csr_matrix:
    """eq. (2) on the off-diagonal entries of a CSR matrix, diagonal kept; zeros dropped."""
    rows = np.repeat(np.arange(Zk.shape[0]), np.diff(Zk.indptr))
    off = rows != Zk.indices
    v = Zk.data.copy()
    v[off] = soft_threshold(v[off], alpha)
    out = sp.csr_matrix((v, Zk.indices.copy(), Zk.indptr.copy()), shape=Zk.shape)
    out.eliminate_zeros()
    out.sort_indices()
    return out


@dataclasses.dataclass
class SparseResult:
    omega: sp.csr_matrix
    iterations: int
    trials: list
    taus: list
    F: list
    rel_change: float
    status: str


def solve_sparse(S, lam1, lam2, eps=1e-6, max_iter=1000, tau0=1.0, shrink=0.5, max_halvings=60,
                 block=512, threads=8, log=None) -> SparseResult:
    """Alg. 2 with a CSR iterate: the same steps and the same line-search rule as ``solve``."""
    p = S.shape[0]
    Omega = _csr_identity(p)
    rel = np.inf
    status = "max_iter"
    trials, taus, F = [], [], []
    for it in range(max_iter):
        Gk, Wsupp = gradient_candidates_cov(S, Omega, lam1, lam2, block, threads)   # steps 3, 5-6
        g = smooth_csr(Omega, _on_pattern(Wsupp, Omega), lam2)                      # step 7
        if it == 0:
            F.append(g + penalty_csr(Omega, lam1))
        Ok = _on_pattern(Omega, Gk)                # Omega on K (K holds supp(Omega))
        Gv = Gk.data
        tau, accepted = tau0, False
        for h in range(max_halvings + 1):
            Zk = sp.csr_matrix((Ok - tau * Gv, Gk.indices, Gk.indptr), shape=(p, p))
            Op = prox_csr(Zk, tau * lam1)                                           # step 9
            if np.all(Op.diagonal() > 0.0):
                wp = w_on_support(S, Op)                                            # step 10
                gp = smooth_csr(Op, wp, lam2)                                       # step 11
                Dk = _on_pattern(Op, Gk) - Ok
                # step 12: g(O+) <= g(O) - <O - O+, G> + ||O+ - O||^2 / (2 tau)
                rhs = g - float(np.sum(-Dk * Gv)) + float(np.sum(Dk * Dk)) / (2.0 * tau)
                if gp <= rhs:
                    accepted = True
                    break
            tau *= shrink
        if not accepted:
            status = "floor" if rel < 1e-8 else "ls_fail"
            break
        rel = float(np.sqrt(np.sum(Dk * Dk)) / np.sqrt(np.sum(Omega.data * Omega.data)))
        Omega = Op
        trials.append(h + 1)
        taus.append(tau)
        F.append(gp + penalty_csr(Omega, lam1))
        if log:
            log(f"it {it + 1}: tau {tau:g} trials {h + 1} nnz {Omega.nnz} rel {rel:.3e} F {F[-1]:.12g}")
        if rel < eps:
            status = "converged"
            break
    return SparseResult(Omega, len(trials), trials, taus, F, rel, status)


def kkt_residual_csr(Gk: sp.csr_matrix, omega: sp.csr_matrix, lam1) -> np.ndarray:
    """The smallest element of the subdifferential of F at Omega, on the entries of K, given G
    on K (``gradient_candidates_*``): G_ii on the diagonal, G_ij + lam1 sign(w_ij) on the
    off-diagonal support, max(|G_ij| - lam1, 0) elsewhere (0 outside K, where |G_ij| <= lam1).

    The smooth part is lam2-strongly convex on symmetric matrices, so an estimate with
    residual r lies within ||r||_F / lam2 of the minimiser in Frobenius norm."""
    rows = np.repeat(np.arange(Gk.shape[0]), np.diff(Gk.indptr))
    w = _on_pattern(omega, Gk)
    g = Gk.data
    diag = rows == Gk.indices
    on = (w != 0.0) & ~diag
    r = np.where(diag, g, np.where(on, g + lam1 * np.sign(w), np.maximum(np.abs(g) - lam1, 0.0)))
    return r


def gradient_candidates_obs(X, Y, omega: sp.csr_matrix, lam1, lam2, block=512):
    """Steps 4-6 of Alg. 3 for a CSR iterate: Z = Y X / n with Y = Omega X^T, and
    G = (Z + Z^T)/2 + lam2 Omega - diag(1/w_ii), formed in row blocks; G kept on K as in
    ``gradient_candidates_cov``.  Returns G on K as CSR."""
    n, p = X.shape
    om = omega
    dinv = 1.0 / om.diagonal()
    gi, gj, gv = [], [], []
    for r0, r1 in _blocks(p, block):
        ZI = (Y[r0:r1] @ X) / n                                     # rows r0..r1 of Z
        ZtI = ((Y @ np.ascontiguousarray(X[:, r0:r1])) / n).T       # rows r0..r1 of Z^T
        OI = om[r0:r1].toarray()
        GI = 0.5 * (ZtI + ZI) + lam2 * OI
        rr = np.arange(r1 - r0)
        GI[rr, r0 + rr] -= dinv[r0:r1]
        keep = (np.abs(GI) > lam1) | (OI != 0.0)
        keep[rr, r0 + rr] = True
        i, j = np.nonzero(keep)
        gi.append(i + r0)
        gj.append(j)
        gv.append(GI[i, j])
    Gk = sp.csr_matrix((np.concatenate(gv), (np.concatenate(gi), np.concatenate(gj))), shape=(p, p))
    Gk.sort_indices()
    return Gk


def solve_obs_sparse(X, lam1, lam2, eps=1e-6, max_iter=1000, tau0=1.0, shrink=0.5, max_halvings=60,
                     block=512, log=None) -> SparseResult:
    """Alg. 3 with a CSR iterate: Y = Omega X^T (steps 2, 10), Z = Y X / n (step 4),
    g from ||Y||_F^2 / n (steps 7, 11); the line-search rule of ``solve_obs``."""
    X = np.asarray(X, dtype=np.float64)
    n, p = X.shape
    Xt = np.ascontiguousarray(X.T)

    def g_of(Om, Y):
        d = Om.diagonal()
        if np.any(d <= 0.0):
            return np.inf
        return -float(np.sum(np.log(d))) + 0.5 * float(np.sum(Y * Y)) / n + \
            0.5 * lam2 * float(np.sum(Om.data * Om.data))

    Omega = _csr_identity(p)
    Y = np.asarray(Omega @ Xt)                                                  # step 2
    rel = np.inf
    status = "max_iter"
    trials, taus = [], []
    F = [g_of(Omega, Y) + penalty_csr(Omega, lam1)]
    for it in range(max_iter):
        Gk = gradient_candidates_obs(X, Y, Omega, lam1, lam2, block)            # steps 4-6
        g = g_of(Omega, Y)                                                      # step 7
        Ok = _on_pattern(Omega, Gk)
        Gv = Gk.data
        tau, accepted = tau0, False
        for h in range(max_halvings + 1):
            Zk = sp.csr_matrix((Ok - tau * Gv, Gk.indices, Gk.indptr), shape=(p, p))
            Op = prox_csr(Zk, tau * lam1)                                       # step 9
            if np.all(Op.diagonal() > 0.0):
                Yp = np.asarray(Op @ Xt)                                        # step 10
                gp = g_of(Op, Yp)                                               # step 11
                Dk = _on_pattern(Op, Gk) - Ok
                rhs = g - float(np.sum(-Dk * Gv)) + float(np.sum(Dk * Dk)) / (2.0 * tau)
                if gp <= rhs:
                    accepted = True
                    break
            tau *= shrink
        if not accepted:
            status = "floor" if rel < 1e-8 else "ls_fail"
            break
        rel = float(np.sqrt(np.sum(Dk * Dk)) / np.sqrt(np.sum(Omega.data * Omega.data)))
        Omega, Y = Op, Yp
        trials.append(h + 1)
        taus.append(tau)
        F.append(gp + penalty_csr(Omega, lam1))
        if log:
            log(f"it {it + 1}: tau {tau:g} trials {h + 1} nnz {Omega.nnz} rel {rel:.3e} F {F[-1]:.12g}")
        if rel < eps:
            status = "converged"
            break
    return SparseResult(Omega, len(trials), trials, taus, F, rel, status)


def objective_from_x(X, omega: sp.csr_matrix, lam1, lam2, chunk=4096) -> float:
    """F(Omega) = -sum log w_ii + ||X Omega||_F^2 / (2n) + lam2/2 ||Omega||_F^2 + lam1 ||Omega_X||_1
    in FP64 for a sparse symmetric Omega, with tr(Omega S Omega) = ||X Omega||_F^2 / n as in
    Alg. 3 step 7, summed over chunks of observations (rows of X)."""
    n = X.shape[0]
    om = sp.csr_matrix(omega, dtype=np.float64)
    d = om.diagonal()
    if np.any(d <= 0.0):
        return np.inf
    omt = om.T.tocsr()
    q = 0.0
    for r0 in range(0, n, chunk):
        Xc = np.asarray(X[r0:r0 + chunk], dtype=np.float64)
        Yc = np.asarray(omt @ Xc.T)              # (X Omega)^T for these rows
        q += float(np.sum(Yc * Yc))
    return -float(np.sum(np.log(d))) + 0.5 * q / n + 0.5 * lam2 * float(np.sum(om.data ** 2)) + \
        penalty_csr(om, lam1)


def heldout_loss_from_x(Xval, omega: sp.csr_matrix, chunk=4096) -> float:
    """L_val(Omega) = -sum log w_ii + ||X_val Omega||_F^2 / (2 n_val): the unpenalised held-out
    pseudolikelihood loss (heldout_loss) with tr(Omega S_val Omega) = ||X_val Omega||^2 / n_val,
    for a sparse Omega at large p."""
    return objective_from_x(Xval, omega, 0.0, 0.0, chunk)
