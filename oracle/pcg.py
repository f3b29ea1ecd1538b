"""Linear solvers of the oracle (test infrastructure only).

``pcg`` follows Algorithm 1 (§3.3): Jacobi-preconditioned conjugate gradients
with the true residual recomputed periodically. Readings where the listing is
silent or inconsistent:
  * stop when r^T P^-1 r <= rtol^2 * b^T P^-1 b (the text asks for a relative
    tolerance; the listing compares delta to an absolute tol);
  * delta_old <- delta_new every iteration (the listing omits it);
  * the true residual is recomputed when i > 0 and i % period == 0.
``solve_direct`` (sparse LU) and ``solve_dense`` (dense Cholesky) solve the
same SPD systems exactly up to rounding; they are the plain definition of the
step solution that PCG approximates.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla


def pcg(A, b: np.ndarray, x0: np.ndarray, pinv: np.ndarray, rtol: float,
        max_iter: int = 20000, resid_period: int = 50, record: list = None):
    """Algorithm 1. Returns (x, iterations, delta_final, delta_b).

    With a list as `record`, each iteration appends its (alpha, beta), the
    coefficients lanczos_extremes turns into a condition estimate."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A @ x
    d = pinv * r
    delta_new = float(r @ d)
    delta_b = float(b @ (pinv * b))
    threshold = rtol * rtol * delta_b
    i = 0
    while i < max_iter and delta_new > threshold:
        q = A @ d
        alpha = delta_new / float(d @ q)
        x = x + alpha * d
        if i > 0 and i % resid_period == 0:
            r = b - A @ x
        else:
            r = r - alpha * q
        s = pinv * r
        delta_old = delta_new
        delta_new = float(r @ s)
        beta = delta_new / delta_old
        d = s + beta * d
        if record is not None:
            record.append((alpha, beta))
        i += 1
    return x, i, delta_new, delta_b


def lanczos_extremes(coeffs):
    """Smallest and largest eigenvalue of the Lanczos tridiagonal matrix that a
    preconditioned CG run builds implicitly (the CG-Lanczos relation, e.g. Saad,
    Iterative Methods for Sparse Linear Systems, 2nd ed., §6.7.3): with the
    run's (alpha_j, beta_j),
        T_jj = 1/alpha_j + beta_{j-1}/alpha_{j-1},   T_{j,j+1} = sqrt(beta_j)/alpha_j.
    Its eigenvalues (Ritz values) approach the extreme eigenvalues of P^-1 A
    from inside, so lam_max / lam_min estimates kappa(P^-1 A) from below."""
    m = len(coeffs)
    if m == 0:
        return float("nan"), float("nan")
    al = np.array([c[0] for c in coeffs])
    be = np.array([c[1] for c in coeffs])
    diag = 1.0 / al
    diag[1:] += be[:-1] / al[:-1]
    off = np.sqrt(be[:-1]) / al[:-1]
    ev = sla.eigh_tridiagonal(diag, off, eigvals_only=True)
    return float(ev[0]), float(ev[-1])


def solve_direct(A, b: np.ndarray) -> np.ndarray:
    """Sparse LU solve (SuperLU) of A x = b."""
    if A.shape[0] == 0:
        return np.zeros(0)
    return spla.splu(A.tocsc()).solve(b)


def solve_dense(A, b: np.ndarray) -> np.ndarray:
    """Dense Cholesky solve of the SPD system A x = b (tiny meshes only)."""
    if A.shape[0] == 0:
        return np.zeros(0)
    Ad = A.toarray() if hasattr(A, "toarray") else np.asarray(A)
    return sla.cho_solve(sla.cho_factor(Ad), b)
