"""Stronger preconditioners for the oracle's CG (test infrastructure only).

The paper preconditions CG with the Jacobi diagonal (§3.3) and compares with
an incomplete-Cholesky CPU solver (§5.2). Two additions follow textbook
definitions:

* Chebyshev-Jacobi: z = p_m(D^-1 A) D^-1 r, the result of m steps of the
  Chebyshev semi-iteration for A z = r preconditioned by D, started from
  z = 0, for an assumed spectrum [lam_lo, lam_hi] of D^-1 A. Its error
  polynomial is R_m(lam) = T_m((theta - lam)/delta) / T_m(theta/delta)
  (theta, delta the interval's centre and half-width), so
  p_m(lam) = (1 - R_m(lam)) / lam, positive on (0, lam_hi]: for an interval
  that contains the spectrum the preconditioner is SPD.
* Incomplete factorisation with a drop tolerance (SuperLU's ILU, the
  nonsymmetric counterpart of incomplete Cholesky) as the CPU baseline's
  preconditioner.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def chebyshev_jacobi(A, pinv: np.ndarray, r: np.ndarray, degree: int, lam_lo: float, lam_hi: float):
    """z = p_m(D^-1 A) D^-1 r by the three-term Chebyshev recurrence
    (m = degree >= 1; m - 1 products with A)."""
    theta = 0.5 * (lam_hi + lam_lo)
    delta = 0.5 * (lam_hi - lam_lo)
    sigma = theta / delta
    rho = 1.0 / sigma
    z = np.zeros_like(r)
    res = np.array(r, dtype=np.float64, copy=True)
    d = pinv * res / theta
    for k in range(degree):
        z = z + d
        if k == degree - 1:
            break
        res = res - A @ d
        rho_next = 1.0 / (2.0 * sigma - rho)
        d = rho_next * rho * d + (2.0 * rho_next / delta) * (pinv * res)
        rho = rho_next
    return z


def chebyshev_polynomial(lam: np.ndarray, degree: int, lam_lo: float, lam_hi: float) -> np.ndarray:
    """p_m(lam) = (1 - T_m((theta - lam)/delta) / T_m(theta/delta)) / lam."""
    theta = 0.5 * (lam_hi + lam_lo)
    delta = 0.5 * (lam_hi - lam_lo)
    T = np.polynomial.chebyshev.Chebyshev.basis(degree)
    return (1.0 - T((theta - lam) / delta) / T(theta / delta)) / lam


def gershgorin_lam_max(A, pinv: np.ndarray) -> float:
    """Upper bound of the spectrum of D^-1 A: max_i sum_j |A_ij| / A_ii."""
    absA = abs(A).tocsr()
    return float(np.max(np.asarray(absA.sum(axis=1)).ravel() * pinv))


def pcg_precond(A, b: np.ndarray, x0: np.ndarray, precond, rtol: float, max_iter: int = 20000):
    """CG with an SPD preconditioner z = precond(r); stops when
    r^T z <= rtol^2 * b^T precond(b). Returns (x, iterations)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A @ x
    z = precond(r)
    delta = float(r @ z)
    threshold = rtol * rtol * float(b @ precond(b))
    d = z.copy()
    i = 0
    while i < max_iter and delta > threshold:
        q = A @ d
        alpha = delta / float(d @ q)
        x = x + alpha * d
        r = r - alpha * q
        z = precond(r)
        delta_new = float(r @ z)
        d = z + (delta_new / delta) * d
        delta = delta_new
        i += 1
    return x, i


def ilu_preconditioner(A, drop_tol: float = 1e-3, fill_factor: float = 10.0):
    """r -> (LU)^-1 r for SuperLU's incomplete factorisation of A."""
    ilu = spla.spilu(A.tocsc(), drop_tol=drop_tol, fill_factor=fill_factor)
    return ilu.solve
