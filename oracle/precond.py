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

The interval's upper end comes from an element-by-element Gershgorin bound
(each node's absolute row sum is at most the sum over its elements of the
element rows' absolute sums, and the ratio of two sums of positive terms is at
most the largest term ratio), and the Chebyshev-preconditioned CG keeps the
stopping rule of Algorithm 1 (r^T P^-1 r against rtol^2 b^T P^-1 b, P the
Jacobi diagonal) so that the preconditioner changes only the search
directions.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import fem


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


def element_lam_max(p) -> float:
    """Upper bound of the spectrum of D^-1 A for A = M/dt + theta K of problem p:
    the largest, over elements e, of sum_b |K^e_ab| / K^e_aa with
    K^e = rho_c_e M_e / dt + theta k_e K_e (the same for every corner a of a
    box element)."""
    h = fem.spacing(p.nx, p.ny, p.nz, p.extent)
    if getattr(p, "element", "q1") == "p1":
        from . import p1
        Me, Ke = p1.box_matrices(*h)  # rows differ by corner: the maximum runs over them too
    else:
        Me, Ke = fem.element_matrices(*h)
    best = 0.0
    for rc, k in zip(np.asarray(p.rho_c, dtype=np.float64), np.asarray(p.k, dtype=np.float64)):
        E = rc / p.dt * Me + p.theta * k * Ke
        best = max(best, float(np.max(np.abs(E).sum(axis=1) / np.diag(E))))
    return best


def chebyshev_interval(lam_hi: float, ratio: float):
    """[lam_hi / ratio, lam_hi]: the interval the Chebyshev preconditioner targets."""
    return lam_hi / ratio, lam_hi


def pcg_cheb(A, b: np.ndarray, x0: np.ndarray, pinv: np.ndarray, degree: int, lam_lo: float, lam_hi: float,
             rtol: float, max_iter: int = 20000, resid_period: int = 50):
    """Algorithm 1 with the Jacobi step s = P^-1 r replaced by the Chebyshev
    step z = p_m(D^-1 A) D^-1 r in the direction update and in the scalar
    r^T z that forms alpha and beta; the stopping test stays r^T P^-1 r <=
    rtol^2 b^T P^-1 b, checked before every iteration, and the true residual
    replaces the recursive one every resid_period iterations as in the
    algorithm. Returns (x, iterations, r^T P^-1 r at exit, b^T P^-1 b)."""
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A @ x
    delta_b = float(b @ (pinv * b))
    threshold = rtol * rtol * delta_b
    delta_j = float(r @ (pinv * r))
    i = 0
    gamma = d = None
    while i < max_iter and delta_j > threshold:
        z = chebyshev_jacobi(A, pinv, r, degree, lam_lo, lam_hi)
        gamma_new = float(r @ z)
        d = z if d is None else z + (gamma_new / gamma) * d
        gamma = gamma_new
        q = A @ d
        alpha = gamma / float(d @ q)
        x = x + alpha * d
        if i > 0 and i % resid_period == 0:
            r = b - A @ x
        else:
            r = r - alpha * q
        delta_j = float(r @ (pinv * r))
        i += 1
    return x, i, delta_j, delta_b


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
