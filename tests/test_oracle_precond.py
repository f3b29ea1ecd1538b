"""Pins of the oracle's stronger preconditioners against facts outside them.

- the Chebyshev recurrence equals the closed form p_m(D^-1 A) D^-1 r built
  from an eigendecomposition (the definition of a polynomial preconditioner);
- degree 1 is Jacobi scaled by 1/theta;
- p_m is positive on the spectrum, so the preconditioner is SPD;
- the Gershgorin bound lies above the largest eigenvalue of D^-1 A;
- preconditioned CG reaches the dense solution within the classical
  iteration bound of its condition number, which falls as the degree grows;
  the incomplete-factorisation CG reaches it too.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import workloads as W
from oracle import pcg, precond, transient


def _system(n=5, contrast=(0.01, 100.0), seed=3, dt=1.0):
    p = W.random_box(n, n - 1, n + 1, seed=seed, flux={5: 1.0}, dt=dt, contrast=contrast,
                     dirichlet={0: 0.0})
    S = transient.build_system(p)
    return S.A_ff, S.pinv_f


def _spectrum(A, pinv):
    Dm = np.sqrt(pinv)
    As = (Dm[:, None] * A.toarray()) * Dm[None, :]  # D^-1/2 A D^-1/2, similar to D^-1 A
    lam, V = sla.eigh(As)
    return lam, V, Dm


@pytest.mark.parametrize("degree", [1, 2, 3, 5, 8])
def test_recurrence_equals_closed_form(degree):
    A, pinv = _system()
    lam, V, Dm = _spectrum(A, pinv)
    lo, hi = lam[0] * 0.5, lam[-1] * 1.1
    r = np.random.default_rng(degree).standard_normal(A.shape[0])
    z = precond.chebyshev_jacobi(A, pinv, r, degree, lo, hi)
    ref = Dm * (V @ (precond.chebyshev_polynomial(lam, degree, lo, hi) * (V.T @ (Dm * r))))
    assert np.linalg.norm(z - ref) <= 1e-11 * np.linalg.norm(ref)


def test_degree_one_is_scaled_jacobi_and_polynomial_positive():
    A, pinv = _system()
    lam, _, _ = _spectrum(A, pinv)
    lo, hi = lam[0], lam[-1]
    r = np.random.default_rng(0).standard_normal(A.shape[0])
    assert np.allclose(precond.chebyshev_jacobi(A, pinv, r, 1, lo, hi), pinv * r / (0.5 * (lo + hi)), rtol=1e-15)
    for m in (2, 4, 7):
        assert np.all(precond.chebyshev_polynomial(lam, m, lo * 0.1, hi * 1.01) > 0)


def test_gershgorin_bounds_the_spectrum():
    for seed in range(3):
        A, pinv = _system(seed=seed)
        lam, _, _ = _spectrum(A, pinv)
        assert precond.gershgorin_lam_max(A, pinv) >= lam[-1] * (1 - 1e-12)


def test_preconditioned_cg_reaches_dense_solution_and_degree_cuts_iterations():
    A, pinv = _system(n=7, dt=10.0)
    b = np.random.default_rng(1).standard_normal(A.shape[0])
    exact = pcg.solve_dense(A, b)
    lam, _, _ = _spectrum(A, pinv)
    its, kappas = [], []
    for m in (1, 2, 3, 4, 8):  # the interval of the true spectrum
        x, it = precond.pcg_precond(A, b, np.zeros_like(b),
                                    lambda r, m=m: precond.chebyshev_jacobi(A, pinv, r, m, lam[0], lam[-1]), 1e-12)
        assert np.linalg.norm(x - exact) <= 1e-9 * np.linalg.norm(exact)
        its.append(it)
        mu = precond.chebyshev_polynomial(lam, m, lam[0], lam[-1]) * lam  # spectrum of p(D^-1 A) D^-1 A
        kappas.append(mu.max() / mu.min())
        # the classical CG bound for this condition number (the b-norm criterion
        # differs from the A-norm one by at most sqrt(kappa))
        bound = 0.5 * np.sqrt(kappas[-1]) * np.log(2.0 * np.sqrt(kappas[-1]) / 1e-12) + 1
        assert it <= bound, (m, it, bound)
    assert all(a > b for a, b in zip(kappas, kappas[1:])), kappas  # the condition number falls with m
    assert its[-1] < its[0] / 2, its
    # an interval from the Gershgorin bound and a guessed ratio still converges (SPD preconditioner)
    hi = precond.gershgorin_lam_max(A, pinv)
    for m in (2, 4):
        x, it = precond.pcg_precond(A, b, np.zeros_like(b),
                                    lambda r, m=m: precond.chebyshev_jacobi(A, pinv, r, m, hi / 200.0, hi), 1e-12)
        assert np.linalg.norm(x - exact) <= 1e-9 * np.linalg.norm(exact)
    x, it = precond.pcg_precond(A, b, np.zeros_like(b), precond.ilu_preconditioner(A), 1e-12)
    assert np.linalg.norm(x - exact) <= 1e-9 * np.linalg.norm(exact) and it < its[0]


@pytest.mark.parametrize("seed,extent,dirichlet", [(0, (1.0, 1.0, 1.0), {0: 0.0}), (1, (2.0, 0.5, 1.0), {}),
                                                   (2, (1.0, 1.0, 3.0), {4: 1.0, 1: 0.0})])
def test_element_bound_lies_above_assembled_gershgorin_and_spectrum(seed, extent, dirichlet):
    p = W.random_box(4, 5, 3, seed=seed, extent=extent, dirichlet=dirichlet, contrast=(0.01, 100.0), dt=0.3)
    S = transient.build_system(p)
    lam, _, _ = _spectrum(S.A_ff, S.pinv_f)
    g = precond.gershgorin_lam_max(S.A_ff, S.pinv_f)
    e = precond.element_lam_max(p)
    assert lam[-1] <= g * (1 + 1e-12) and g <= e * (1 + 1e-12)


def test_element_bound_closed_forms():
    # Q1 mass rows on a box sum to h^3/8 against a diagonal of h^3/27: 27/8;
    # Q1 stiffness rows on a cube: diagonal h/3, absolute off-diagonal sum h/3: 2
    p = W.random_box(3, 3, 3, seed=0, extent=(0.6, 0.9, 1.2), dt=1.0, contrast=(1.0, 1.0))
    p.k[:] = 1e-300
    assert abs(precond.element_lam_max(p) - 27.0 / 8.0) < 1e-13
    p = W.random_box(3, 3, 3, seed=0, dt=1.0, contrast=(1.0, 1.0))
    p.rho_c[:] = 1e-300
    assert abs(precond.element_lam_max(p) - 2.0) < 1e-13


def test_chebyshev_pcg_degree_one_is_algorithm_one_and_degree_cuts_iterations():
    p = W.random_box(6, 5, 7, seed=4, dt=10.0, contrast=(0.01, 100.0), dirichlet={4: 1.0})
    S = transient.build_system(p)
    b = transient.step_rhs(p, S, p.u0, 1)
    x0 = p.u0[S.free]
    exact = pcg.solve_dense(S.A_ff, b)
    x1, it1, dj1, db1 = pcg.pcg(S.A_ff, b, x0, S.pinv_f, 1e-10, resid_period=7)
    lo, hi = precond.chebyshev_interval(precond.element_lam_max(p), 10.0)
    # degree 1 scales P^-1 by a constant, which leaves every CG iterate unchanged
    xc, itc, djc, dbc = precond.pcg_cheb(S.A_ff, b, x0, S.pinv_f, 1, lo, hi, 1e-10, resid_period=7)
    assert itc == it1 and dbc == db1
    assert np.linalg.norm(xc - x1) <= 1e-12 * np.linalg.norm(x1)
    its = [itc]
    for m in (2, 3, 4):
        x, it, dj, _ = precond.pcg_cheb(S.A_ff, b, x0, S.pinv_f, m, lo, hi, 1e-10, resid_period=7)
        assert dj <= 1e-20 * dbc
        assert np.linalg.norm(x - exact) <= 1e-8 * np.linalg.norm(exact)
        its.append(it)
    assert all(a > b for a, b in zip(its, its[1:])), its
