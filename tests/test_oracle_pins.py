"""Pins of the CPU oracle against facts the paper's equations fix (no GPU).

Each test ties an oracle function to something other than itself: exact
textbook element matrices, symbolic integration, exact discrete eigenmodes of
the theta-scheme, conservation of energy, the linear patch test, dense direct
solves, and the continuum decay rate exp(-3 pi^2 kappa t).
"""
import numpy as np
import pytest

import pins
import workloads as W
from oracle import fem, pcg, transient


def test_element_matrices_match_golden_unit_cube():
    assert pins.check_element_golden() < 1e-15


def test_element_matrices_match_kronecker_closed_form_on_box():
    assert pins.check_element_box_closed_form() < 1e-14


def test_element_matrices_match_symbolic_integration():
    sympy = pytest.importorskip("sympy")
    x, y, z = sympy.symbols("x y z")
    hx, hy, hz = sympy.Rational(1, 2), sympy.Rational(3, 1), sympy.Rational(2, 5)
    phis = []
    for c in range(8):
        cx, cy, cz = c & 1, (c >> 1) & 1, (c >> 2) & 1
        fx = x / hx if cx else 1 - x / hx
        fy = y / hy if cy else 1 - y / hy
        fz = z / hz if cz else 1 - z / hz
        phis.append(fx * fy * fz)
    Me, Ke = fem.element_matrices(float(hx), float(hy), float(hz))
    for a in range(8):
        for b in range(a, 8):
            m = sympy.integrate(phis[a] * phis[b], (x, 0, hx), (y, 0, hy), (z, 0, hz))
            g = sum(sympy.diff(phis[a], v) * sympy.diff(phis[b], v) for v in (x, y, z))
            kk = sympy.integrate(g, (x, 0, hx), (y, 0, hy), (z, 0, hz))
            assert abs(Me[a, b] - float(m)) < 1e-14
            assert abs(Ke[a, b] - float(kk)) < 1e-13


def test_element_matrix_invariants():
    Me, Ke = fem.element_matrices(0.3, 0.5, 0.2)
    assert abs(Me.sum() - 0.3 * 0.5 * 0.2) < 1e-15
    assert np.abs(Ke @ np.ones(8)).max() < 1e-13
    assert np.allclose(Me, Me.T) and np.allclose(Ke, Ke.T)
    ev = np.linalg.eigvalsh(Ke)
    assert abs(ev[0]) < 1e-12 and ev[1] > 1e-3  # one-dimensional null space


def test_assembly_totals_and_symmetry():
    p = W.random_box(4, 5, 3, seed=1, extent=(2.0, 1.0, 0.5))
    M = fem.assemble(p.nx, p.ny, p.nz, p.extent, p.rho_c, "M")
    K = fem.assemble(p.nx, p.ny, p.nz, p.extent, p.k, "K")
    vol = np.prod(p.extent) / p.n_elems
    one = np.ones(p.n_nodes)
    assert abs(one @ (M @ one) - p.rho_c.sum() * vol) < 1e-12
    assert np.abs(K @ one).max() < 1e-12
    assert abs(M - M.T).max() < 1e-15 and abs(K - K.T).max() < 1e-14
    assert M.nnz <= 27 * p.n_nodes


def test_patch_test_linear_field():
    assert pins.check_patch_linear() < 1e-12


def test_face_load_totals_and_shares():
    assert pins.check_face_load() < 1e-14


@pytest.mark.parametrize("kind", ["dirichlet", "mixed", "neumann"])
def test_exact_discrete_eigenmode(kind):
    assert pins.check_eigenmode(kind) < 1e-12


@pytest.mark.parametrize("kind", ["dirichlet", "mixed", "neumann"])
def test_exact_discrete_eigenmode_with_pcg(kind):
    assert pins.check_eigenmode(kind, solver="pcg") < 1e-11


def test_energy_balance():
    assert pins.check_energy_balance() < 1e-12


def test_steady_state_with_dirichlet_lift():
    assert pins.check_steady_dirichlet() < 1e-9


def test_pcg_matches_dense_cholesky():
    assert pins.check_pcg_vs_dense() < 1e-11


def test_direct_matches_dense_cholesky():
    p = W.random_box(3, 3, 4, seed=5, dirichlet={1: 2.0}, flux={4: 1.0})
    S = transient.build_system(p)
    b = transient.step_rhs(p, S, p.u0, 1)
    x1 = pcg.solve_direct(S.A_ff, b)
    x2 = pcg.solve_dense(S.A_ff, b)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x2) < 1e-13


def test_continuum_decay_rate():
    # O(h^2 + dt^2) agreement with the PDE's exact decay exp(-3 pi^2 t)
    assert pins.check_continuum_decay() < 5e-3


def test_pcg_finite_termination_and_iteration_count():
    # CG on an n x n SPD system converges in at most n iterations (exact
    # arithmetic); allow a few extra for rounding.
    p = W.random_box(2, 2, 1, seed=9, theta=1.0, dt=0.1)
    S = transient.build_system(p)
    b = transient.step_rhs(p, S, p.u0, 1)
    x, it, delta, delta_b = pcg.pcg(S.A_ff, b, np.zeros_like(b), S.pinv_f, 1e-13, 1000)
    assert it <= S.A_ff.shape[0] + 3
    assert delta <= 1e-26 * delta_b
    assert pins.check_pcg_finite_termination() <= 1.0


def test_pcg_zero_rhs_converges_immediately():
    p = W.random_box(2, 2, 2, seed=9)
    S = transient.build_system(p)
    b = np.zeros(S.A_ff.shape[0])
    x, it, _, _ = pcg.pcg(S.A_ff, b, np.zeros_like(b), S.pinv_f, 1e-10)
    assert it == 0 and not x.any()


def test_apply_rows_matches_csr():
    p = W.random_box(3, 4, 2, seed=4, dirichlet={2: 1.0, 5: 0.0})
    S = transient.build_system(p)
    x = np.random.default_rng(0).standard_normal(p.n_nodes)
    x_free = np.zeros_like(x)
    x_free[S.free] = x[S.free]
    sa, sb = 1.0 / p.dt, p.theta
    ref = S.A @ x_free
    ref[S.dir_ids] = x[S.dir_ids]
    rows = np.arange(p.n_nodes)
    got = fem.apply_rows(p, x, rows, sa, sb)
    assert np.abs(got - ref).max() < 1e-12 * np.abs(ref).max()


def test_all_dirichlet_tiny_mesh_has_no_free_rows():
    p = W.random_box(1, 1, 1, seed=2, dirichlet={f: 0.25 * f for f in range(6)})
    res = transient.run(p, solver="pcg")
    ids, vals = fem.dirichlet_nodes(p)
    assert ids.size == 8
    assert np.allclose(res.u[1][ids], vals)
    # lowest face id wins on shared corners: node 0 lies on faces 0, 2, 4 -> face 0
    assert vals[0] == 0.0
