"""Plant plausible mistakes in the oracle's six-tetrahedra discretisation and
Chebyshev preconditioner (on the CPU) and show that their pins catch each one."""
from itertools import permutations

import numpy as np
import pytest

import test_oracle_p1 as TP
import test_oracle_precond as TC
from oracle import p1, precond

_orig_tet = p1.tet_matrices
_orig_face = p1.face_load_elements
_orig_bt = p1.boundary_triangles
_orig_cheb = precond.chebyshev_jacobi
_orig_bound = precond.element_lam_max


def _tet_mass_24(X):
    M, K, V = _orig_tet(X)
    return M * 20.0 / 24.0, K, V


def _tet_mass_lumped(X):
    M, K, V = _orig_tet(X)
    return np.eye(4) * V / 4.0, K, V


def _tet_grad_transposed(X):
    T = np.hstack([np.ones((4, 1)), X])
    V = abs(np.linalg.det(T)) / 6.0
    g = np.linalg.inv(T)[:, 1:]  # rows of the inverse taken as gradients: a transposition
    M = V * (np.ones((4, 4)) + np.eye(4)) / 20.0
    return M, V * g @ g.T, V


def _face_quarter(nx, ny, nz, extent, face, q_elem):
    return _orig_face(nx, ny, nz, extent, face, q_elem) * 0.75  # A/4 instead of A/3 per vertex


def _bt_quad_transposed(nx, ny, nz, extent):
    tri, area, face, quad = _orig_bt(nx, ny, nz, extent)
    counts = {0: (ny, nz), 1: (nx, nz), 2: (nx, ny)}
    q = quad.copy()
    for f in range(6):
        na, nb = counts[f // 2]
        sel = face == f
        a, b = quad[sel] % na, quad[sel] // na
        q[sel] = (b + nb * a) % (na * nb)  # upper index fastest
    return tri, area, face, q


def _cheb_residual_sign(A, pinv, r, degree, lam_lo, lam_hi):
    return _orig_cheb(-A, pinv, r, degree, lam_lo, lam_hi) if degree > 1 else _orig_cheb(A, pinv, r, degree, lam_lo, lam_hi)


def _cheb_one_step_short(A, pinv, r, degree, lam_lo, lam_hi):
    return _orig_cheb(A, pinv, r, max(1, degree - 1), lam_lo, lam_hi)


def _bound_no_abs(p):
    from oracle import fem
    h = fem.spacing(p.nx, p.ny, p.nz, p.extent)
    Me, Ke = (p1.box_matrices(*h) if getattr(p, "element", "q1") == "p1" else fem.element_matrices(*h))
    best = 0.0
    for rc, k in zip(p.rho_c, p.k):
        E = rc / p.dt * Me + p.theta * k * Ke
        best = max(best, float(np.max(E.sum(axis=1) / np.diag(E))))  # signed row sums
    return best


PINS = [
    TP.test_unit_cube_matrices_match_hand_worked_fixture,
    TP.test_box_matrices_scale_and_keep_the_sparsity_on_any_box,
    TP.test_split_tiles_the_box_conformingly,
    TP.test_patch_tests_of_the_assembled_matrices,
    TP.test_assembled_stiffness_is_the_seven_point_laplacian,
    lambda: TP.test_boundary_loads(3),
    TP.test_single_loaded_quad_shares,
    TP.test_transient_energy_balance_and_spectral_bound,
    lambda: TC.test_recurrence_equals_closed_form(3),
    TC.test_gershgorin_bounds_the_spectrum,
    lambda: TC.test_element_bound_lies_above_assembled_gershgorin_and_spectrum(0, (1.0, 1.0, 1.0), {0: 0.0}),
    TC.test_element_bound_closed_forms,
]

MUTANTS = {
    "tet_mass_1_24": (p1, "tet_matrices", _tet_mass_24),
    "tet_mass_lumped": (p1, "tet_matrices", _tet_mass_lumped),
    "tet_gradient_transposed": (p1, "tet_matrices", _tet_grad_transposed),
    "split_reversed_paths": (p1, "TETS", [(0, p1.AXIS_BIT[c], p1.AXIS_BIT[a] | p1.AXIS_BIT[c], 7)
                                          for a, _, c in permutations(range(3))][:3] * 2),
    "boundary_share_quarter": (p1, "face_load_elements", _face_quarter),
    "boundary_quad_transposed": (p1, "boundary_triangles", _bt_quad_transposed),
    "chebyshev_residual_sign": (precond, "chebyshev_jacobi", _cheb_residual_sign),
    "chebyshev_one_pass_short": (precond, "chebyshev_jacobi", _cheb_one_step_short),
    "bound_without_abs": (precond, "element_lam_max", _bound_no_abs),
}


def _all_pins_pass():
    for pin in PINS:
        try:
            pin()
        except AssertionError:
            return False
    return True


def test_correct_oracle_passes_every_pin():
    assert _all_pins_pass()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, monkeypatch):
    mod, attr, fn = MUTANTS[name]
    monkeypatch.setattr(mod, attr, fn)
    assert not _all_pins_pass(), f"mutant {name} passed every pin"
