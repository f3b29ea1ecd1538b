"""Plant plausible mistakes in the oracle's inverse-problem pieces (on the
CPU) and show that the pins of test_oracle_inverse catch each one."""
import math

import numpy as np
import pytest

import test_oracle_inverse as T
from oracle import fem, inverse

_orig_face = fem.face_load_elements
_orig_corr = inverse.corrosion_coefficients
_orig_loglik = inverse.loglik
_orig_forward = inverse.forward
_orig_mh = inverse.mh_chain


def _mut_face_transposed(nx, ny, nz, extent, face, q_elem):
    axis = face // 2
    dims = [d for d in range(3) if d != axis]
    counts = (nx, ny, nz)
    na, nb = counts[dims[0]], counts[dims[1]]
    q = np.asarray(q_elem).reshape(nb, na).T.ravel()[: na * nb]  # upper index fastest
    return _orig_face(nx, ny, nz, extent, face, q)


def _mut_face_one_corner(nx, ny, nz, extent, face, q_elem):
    F = _orig_face(nx, ny, nz, extent, face, q_elem)
    ids = fem.face_nodes(nx, ny, nz, face)
    G = np.zeros_like(F)
    G[ids] = np.roll(F[ids], 1)  # loads land on a neighbouring node
    return G


def _mut_corr_sign(nx, ny, nz, origin, extent, geom, depth):
    flipped = dict(geom, rho_c_corr=geom["rho_c_sound"], k_corr=geom["k_sound"],
                   rho_c_sound=geom["rho_c_corr"], k_sound=geom["k_corr"])
    return _orig_corr(nx, ny, nz, origin, extent, flipped, depth)


def _mut_corr_front(nx, ny, nz, origin, extent, geom, depth):
    rc, k = _orig_corr(nx, ny, nz, origin, extent, geom, depth)  # measured from the front face
    return rc.reshape(nz, ny, nx)[:, ::-1, :].ravel(), k.reshape(nz, ny, nx)[:, ::-1, :].ravel()


def _mut_loglik_no_half(u, d, sigma):
    return 2.0 * _orig_loglik(u, d, sigma)


def _mut_forward_no_flux(plate, depth):
    saved = plate.flux_q
    plate.flux_q = np.zeros_like(saved)
    try:
        return _orig_forward(plate, depth)
    finally:
        plate.flux_q = saved


def _mut_forward_sound_only(plate, depth):
    return _orig_forward(plate, 0.0)


def _mut_mh_reversed(state, state_ll, normals, uniforms, step, depth_max, loglik_fn):
    return _orig_mh(state, -np.asarray(state_ll), normals, uniforms, step, depth_max,
                    lambda d: -np.asarray(loglik_fn(d)))


def _mut_mh_no_prior(state, state_ll, normals, uniforms, step, depth_max, loglik_fn):
    return _orig_mh(state, state_ll, normals, uniforms, step, math.inf, loglik_fn)


PINS = [
    lambda: T.test_uniform_element_flux_equals_uniform_face_load(2),
    T.test_single_loaded_quad_gives_quarter_area_to_each_corner,
    T.test_corrosion_depth_zero_is_sound_and_full_cover_is_corroded,
    T.test_corrosion_hand_worked_case,
    T.test_loglik_closed_form,
    T.test_mh_deterministic_cases,
    T.test_forward_energy_balance,
    T.test_forward_uses_the_corrosion_coefficients,
]

MUTANTS = {
    "face_transposed": (fem, "face_load_elements", _mut_face_transposed),
    "face_one_corner": (fem, "face_load_elements", _mut_face_one_corner),
    "corrosion_materials_swapped": (inverse, "corrosion_coefficients", _mut_corr_sign),
    "corrosion_from_front": (inverse, "corrosion_coefficients", _mut_corr_front),
    "loglik_no_half": (inverse, "loglik", _mut_loglik_no_half),
    "forward_no_flux": (inverse, "forward", _mut_forward_no_flux),
    "forward_ignores_depth": (inverse, "forward", _mut_forward_sound_only),
    "mh_reversed_ratio": (inverse, "mh_chain", _mut_mh_reversed),
    "mh_no_prior": (inverse, "mh_chain", _mut_mh_no_prior),
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
