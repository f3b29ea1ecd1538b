"""Plant plausible mistakes in the oracle (on the CPU) and show a pin catches each.

A pin set that passes the correct oracle and fails every mutant below is
evidence that the pins constrain the oracle's arithmetic, not just its shape.
"""
import numpy as np
import pytest

import pins
from oracle import fem, pcg, transient

_orig_elem = fem.element_matrices
_orig_node_id = fem.node_id
_orig_build = transient.build_system
_orig_face_load = fem.face_load
_orig_pcg = pcg.pcg


def _mut_drop_kz(hx, hy, hz):
    Me, Ke = _orig_elem(hx, hy, hz)
    # remove the z-gradient term (what a dropped term in grad.grad looks like)
    m1 = lambda s: s / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
    k1 = lambda s: 1.0 / s * np.array([[1.0, -1.0], [-1.0, 1.0]])
    return Me, Ke - np.kron(k1(hz), np.kron(m1(hy), m1(hx)))


def _mut_swap_hx_hy(hx, hy, hz):
    return _orig_elem(hy, hx, hz)


def _mut_lumped_mass(hx, hy, hz):
    Me, Ke = _orig_elem(hx, hy, hz)
    return np.diag(Me.sum(axis=1)), Ke


def _mut_transposed_node_id(nx, ny, i, j, k):
    return j + (ny + 1) * (i + (nx + 1) * k) if nx == ny else _orig_node_id(nx, ny, j, i, k)


def _mut_L_sign(p):
    S = _orig_build(p)
    S.L = (S.M / p.dt + (1.0 - p.theta) * S.K).tocsr()
    return S


def _mut_no_lift(p):
    S = _orig_build(p)
    S.A_fD = S.A_fD * 0.0
    return S


def _mut_face_load_no_quarter(nx, ny, nz, extent, face, q):
    return 4.0 * _orig_face_load(nx, ny, nz, extent, face, q)


def _mut_pcg_stale_delta(A, b, x0, pinv, rtol, max_iter=20000, resid_period=50):
    x = np.array(x0, dtype=np.float64, copy=True)
    r = b - A @ x
    d = pinv * r
    delta_new = float(r @ d)
    delta0 = delta_new
    thr = rtol * rtol * float(b @ (pinv * b))
    i = 0
    while i < max_iter and delta_new > thr:
        q = A @ d
        alpha = delta_new / float(d @ q)
        x = x + alpha * d
        r = r - alpha * q
        s = pinv * r
        delta_new = float(r @ s)
        d = s + (delta_new / delta0) * d  # delta_old never updated
        i += 1
    return x, i, delta_new, thr


def _mut_pcg_sign(A, b, x0, pinv, rtol, max_iter=20000, resid_period=50):
    x, it, dn, db = _orig_pcg(A, -b, x0, pinv, rtol, max_iter, resid_period)
    return -x if it % 2 else x, it, dn, db


ALL_PINS = {
    "golden": lambda: pins.check_element_golden() < 1e-15,
    "box": lambda: pins.check_element_box_closed_form() < 1e-14,
    "mode_dirichlet": lambda: pins.check_eigenmode("dirichlet") < 1e-12,
    "mode_mixed": lambda: pins.check_eigenmode("mixed") < 1e-12,
    "mode_neumann": lambda: pins.check_eigenmode("neumann") < 1e-12,
    "energy": lambda: pins.check_energy_balance() < 1e-12,
    "steady": lambda: pins.check_steady_dirichlet() < 1e-9,
    "face": lambda: _safe(pins.check_face_load) < 1e-14,
    "pcg_dense": lambda: pins.check_pcg_vs_dense() < 1e-11,
    "decay": lambda: pins.check_continuum_decay() < 5e-3,
    "cg_termination": lambda: pins.check_pcg_finite_termination() <= 1.0,
}


def _safe(fn):
    try:
        return fn()
    except AssertionError:
        return np.inf


MUTANTS = {
    "drop_kz": (fem, "element_matrices", _mut_drop_kz),
    "swap_hx_hy": (fem, "element_matrices", _mut_swap_hx_hy),
    "lumped_mass": (fem, "element_matrices", _mut_lumped_mass),
    "transposed_node_id": (fem, "node_id", _mut_transposed_node_id),
    "L_sign": (transient, "build_system", _mut_L_sign),
    "no_dirichlet_lift": (transient, "build_system", _mut_no_lift),
    "face_load_x4": (fem, "face_load", _mut_face_load_no_quarter),
    "pcg_stale_delta": (pcg, "pcg", _mut_pcg_stale_delta),
    "pcg_sign": (pcg, "pcg", _mut_pcg_sign),
}


def test_correct_oracle_passes_every_pin():
    failed = [k for k, f in ALL_PINS.items() if not f()]
    assert failed == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, monkeypatch):
    mod, attr, fn = MUTANTS[name]
    monkeypatch.setattr(mod, attr, fn)
    caught = []
    for pin, check in ALL_PINS.items():
        try:
            ok = check()
        except Exception:
            ok = False
        if not ok:
            caught.append(pin)
    assert caught, f"mutant {name} passed every pin"
