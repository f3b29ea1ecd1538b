"""Pins of the oracle's inverse-problem pieces (§5.3) against facts outside it.

- per-element face loads: a uniform density reproduces the pinned uniform
  face load; one loaded quad gives each of its four corners q*area/4 (the
  integral of a bilinear corner function); the total is sum(q * area);
- corrosion coefficients: depth 0 is all sound, an all-covering profile is
  all corroded, and a hand-worked small mesh;
- log-likelihood: the closed form on a tiny case;
- Metropolis-Hastings: deterministic accept/reject cases, and the sample
  moments of long chains on a Gaussian target whose moments are known;
- forward model: energy balance (1^T M U^n = 1^T M U^0 + n dt 1^T F for flux
  on every step and no Dirichlet face, whatever the coefficients), and no
  dependence on the depth when both materials are the same.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import fem, inverse


@pytest.mark.parametrize("face", range(6))
def test_uniform_element_flux_equals_uniform_face_load(face):
    nx, ny, nz, ext = 3, 4, 5, (1.5, 0.7, 2.0)
    na = (ny, nx, nx)[face // 2]
    nb = (nz, nz, ny)[face // 2]
    got = fem.face_load_elements(nx, ny, nz, ext, face, np.full(na * nb, 0.37))
    ref = fem.face_load(nx, ny, nz, ext, face, 0.37)
    assert np.allclose(got, ref, rtol=1e-14, atol=0.0)


def test_single_loaded_quad_gives_quarter_area_to_each_corner():
    nx, ny, nz, ext = 4, 3, 5, (2.0, 3.0, 1.0)
    hx, hy, hz = 0.5, 1.0, 0.2
    q = np.zeros(nx * nz)
    q[2 + nx * 3] = 1.7  # face y=0, quad (i=2, k=3)
    F = fem.face_load_elements(nx, ny, nz, ext, 2, q)
    corners = [fem.node_id(nx, ny, i, 0, k) for i in (2, 3) for k in (3, 4)]
    assert np.allclose(F[corners], 1.7 * hx * hz / 4.0, rtol=1e-14)
    assert np.count_nonzero(F) == 4
    rng = np.random.default_rng(0)
    q = rng.uniform(0, 2, nx * ny)
    F = fem.face_load_elements(nx, ny, nz, ext, 5, q)
    assert math.isclose(F.sum(), q.sum() * hx * hy, rel_tol=1e-13)


GEOM = {"z0": 1.0, "half_width": 0.75, "rho_c_sound": 2.0, "k_sound": 3.0, "rho_c_corr": 0.5, "k_corr": 0.25}


def test_corrosion_depth_zero_is_sound_and_full_cover_is_corroded():
    rc, k = inverse.corrosion_coefficients(3, 4, 5, (0, 0, 0), (1.0, 1.0, 2.0), GEOM, 0.0)
    assert np.all(rc == 2.0) and np.all(k == 3.0)
    g = dict(GEOM, half_width=1e9)
    rc, k = inverse.corrosion_coefficients(3, 4, 5, (0, 0, 0), (1.0, 1.0, 2.0), g, 2.0)
    assert np.all(rc == 0.5) and np.all(k == 0.25)


def test_corrosion_hand_worked_case():
    # 1 x 4 x 4 elements on [0,1]x[0,4]x[0,4] (h = 1): z centroids 0.5..3.5,
    # y centroids 0.5..3.5, rear face y = 4. z0 = 2, w = 2, depth 2.5:
    #   z_c = 0.5: t = -0.75, d = 2.5*(1-0.5625) = 1.09375 -> y_c = 3.5 (dist 0.5)
    #   z_c = 1.5: t = -0.25, d = 2.34375 -> y_c = 3.5, 2.5 (dist 0.5, 1.5)
    #   z_c = 2.5, 3.5: mirror images.
    g = {"z0": 2.0, "half_width": 2.0, "rho_c_sound": 1.0, "k_sound": 1.0, "rho_c_corr": 7.0, "k_corr": 9.0}
    rc, _ = inverse.corrosion_coefficients(1, 4, 4, (0, 0, 0), (1.0, 4.0, 4.0), g, 2.5)
    got = (rc.reshape(4, 4) == 7.0)  # [k, j]
    want = np.array([[0, 0, 0, 1], [0, 0, 1, 1], [0, 0, 1, 1], [0, 0, 0, 1]], dtype=bool)
    assert np.array_equal(got, want)


def test_loglik_closed_form():
    assert inverse.loglik([1.0, 2.0], [0.5, 2.5], 0.5) == -0.5 * (1.0 + 1.0)


def test_mh_deterministic_cases():
    normals = np.array([[0.5, 3.0]])
    uniforms = np.array([[0.999, 0.5]])
    flat = lambda d: np.zeros(len(d))
    dtr, ltr, acc = inverse.mh_chain([1.0, 1.0], [0.0, 0.0], normals, uniforms, 1.0, 2.0, flat)
    # chain 0: proposal 1.5 inside, log(0.999) < 0: accepted; chain 1: 4.0 outside: rejected
    assert acc.tolist() == [[True, False]] and dtr.tolist() == [[1.5, 1.0]]
    worse = lambda d: -10.0 * np.ones(len(d))
    dtr, _, acc = inverse.mh_chain([1.0], [0.0], np.array([[0.1]]), np.array([[0.5]]), 1.0, 2.0, worse)
    assert not acc[0, 0] and dtr[0, 0] == 1.0  # log 0.5 > -10
    dtr, _, acc = inverse.mh_chain([1.0], [0.0], np.array([[0.1]]), np.array([[1e-6]]), 1.0, 2.0, worse)
    assert acc[0, 0]  # log 1e-6 = -13.8 < -10


def test_mh_samples_a_known_gaussian():
    mu, s = 2.0, 0.3
    target = lambda d: -0.5 * ((np.asarray(d) - mu) / s) ** 2
    rng = np.random.default_rng(7)
    niter, n = 20000, 8
    dtr, _, acc = inverse.mh_chain(np.full(n, 1.0), target(np.full(n, 1.0)), rng.standard_normal((niter, n)),
                                   rng.uniform(size=(niter, n)), 0.5, 10.0, target)
    x = dtr[2000:].ravel()
    assert abs(x.mean() - mu) < 0.02
    assert abs(x.std() - s) < 0.02
    assert 0.2 < acc.mean() < 0.9


def _tiny_plate(**kw):
    return W.corrosion_plate(6, 3, 6, nsteps=4, dt=2.0, **kw)


def test_forward_energy_balance():
    pl = _tiny_plate()
    u = inverse.forward(pl, 4.0)
    p = pl.problem()
    p.rho_c, p.k = inverse.corrosion_coefficients(p.nx, p.ny, p.nz, p.origin, p.extent, pl.geom, 4.0)
    M = fem.assemble(p.nx, p.ny, p.nz, p.extent, p.rho_c, "M")
    F = fem.face_load_elements(p.nx, p.ny, p.nz, p.extent, pl.flux_face, pl.flux_q)
    one = np.ones(p.n_nodes)
    lhs = one @ (M @ u)
    rhs = one @ (M @ np.full(p.n_nodes, pl.u0)) + pl.nsteps * pl.dt * F.sum()
    assert math.isclose(lhs, rhs, rel_tol=1e-10)


def test_forward_independent_of_depth_for_one_material():
    pl = _tiny_plate()
    pl.geom = dict(pl.geom, rho_c_corr=pl.geom["rho_c_sound"], k_corr=pl.geom["k_sound"])
    assert np.array_equal(inverse.forward(pl, 0.0), inverse.forward(pl, 6.0))


def test_forward_uses_the_corrosion_coefficients():
    # all-covering corrosion must equal a plate built with the corroded
    # material everywhere (coefficients set directly, not by the profile test)
    pl = _tiny_plate()
    pl.geom = dict(pl.geom, half_width=1e9)
    u = inverse.forward(pl, 2.0 * pl.extent[1])
    p = pl.problem()
    p.rho_c[:] = pl.geom["rho_c_corr"]
    p.k[:] = pl.geom["k_corr"]
    from oracle import transient
    S = transient.build_system(p)
    S.F = fem.face_load_elements(p.nx, p.ny, p.nz, p.extent, pl.flux_face, pl.flux_q)
    ref = transient.run(p, solver="direct", system=S).u[-1]
    assert np.allclose(u, ref, rtol=1e-12, atol=0.0)
    assert not np.array_equal(inverse.forward(_tiny_plate(), 0.0), u)
