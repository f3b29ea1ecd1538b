"""The inverse-problem pieces (§5.3) on the GPU against the oracle.

- per-element face flux: the flux vector equals the oracle's face loads;
- corrosion coefficients: bitwise the oracle's (an FP64 test decides each
  element, both sides round every operation alike);
- face log-likelihood of a given state: the oracle's sum of squares;
- batched Metropolis-Hastings: each proposal's log-likelihood matches the
  oracle's forward model, and with the same random draws the chains make the
  oracle's accept/reject decisions.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, inverse

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _plate():
    return W.corrosion_plate(12, 5, 10, nsteps=6, dt=1.0, rtol=1e-12)


def _geom(hg, g):
    return hg.make_corrosion(g["z0"], g["half_width"], g["rho_c_sound"], g["k_sound"], g["rho_c_corr"], g["k_corr"])


def _sim(hg, pl, p):
    return hg.Simulation.from_problem(p, precision="fp64")


@pytest.mark.parametrize("face", [0, 3, 5])
def test_face_flux_vector_matches_oracle(face):
    import paper_1905_07622_gb300 as hg
    p = W.random_box(7, 5, 6, seed=31, extent=(1.4, 0.5, 0.9), flux={2: 0.3, 4: -0.2})
    na = (p.ny, p.nx, p.nx)[face // 2]
    nb = (p.nz, p.nz, p.ny)[face // 2]
    q = np.random.default_rng(face).uniform(-1, 2, na * nb)
    with hg.Simulation.from_problem(p) as s:
        hg.heat_set_face_flux(s.sim, face, q)
        F = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
        hg.heat_flux_vector(s.sim, F)
        got = F.cpu().numpy()
        hg.heat_set_face_flux(s.sim, face, None)  # back to uniform
        hg.heat_flux_vector(s.sim, F)
        back = F.cpu().numpy()
    ref_uniform = fem.flux_vector(p)
    ref = ref_uniform - fem.face_load(p.nx, p.ny, p.nz, p.extent, face, p.flux.get(face, 0.0)) + \
        fem.face_load_elements(p.nx, p.ny, p.nz, p.extent, face, q)
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-14 * scale
    assert np.abs(back - ref_uniform).max() <= 1e-14 * np.abs(ref_uniform).max()


@pytest.mark.parametrize("depth", [0.0, 1.3, 3.175, 7.9, 12.7])
def test_corrosion_coefficients_bitwise(depth):
    import paper_1905_07622_gb300 as hg
    pl = W.corrosion_plate(17, 9, 23)
    p = pl.problem()
    with hg.Simulation.from_problem(p) as s:
        hg.heat_set_coeffs_corrosion(s.sim, _geom(hg, pl.geom), depth)
        rc, k = hg.heat_get_coeffs(s.sim, p.n_elems)
    ref_rc, ref_k = inverse.corrosion_coefficients(p.nx, p.ny, p.nz, p.origin, p.extent, pl.geom, depth)
    assert np.array_equal(rc, ref_rc) and np.array_equal(k, ref_k)


@pytest.mark.parametrize("face", [2, 1, 4])
def test_face_loglik_matches_oracle(face):
    import paper_1905_07622_gb300 as hg
    p = W.random_box(9, 6, 7, seed=32)
    rng = np.random.default_rng(3)
    ids = fem.face_nodes(p.nx, p.ny, p.nz, face)
    data = p.u0[ids] + rng.normal(0, 0.2, len(ids))
    with hg.Simulation.from_problem(p) as s:
        d = torch.tensor(data, device="cuda")
        out = torch.zeros(1, dtype=torch.float64, device="cuda")
        hg.heat_face_loglik(s.sim, face, d, 0.2, out)
        got = float(out.item())
    ref = inverse.loglik(inverse.face_values(p.u0, p.nx, p.ny, p.nz, face), data, 0.2)
    assert abs(got - ref) <= 1e-12 * abs(ref)


def _driver(hg, pl, data, nchains, precision="fp64"):
    return hg.MHDriver(pl.nx, pl.ny, pl.nz, pl.extent, _geom(hg, pl.geom), data, pl.sigma, nchains, pl.nsteps,
                       pl.depth_max, flux_face=pl.flux_face, flux_q=pl.flux_q, obs_face=pl.obs_face, u0=pl.u0,
                       theta=pl.theta, dt=pl.dt, rtol=pl.rtol, precision=precision)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_mh_loglik_matches_oracle_forward_model(precision):
    import paper_1905_07622_gb300 as hg
    pl = _plate()
    u_true = inverse.forward(pl, pl.depth_true)
    data = pl.camera(inverse.face_values(u_true, pl.nx, pl.ny, pl.nz, pl.obs_face))
    depths = np.array([0.0, 2.0, pl.depth_true, 6.5])
    with _driver(hg, pl, data, len(depths), precision) as mh:
        got = mh.loglik(depths)
    for d, g in zip(depths, got):
        u = inverse.forward(pl, d)
        ref = inverse.loglik(inverse.face_values(u, pl.nx, pl.ny, pl.nz, pl.obs_face), data, pl.sigma)
        assert abs(g - ref) <= 1e-7 * (1.0 + abs(ref)), (d, g, ref)


def test_mh_chains_make_the_oracle_decisions():
    import paper_1905_07622_gb300 as hg
    pl = _plate()
    u_true = inverse.forward(pl, pl.depth_true)
    data = pl.camera(inverse.face_values(u_true, pl.nx, pl.ny, pl.nz, pl.obs_face))
    nchains, niter, step = 4, 5, 1.5
    normals, uniforms = pl.draws(niter, nchains)
    start = np.array([1.0, 4.0, 8.0, 11.0])

    calls = []

    def oracle_ll(depths):
        out = []
        for d in depths:
            u = inverse.forward(pl, d)
            out.append(inverse.loglik(inverse.face_values(u, pl.nx, pl.ny, pl.nz, pl.obs_face), data, pl.sigma))
        calls.append(np.array(out))
        return calls[-1]

    ll0 = oracle_ll(start)
    dtr_ref, ltr_ref, acc_ref = inverse.mh_chain(start, ll0, normals, uniforms, step, pl.depth_max, oracle_ll)
    # every in-prior decision is far from the threshold log(u) = ll' - ll, so
    # rounding differences below 1e-6 cannot flip it
    prev = ll0
    for it in range(niter):
        prop = np.where(acc_ref[it], dtr_ref[it], (dtr_ref[it - 1] if it else start) + step * normals[it])
        inside = (prop >= 0) & (prop <= pl.depth_max)
        margin = np.abs(np.log(uniforms[it]) - (calls[it + 1] - prev))
        assert np.all(margin[inside] > 1e-6), (it, margin)
        prev = ltr_ref[it]
    with _driver(hg, pl, data, nchains) as mh:
        st, ll, dtr, ltr, acc = mh.run(niter, step, normals, uniforms, start)
    # no decision of this draw sequence lies within 1e-6 of the acceptance threshold
    assert np.array_equal(acc, acc_ref)
    assert np.array_equal(dtr, dtr_ref)
    assert np.allclose(ltr, ltr_ref, rtol=1e-7, atol=1e-7)
    assert np.array_equal(st, dtr_ref[-1])
