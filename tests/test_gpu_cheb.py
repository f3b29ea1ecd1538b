"""The Chebyshev-Jacobi preconditioner on the GPU against the oracle.

- interval: lam_hi equals the oracle's element-wise Gershgorin bound (the
  same definition, summed in another order) and follows coefficient and
  parameter changes; lam_lo = lam_hi / ratio;
- FP64 path: per-step CG iterations within 2 of the oracle's Chebyshev PCG
  (same x0, interval, stopping rule and true-residual period), fewer than
  Jacobi's, and every step's state within 1e-9 of the exact step solution;
- FP32 refined path: every step within 1e-8 of the exact step solution,
  plain and ragged meshes, a mesh with no free node;
- a batch mixing degrees and Jacobi members gives each member bitwise its
  result alone; switching the preconditioner on and off between steps, and a
  fused tuning variant (replaced by its register-prefetch form), still agree
  with the oracle;
- parameter validation.
"""
import numpy as np
import pytest

import workloads as W
from oracle import precond, transient

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _run(p, precision, nsteps=None, **kw):
    import paper_1905_07622_gb300 as hg
    us, stats = [], []
    with hg.Simulation.from_problem(p, precision=precision, **kw) as s:
        us.append(s.state())
        for _ in range((nsteps or p.nsteps)):
            stats.append(s.step(1))
            us.append(s.state())
    return us, stats


def _stiff(nsteps=4, seed=4, dims=(12, 10, 14)):
    return W.random_box(*dims, seed=seed, dt=10.0, contrast=(0.01, 100.0), dirichlet={4: 1.0}, flux={3: 0.5},
                        nsteps=nsteps, rtol=1e-10)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
@pytest.mark.parametrize("seed,extent,ratio", [(0, (1.0, 1.0, 1.0), 10.0), (1, (2.0, 0.5, 1.0), 4.0),
                                               (2, (0.3, 1.0, 3.0), 100.0)])
def test_interval_is_the_element_bound(precision, seed, extent, ratio):
    import paper_1905_07622_gb300 as hg
    p = W.random_box(7, 5, 6, seed=seed, extent=extent, contrast=(0.001, 1000.0), dt=0.05)
    with hg.Simulation.from_problem(p, precision=precision, cheb_degree=3, cheb_ratio=ratio) as s:
        lo, hi = hg.heat_cheb_interval(s.sim)
        ref = precond.element_lam_max(p)
        assert abs(hi - ref) <= 1e-13 * ref and lo == hi / ratio
        # new coefficients and a new dt move the bound
        p.k = np.random.default_rng(seed).uniform(0.5, 2.0, p.n_elems)
        hg.heat_set_coeffs(s.sim, p.rho_c, p.k, p.n_elems)
        p.dt = 0.7
        s.set_params(theta=p.theta, dt=p.dt, rtol=p.rtol, precision=precision, cheb_degree=3, cheb_ratio=ratio)
        lo, hi = hg.heat_cheb_interval(s.sim)
        ref = precond.element_lam_max(p)
        assert abs(hi - ref) <= 1e-13 * ref


@pytest.mark.parametrize("degree", [2, 3, 5])
def test_fp64_iterations_match_oracle_chebyshev_pcg(degree):
    p = _stiff()
    S = transient.build_system(p)
    exact = transient.run(p, solver="direct", system=S)
    ref = transient.run(p, solver="pcg", system=S, cheb=(degree, 10.0))
    jac = transient.run(p, solver="pcg", system=S)
    us, stats = _run(p, "fp64", cheb_degree=degree, cheb_ratio=10.0)
    got = [st["iters"] for st in stats]
    assert all(st["status"] == 0 for st in stats)
    assert all(abs(a - b) <= 2 for a, b in zip(got, ref.iters)), (got, ref.iters)
    assert sum(got) < sum(jac.iters), (got, jac.iters)
    errs = [_rel(us[n], exact.u[n]) for n in range(1, p.nsteps + 1)]
    assert max(errs) <= 1e-9, errs


def test_fp64_true_residual_period_with_chebyshev():
    # a long solve crosses two true-residual replacements (every 50 iterations):
    # a 16^3 laminate of 8 layers, k alternating 1 / 1000
    p = W.layered_cube(n=16, n_layers=8, n_pockets=4)
    p.dt, p.nsteps, p.rtol = 1.0, 2, 1e-11
    S = transient.build_system(p)
    exact = transient.run(p, solver="direct", system=S)
    ref = transient.run(p, solver="pcg", system=S, cheb=(2, 30.0))
    us, stats = _run(p, "fp64", cheb_degree=2, cheb_ratio=30.0)
    got = [st["iters"] for st in stats]
    assert max(got) > 100, got
    assert all(abs(a - b) <= 2 for a, b in zip(got, ref.iters)), (got, ref.iters)
    assert max(_rel(us[n], exact.u[n]) for n in range(1, p.nsteps + 1)) <= 1e-9


@pytest.mark.parametrize("degree", [2, 4, 8])
@pytest.mark.parametrize("dims,dirichlet", [((12, 10, 14), {4: 1.0}), ((33, 5, 9), {0: 1.0, 3: -0.5}),
                                            ((3, 40, 2), {}), ((1, 1, 1), {f: 0.3 for f in range(6)})])
def test_fp32_refined_every_step(degree, dims, dirichlet):
    p = W.random_box(*dims, seed=4, dt=1.0, contrast=(0.01, 100.0), dirichlet=dirichlet, flux={2: 1.0}, nsteps=3,
                     rtol=1e-12)
    exact = transient.run(p, solver="direct")
    us, stats = _run(p, "fp32_refined", cheb_degree=degree)
    assert all(st["status"] == 0 for st in stats)
    errs = [_rel(us[n], exact.u[n]) for n in range(1, p.nsteps + 1)]
    assert max(errs) <= 1e-8, errs


def test_batch_mixing_degrees_is_bitwise_alone():
    import paper_1905_07622_gb300 as hg
    probs = [_stiff(3, seed=s, dims=d) for s, d in ((1, (12, 10, 14)), (2, (9, 17, 6)), (3, (20, 8, 11)))]
    degrees = [2, 0, 4]
    for precision in ("fp32_refined", "fp64"):
        alone = []
        for p, m in zip(probs, degrees):
            us, _ = _run(p, precision, cheb_degree=m)
            alone.append(us[-1])
        sims = [hg.Simulation.from_problem(p, precision=precision, cheb_degree=m) for p, m in zip(probs, degrees)]
        try:
            batch = hg.heat_batch_create([s.sim for s in sims])
            try:
                rc, per = hg.heat_batch_step(batch, probs[0].nsteps, len(sims))
                assert rc == 0
            finally:
                hg.heat_destroy_batch(batch)
            for s, a in zip(sims, alone):
                assert np.array_equal(s.state(), a)
        finally:
            for s in sims:
                s.close()


def test_switching_the_preconditioner_between_steps():
    import paper_1905_07622_gb300 as hg
    p = _stiff(6)
    exact = transient.run(p, solver="direct")
    kw = dict(theta=p.theta, dt=p.dt, rtol=p.rtol, precision="fp32_refined")
    with hg.Simulation.from_problem(p, precision="fp32_refined") as s:
        for n, m in enumerate((0, 0, 3, 3, 0, 2), start=1):
            s.set_params(cheb_degree=m, **kw)
            st = s.step(1)
            assert st["status"] == 0
            assert _rel(s.state(), exact.u[n]) <= 1e-8


def test_fused_variant_is_replaced_with_chebyshev():
    import paper_1905_07622_gb300 as hg
    saved = hg.heat_tuning_get()
    fused = [v for v in range(hg.heat_tuning_num_variants()) if hg.heat_tuning_variant(v)["fused"]]
    try:
        hg.heat_tuning_set([saved["variant"][0], fused[0], fused[0]], saved["seg_nodes"], saved["pw_quads"])
        p = _stiff(3)
        exact = transient.run(p, solver="direct")
        us, stats = _run(p, "fp32_refined", cheb_degree=3)
        assert max(_rel(us[n], exact.u[n]) for n in range(1, p.nsteps + 1)) <= 1e-8
        us0, _ = _run(p, "fp32_refined")  # the fused iteration itself, for contrast
        assert max(_rel(us0[n], exact.u[n]) for n in range(1, p.nsteps + 1)) <= 1e-8
    finally:
        hg.heat_tuning_set(saved["variant"], saved["seg_nodes"], saved["pw_quads"])


def test_parameter_validation():
    import paper_1905_07622_gb300 as hg
    p = W.random_box(3, 3, 3, seed=0)
    with hg.Simulation.from_problem(p) as s:
        with pytest.raises(hg.HeatError):
            hg.heat_cheb_interval(s.sim)  # preconditioner off
        for bad in (dict(cheb_degree=9), dict(cheb_degree=-1), dict(cheb_degree=2, cheb_ratio=1.0),
                    dict(cheb_degree=2, cheb_ratio=float("inf"))):
            with pytest.raises(hg.HeatError):
                s.set_params(**bad)
        s.set_params(cheb_degree=1, cheb_ratio=1.0)  # degree 1 is Jacobi: the ratio is unused
        with pytest.raises(hg.HeatError):
            hg.heat_cheb_interval(s.sim)
