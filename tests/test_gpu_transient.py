"""GPU transient solves through the C ABI vs the CPU oracle.

Tolerances (relative L2 per step against the oracle's exact step solution):
FP64 path <= 1e-9, refined FP32 path <= 1e-8; the plain FP32 error is only
reported (bounded loosely so a broken path still fails).
"""
import numpy as np
import pytest

import pins
import workloads as W
from oracle import pcg, transient

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _run_gpu(p, precision, nsteps=None, **kw):
    import paper_1905_07622_gb300 as hg
    us, stats = [], []
    with hg.Simulation.from_problem(p, precision=precision, **kw) as s:
        us.append(s.state())
        for n in range(1, (nsteps or p.nsteps) + 1):
            stats.append(s.step(1))
            us.append(s.state())
    return us, stats


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module")
def two_phase():
    p = W.two_phase_cube()
    return p, transient.run(p, solver="direct")


def test_two_phase_cube_fp64_every_step(two_phase):
    p, ref = two_phase
    us, stats = _run_gpu(p, "fp64")
    errs = [_rel(us[n], ref.u[n]) for n in range(1, p.nsteps + 1)]
    assert max(errs) <= 1e-9, errs
    assert all(st["status"] == 0 for st in stats)


def test_two_phase_cube_iteration_counts_match_oracle_pcg(two_phase):
    """Same x0 and stopping rule: per-step CG iterations within a few of the oracle's."""
    p, _ = two_phase
    ref = transient.run(p, solver="pcg")
    _, stats = _run_gpu(p, "fp64")
    got = [st["iters"] for st in stats]
    assert all(abs(a - b) <= 2 for a, b in zip(got, ref.iters)), (got, ref.iters)


def test_two_phase_cube_fp32_refined_every_step(two_phase):
    p, ref = two_phase
    us, stats = _run_gpu(p, "fp32_refined")
    errs = [_rel(us[n], ref.u[n]) for n in range(1, p.nsteps + 1)]
    assert max(errs) <= 1e-8, errs
    assert all(st["outer"] >= 1 for st in stats)


def test_two_phase_cube_fp32_plain_error_reported(two_phase):
    p, ref = two_phase
    us, _ = _run_gpu(p, "fp32_plain")
    errs = [_rel(us[n], ref.u[n]) for n in range(1, p.nsteps + 1)]
    print("plain FP32 max relative error per step:", max(errs))
    assert max(errs) <= 1e-4


@pytest.mark.parametrize("kind", ["dirichlet", "mixed", "neumann"])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32_refined", 1e-9)])
def test_exact_discrete_eigenmode_on_gpu(kind, precision, tol):
    """The GPU path reproduces U^n = g^n U^0 for exact discrete eigenmodes (closed form)."""
    p, g = pins.mode_problem(kind)
    p.rtol = 1e-12
    us, _ = _run_gpu(p, precision)
    for n, u in enumerate(us):
        assert _rel(u, g ** n * us[0]) <= tol


def test_energy_balance_on_gpu():
    p = W.random_box(9, 7, 12, seed=21, extent=(1.0, 0.5, 2.0), flux={5: 1.5, 0: -0.4},
                     theta=0.5, dt=0.05, nsteps=4, flux_steps=2, rtol=1e-12)
    S = transient.build_system(p)
    us, _ = _run_gpu(p, "fp64")
    one = np.ones(p.n_nodes)
    for n in range(1, p.nsteps + 1):
        lhs = one @ (S.M @ (us[n] - us[n - 1]))
        rhs = p.dt * (one @ S.F) if transient.flux_on(p, n) else 0.0
        assert abs(lhs - rhs) <= 1e-10 * (abs(one @ (S.M @ us[0])) + 1.0)


@pytest.mark.parametrize("dims,dirichlet,theta", [
    ((1, 1, 1), {}, 1.0),
    ((1, 1, 1), {f: 0.3 for f in range(6)}, 0.5),   # no free node at all
    ((33, 5, 9), {0: 1.0, 3: -0.5}, 0.5),
    ((3, 40, 2), {5: 2.0}, 0.7),
])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_small_and_ragged_meshes(dims, dirichlet, theta, precision):
    p = W.random_box(*dims, seed=4, dirichlet=dirichlet, flux={2: 1.0}, theta=theta, dt=0.01,
                     nsteps=3, rtol=1e-12)
    ref = transient.run(p, solver="direct")
    us, _ = _run_gpu(p, precision)
    for n in range(1, p.nsteps + 1):
        assert _rel(us[n], ref.u[n]) <= (1e-9 if precision == "fp64" else 1e-8)


def test_zero_state_zero_rhs_converges_without_iterations():
    p = W.random_box(5, 5, 5, seed=2, nsteps=2)
    p.u0 = np.zeros(p.n_nodes)
    us, stats = _run_gpu(p, "fp64")
    assert all(st["iters"] == 0 for st in stats)
    assert not np.any(us[-1])


def test_inclusions_cube_first_steps_fp64_and_refined():
    """Full-size 100^3 workload (1,030,301 nodes): first 3 steps vs the oracle."""
    p = W.inclusions_cube().truncated(3)
    S = transient.build_system(p)
    ref = transient.run(p, solver="pcg", rtol=1e-13, system=S)
    for prec, tol in (("fp64", 1e-9), ("fp32_refined", 1e-8)):
        us, stats = _run_gpu(p, prec)
        for n in range(1, p.nsteps + 1):
            assert _rel(us[n], ref.u[n]) <= tol, (prec, n)
