"""Checkpoint/resume, failure statuses and parameter changes between steps.

Failures are made on the host side of the data (a NaN placed in a device
array, an iteration cap that cannot be met): the kernels detect them and
return a status; nothing faults or hangs the GPU.
"""
import numpy as np
import pytest

import pins
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_checkpoint_resume_is_bitwise(precision):
    import paper_1905_07622_gb300 as hg
    p = W.random_box(14, 9, 11, seed=8, dirichlet={3: 0.25}, flux={5: 1.0}, flux_steps=4, theta=0.5,
                     dt=0.01, nsteps=6, rtol=1e-11)
    with hg.Simulation.from_problem(p, precision=precision) as a:
        a.step(6)
        straight = a.state()
    with hg.Simulation.from_problem(p, precision=precision) as b:
        b.step(3)
        u1, u2, step = hg.heat_get_history(b.sim, p.n_nodes)
    assert step == 3 and u2 is not None
    with hg.Simulation.from_problem(p, precision=precision) as c:
        hg.heat_set_history(c.sim, u1, u2, step, p.n_nodes)
        c.step(3)  # steps 4..6: the flux switches off after step 4 as in the straight run
        resumed = c.state()
    assert np.array_equal(resumed, straight)


def test_nan_in_device_state_returns_nonfinite_then_recovers():
    import paper_1905_07622_gb300 as hg
    p = W.random_box(10, 10, 10, seed=3, flux={5: 1.0}, nsteps=1, rtol=1e-10)
    with hg.Simulation.from_problem(p) as s:
        bad = torch.tensor(p.u0, device="cuda")
        bad[17] = float("nan")
        hg.heat_set_state(s.sim, bad, p.n_nodes)  # device input is not scanned on the host
        rc, st = hg.heat_step_nocheck(s.sim, 1)
        assert rc == hg.HEAT_ERR_NONFINITE and st["status"] == hg.HEAT_ERR_NONFINITE
        hg.heat_set_state(s.sim, p.u0, p.n_nodes)
        st = s.step(1)
        assert st["status"] == 0 and np.isfinite(s.state()).all()


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_iteration_cap_reports_not_converged(precision):
    import paper_1905_07622_gb300 as hg
    p = W.random_box(20, 20, 20, seed=5, flux={5: 1.0}, nsteps=1, dt=1.0, rtol=1e-12, contrast=(0.01, 100.0))
    with hg.Simulation.from_problem(p, precision=precision, max_iter=3, max_outer=2) as s:
        before = s.state()
        rc, st = hg.heat_step_nocheck(s.sim, 1)
        assert rc == hg.HEAT_ERR_NOT_CONVERGED and st["status"] == hg.HEAT_ERR_NOT_CONVERGED
        assert st["steps"] == 0
        assert np.array_equal(s.state(), before)  # the step was not committed


def test_params_and_precision_change_between_steps():
    import paper_1905_07622_gb300 as hg
    p = W.random_box(8, 7, 9, seed=6, flux={0: 1.0}, theta=0.5, dt=0.01, nsteps=2, rtol=1e-12)
    with hg.Simulation.from_problem(p, precision="fp64") as s:
        s.step(2)
        mid = s.state()
        s.set_params(theta=1.0, dt=0.03, rtol=1e-12, precision="fp32_refined")
        s.step(2)
        got = s.state()
    # oracle: two steps of the first scheme, then two of the second from there
    p1 = W.random_box(8, 7, 9, seed=6, flux={0: 1.0}, theta=0.5, dt=0.01, nsteps=2, rtol=1e-12)
    r1 = pins.oracle_steps(p1)
    assert np.linalg.norm(mid - r1.u[-1]) <= 1e-9 * np.linalg.norm(r1.u[-1])
    p2 = W.random_box(8, 7, 9, seed=6, flux={0: 1.0}, theta=1.0, dt=0.03, nsteps=2, rtol=1e-12)
    p2.u0 = r1.u[-1]
    r2 = pins.oracle_steps(p2)
    assert np.linalg.norm(got - r2.u[-1]) <= 1e-8 * np.linalg.norm(r2.u[-1])


def test_step_argument_checks():
    import paper_1905_07622_gb300 as hg
    p = W.random_box(3, 3, 3, seed=1)
    with hg.Simulation.from_problem(p) as s:
        assert s.step(0)["steps"] == 0
        with pytest.raises(hg.HeatError):
            hg.heat_step(s.sim, -1)
        with pytest.raises(hg.HeatError):
            s.set_params(theta=0.0)
