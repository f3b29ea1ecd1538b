"""Batched simulations: each member alone and in the batch, vs the oracle.

A batch carries simulations of different sizes, coefficient fields and
boundary conditions in every launch. Each member's reductions run in the same
order as when it runs alone, so its states must be bitwise identical; and each
must match the oracle's step solutions within the path's tolerance.
"""
import numpy as np
import pytest

import pins
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _problems():
    return [
        W.random_box(7, 5, 3, seed=1, dirichlet={0: 0.5}, flux={5: 1.0}, theta=0.5, dt=0.01, nsteps=4,
                     rtol=1e-11),
        W.random_box(20, 13, 9, seed=2, flux={2: -1.0}, theta=1.0, dt=0.02, nsteps=4, rtol=1e-11,
                     contrast=(0.1, 10.0)),
        W.lognormal_cube(0, n=40, nsteps=4),
        W.random_box(33, 9, 17, seed=3, dirichlet={4: 1.0, 3: -0.5}, theta=0.5, dt=0.005, nsteps=4,
                     rtol=1e-11),
        W.random_box(12, 12, 12, seed=4, flux={0: 2.0}, flux_steps=2, theta=0.7, dt=0.01, nsteps=4,
                     rtol=1e-11),
    ]


def _run_alone(p, precision):
    import paper_1905_07622_gb300 as hg
    with hg.Simulation.from_problem(p, precision=precision) as s:
        us = []
        for _ in range(p.nsteps):
            s.step(1)
            us.append(s.state())
        return us


def _run_batch(ps, precision):
    import paper_1905_07622_gb300 as hg
    sims = [hg.Simulation.from_problem(p, precision=precision) for p in ps]
    try:
        b = hg.heat_batch_create([s.sim for s in sims])
        try:
            out = [[] for _ in ps]
            for _ in range(max(p.nsteps for p in ps)):
                rc, stats = hg.heat_batch_step(b, 1, len(ps))
                assert rc == 0, hg.heat_last_error()
                assert all(st["steps"] == 1 for st in stats)
                for k, s in enumerate(sims):
                    out[k].append(s.state())
            return out
        finally:
            hg.heat_destroy_batch(b)
    finally:
        for s in sims:
            s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32_refined", 1e-8)])
def test_batch_members_bitwise_equal_to_alone_and_match_oracle(precision, tol):
    ps = _problems()
    batch = _run_batch(ps, precision)
    for k, p in enumerate(ps):
        alone = _run_alone(p, precision)
        for n in range(p.nsteps):
            assert np.array_equal(batch[k][n], alone[n]), (k, n)
        ref = pins.oracle_steps(p)
        for n in range(1, p.nsteps + 1):
            err = np.linalg.norm(batch[k][n - 1] - ref.u[n]) / np.linalg.norm(ref.u[n])
            assert err <= tol, (k, n, err)


def test_lognormal_batch_of_eight():
    """Eight log-normal 40^3 samples (the batched workload's shape), 3 steps."""
    ps = [W.lognormal_cube(s, n=40, nsteps=3) for s in range(8)]
    batch = _run_batch(ps, "fp32_refined")
    for k in (0, 5):
        ref = pins.oracle_steps(ps[k])
        for n in range(1, 4):
            err = np.linalg.norm(batch[k][n - 1] - ref.u[n]) / np.linalg.norm(ref.u[n])
            assert err <= 1e-8
    # distinct samples give distinct fields
    assert not np.array_equal(batch[0][-1], batch[1][-1])


def test_batch_rejects_mixed_precision_and_duplicates():
    import paper_1905_07622_gb300 as hg
    p = W.random_box(4, 4, 4, seed=1)
    with hg.Simulation.from_problem(p, precision="fp64") as a, \
            hg.Simulation.from_problem(p, precision="fp32_refined") as b:
        with pytest.raises(hg.HeatError):
            hg.heat_batch_create([a.sim, b.sim])
        with pytest.raises(hg.HeatError):
            hg.heat_batch_create([a.sim, a.sim])
