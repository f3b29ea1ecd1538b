"""Full-size solves in the launch configuration bench.py times, checked at
sampled rows.

The 200^3 layered cube (8,120,601 nodes) and the 256 x 40^3 batch are too
large for the oracle's solvers, but any row of the step equation of §3.1,

    sum_j (M/dt + theta K)_ij u^n_j = sum_j (M/dt - (1-theta) K)_ij u^{n-1}_j + F^n_i

(free rows i; u^n and u^{n-1} hold the Dirichlet values on Dirichlet nodes),
is a plain sum the oracle's row apply computes element by element. The
solver's stopping rule bounds the whole residual relative to the right-hand
side by rtol, so the sampled residual must be small relative to the sampled
right-hand side; a wrong operator, boundary or schedule anywhere in the
sampled rows gives a residual of the order of the right-hand side. The kernel
table is tuned first, as bench.py does.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# rtol 1e-10 solves; the sampled relative residual may exceed rtol (the
# solver bounds the P^-1-weighted norm of the whole vector), but a defect
# gives O(1e-3 .. 1).
SAMPLED_BOUND = 1e-7


def _sample_rows(p, rng, n):
    dirs = set(fem.dirichlet_nodes(p)[0].tolist())
    rows = [int(i) for i in rng.integers(0, p.n_nodes, 3 * n) if int(i) not in dirs][:n]
    # corners and face centres of the box as well
    nx, ny, nz = p.nx, p.ny, p.nz
    for (i, j, k) in [(0, 0, nz), (nx, ny, nz), (nx // 2, ny // 2, nz), (nx, 0, nz // 2), (0, ny // 2, 1)]:
        m = fem.node_id(nx, ny, i, j, k)
        if m not in dirs:
            rows.append(m)
    return np.array(rows)


def _step_residual(p, u_prev, u_new, n, rows):
    """(A u^n - L u^{n-1} - F^n) and (L u^{n-1} + F^n) at the sampled free rows."""
    lhs = fem.apply_rows(p, u_new, rows, 1.0 / p.dt, p.theta, eliminate=False)
    rhs = fem.apply_rows(p, u_prev, rows, 1.0 / p.dt, p.theta - 1.0, eliminate=False)
    if p.flux and (p.flux_steps < 0 or n <= p.flux_steps):
        rhs = rhs + fem.flux_vector(p)[rows]
    return lhs - rhs, rhs


def _tune(hg, p, precision):
    with hg.Simulation.from_problem(p, precision=precision) as s:
        s.step(1)
        hg.heat_autotune(s.sim, 16)


@pytest.fixture
def restore_table():
    import paper_1905_07622_gb300 as hg
    old = hg.heat_tuning_get()
    yield
    hg.heat_tuning_set(old["variant"], old["seg_nodes"], old["pw_quads"])


def test_inclusions_100_tuned_steps_satisfy_step_equation(restore_table):
    import paper_1905_07622_gb300 as hg
    p = W.inclusions_cube(nsteps=3)
    _tune(hg, p, "fp32_refined")  # the headline configuration, tuned as bench.py does
    with hg.Simulation.from_problem(p, precision="fp32_refined") as s:
        us = [s.state()]
        for _ in range(3):
            assert s.step(1)["status"] == 0
            us.append(s.state())
    rng = np.random.default_rng(4)
    rows = _sample_rows(p, rng, 800)
    for n in (1, 2, 3):
        res, rhs = _step_residual(p, us[n - 1], us[n], n, rows)
        rel = np.linalg.norm(res) / np.linalg.norm(rhs)
        assert rel <= SAMPLED_BOUND, (n, rel)


@pytest.mark.parametrize("precision", ["fp32_refined", "fp64"])
def test_layered_200_steps_satisfy_step_equation(precision, restore_table):
    import paper_1905_07622_gb300 as hg
    p = W.layered_cube(nsteps=2)
    _tune(hg, p, precision)
    with hg.Simulation.from_problem(p, precision=precision) as s:
        us = [s.state()]
        for _ in range(2):
            st = s.step(1)
            assert st["status"] == 0
            us.append(s.state())
    rng = np.random.default_rng(5)
    rows = _sample_rows(p, rng, 600)
    for n in (1, 2):
        res, rhs = _step_residual(p, us[n - 1], us[n], n, rows)
        rel = np.linalg.norm(res) / np.linalg.norm(rhs)
        assert rel <= SAMPLED_BOUND, (precision, n, rel)
    # Dirichlet nodes keep their values (z = 0 face at 1)
    dn, dv = fem.dirichlet_nodes(p)
    assert np.array_equal(us[2][dn[:1000]], dv[:1000])


def test_batch_256x40_members_satisfy_step_equation(restore_table):
    import paper_1905_07622_gb300 as hg
    ps = [W.lognormal_cube(s, n=40, nsteps=2) for s in range(256)]
    sims = [hg.Simulation.from_problem(p, precision="fp32_refined") for p in ps]
    try:
        b = hg.heat_batch_create([s.sim for s in sims])
        try:
            rc, _ = hg.heat_batch_step(b, 1, len(ps))
            assert rc == 0
            hg.heat_batch_autotune(b, 16)  # as bench.py tunes the batch
            for s, p in zip(sims, ps):
                hg.heat_set_history(s.sim, p.u0, None, 0, p.n_nodes)
            got = {k: [ps[k].u0.copy()] for k in (0, 7, 100, 255)}
            for _ in range(2):
                rc, stats = hg.heat_batch_step(b, 1, len(ps))
                assert rc == 0, hg.heat_last_error()
                for k in got:
                    got[k].append(sims[k].state())
        finally:
            hg.heat_destroy_batch(b)
    finally:
        for s in sims:
            s.close()
    rng = np.random.default_rng(6)
    for k, us in got.items():
        p = ps[k]
        rows = _sample_rows(p, rng, 300)
        for n in (1, 2):
            res, rhs = _step_residual(p, us[n - 1], us[n], n, rows)
            rel = np.linalg.norm(res) / np.linalg.norm(rhs)
            assert rel <= SAMPLED_BOUND, (k, n, rel)
    # a member run alone under the same table is bitwise the batch member
    with hg.Simulation.from_problem(ps[7], precision="fp32_refined") as s:
        alone = []
        for _ in range(2):
            s.step(1)
            alone.append(s.state())
    assert np.array_equal(alone[0], got[7][1]) and np.array_equal(alone[1], got[7][2])
