"""Full-size solves in the launch configuration bench.py times, checked over
every row of the step equation.

The 200^3 layered cube (8,120,601 nodes), the 100^3 inclusions cube and the
256 x 40^3 batch are too large for the oracle's solvers, but the residual of
the step equation of §3.1 on the free rows,

    r = (M/dt + theta K) u^n - (M/dt - (1-theta) K) u^{n-1} - F^n

(u^n and u^{n-1} hold the Dirichlet values on Dirichlet nodes), is a plain
element-by-element product the oracle forms over the whole mesh
(fem.apply_all). The solver's stopping rule (Algorithm 1 with the relative
reading) ends a step when r^T P^-1 r <= rtol^2 b^T P^-1 b, P the Jacobi
diagonal and b the right-hand side of the eliminated system on the free rows,
b = (L u^{n-1} + F^n) - A_{fD} g: the Dirichlet columns of A move to the
right-hand side. So in the P^-1-weighted norm

    rho = ||r||_{P^-1} / ||b||_{P^-1}  <=  rtol + c * u * ||A||u^n|| ||_{P^-1} / ||b||_{P^-1},

where the second term bounds the rounding in forming r, on the GPU (the
quantity the stopping test saw) and in the oracle (the quantity checked here):
|A||u| is the product with every term taken by magnitude, u the unit roundoff
of the arithmetic that formed the tested residual and c the number of rounded
operations one output of the operator passes through, at most 64 on both
sides (27 terms, or the factorised form's three butterfly levels each way, its
scaling and the face and node sums). Both paths close a step on a true
residual b - A x: the FP64 path recomputes it in FP64 once its recurrence
residual meets the rule, and the refined path forms it in double-float
arithmetic (u = 2^-48). A defect in the operator, a boundary or the schedule gives
rho of the order of 1 against bounds of 1e-10 to 1e-8.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, transient

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U64, UDF = 2.0 ** -53, 2.0 ** -48
C_OPS = 64


def rounding_unit(precision):
    """Unit roundoff times operations: the GPU's evaluation of the residual
    its stopping test saw, plus the oracle's evaluation here (FP64)."""
    if precision == "fp64":
        return 2 * C_OPS * U64
    return C_OPS * UDF + C_OPS * U64


def step_residual(p, u_prev, u_new, n):
    """(rho, bound scale) of step n over every free row: rho as above, and
    ||A||u^n|| ||_{P^-1} / ||b||_{P^-1}."""
    b = fem.apply_all(p, u_prev, 1.0 / p.dt, p.theta - 1.0, eliminate=False)
    if p.flux and transient.flux_on(p, n):
        b += fem.flux_vector(p)
    au = fem.apply_all(p, u_new, 1.0 / p.dt, p.theta, eliminate=False)
    dn = fem.dirichlet_nodes(p)[0]
    g = np.zeros(p.n_nodes)
    g[dn] = u_new[dn]
    lift = fem.apply_all(p, g, 1.0 / p.dt, p.theta, eliminate=False)  # A_{.D} g
    # r = A_ff u_f - b_f with b_f = b - A_fD g on the free rows: au - b as before
    b = b - lift
    absau = fem.apply_all(p, u_new, 1.0 / p.dt, p.theta, eliminate=False, absolute=True)
    d = fem.diagonal_all(p, 1.0 / p.dt, p.theta)
    free = np.ones(p.n_nodes, dtype=bool)
    free[dn] = False
    w = 1.0 / d[free]
    nb = np.sqrt(np.sum(b[free] ** 2 * w))
    rho = np.sqrt(np.sum((au - lift - b)[free] ** 2 * w)) / nb
    scale = np.sqrt(np.sum(absau[free] ** 2 * w)) / nb
    return rho, scale


def check_steps(p, us, precision, rtol):
    for n in range(1, len(us)):
        rho, scale = step_residual(p, us[n - 1], us[n], n)
        bound = rtol * (1 + 1e-6) + rounding_unit(precision) * scale
        print(f"{p.name} {precision} step {n}: rho {rho:.3e}  bound {bound:.3e}  |A||u|/b {scale:.2e}")
        assert rho <= bound, (p.name, precision, n, rho, bound)


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


def _run(hg, p, precision, nsteps):
    with hg.Simulation.from_problem(p, precision=precision) as s:
        us = [s.state()]
        for _ in range(nsteps):
            st = s.step(1)
            assert st["status"] == 0, st
            us.append(s.state())
    return us


def test_inclusions_100_tuned_steps_satisfy_step_equation(restore_table):
    import paper_1905_07622_gb300 as hg
    p = W.inclusions_cube(nsteps=3)
    _tune(hg, p, "fp32_refined")  # the headline configuration, tuned as bench.py does
    us = _run(hg, p, "fp32_refined", 3)
    check_steps(p, us, "fp32_refined", p.rtol)


@pytest.mark.parametrize("precision", ["fp32_refined", "fp64"])
def test_layered_200_steps_satisfy_step_equation(precision, restore_table):
    import paper_1905_07622_gb300 as hg
    p = W.layered_cube(nsteps=2)
    _tune(hg, p, precision)
    us = _run(hg, p, precision, 2)
    check_steps(p, us, precision, p.rtol)
    # Dirichlet nodes keep their values (z = 0 face at 1)
    dn, dv = fem.dirichlet_nodes(p)
    assert np.array_equal(us[2][dn], dv)


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
    for k, us in got.items():
        check_steps(ps[k], us, "fp32_refined", ps[k].rtol)
    # a member run alone under the same table is bitwise the batch member
    with hg.Simulation.from_problem(ps[7], precision="fp32_refined") as s:
        alone = []
        for _ in range(2):
            s.step(1)
            alone.append(s.state())
    assert np.array_equal(alone[0], got[7][1]) and np.array_equal(alone[1], got[7][2])
