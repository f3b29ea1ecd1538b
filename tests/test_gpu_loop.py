"""The persistent inner iteration (tuning loop = 1, k_cg_loop).

One cooperative kernel runs a tick's CG iterations (Algorithm 1's loop body,
§3.3) with a grid barrier after the apply phase and after the update phase,
on the same work items and the same per-item arithmetic as the separate
apply and update launches. So its fields, iteration counts and convergence
decisions must be bitwise those of the replayed tick graph, alone and in a
batch, and within the path's tolerance of the oracle. Its barrier waits are
bounded: a barrier that can never complete (the test hook's extra arrival)
must end the kernel with HEAT_ERR_TIMEOUT and leave the GPU usable.
"""
import numpy as np
import pytest

import pins
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def restore_table():
    import paper_1905_07622_gb300 as hg
    old = hg.heat_tuning_get()
    yield
    hg.heat_debug_loop_wait(0, 0.0)
    hg.heat_tuning_set(old["variant"], old["seg_nodes"], old["pw_quads"], old["open_w"], old["loop"])


def _problem():
    # ragged in every direction against 16- and 32-wide segments; several
    # inner solves and refinement sweeps per step
    return W.random_box(37, 11, 19, seed=21, dirichlet={2: 0.5}, flux={5: 1.0}, theta=0.5, dt=0.01, nsteps=3,
                        rtol=1e-11, contrast=(0.1, 10.0))


def _loop_variants():
    """Register-prefetch, non-fused warp variants: the shapes with a persistent form."""
    import paper_1905_07622_gb300 as hg
    out = []
    for v in range(hg.heat_tuning_num_variants()):
        i = hg.heat_tuning_variant(v)
        if i["stages"] == 0 and not i["fused"]:
            out.append(v)
    return out


def _set(precision, v, quads, loop):
    import paper_1905_07622_gb300 as hg
    pid = hg.PRECISIONS[precision]
    t = hg.heat_tuning_get()
    t["variant"][pid] = v
    t["pw_quads"][pid] = quads
    t["loop"][pid] = loop
    hg.heat_tuning_set(t["variant"], t["seg_nodes"], t["pw_quads"], t["open_w"], t["loop"])


def _solve(p, precision):
    import paper_1905_07622_gb300 as hg
    with hg.Simulation.from_problem(p, precision=precision) as s:
        us, its = [], []
        for _ in range(p.nsteps):
            st = s.step(1)
            assert st["status"] == 0
            us.append(s.state())
            its.append((st["iters"], st["outer"]))
        return us, its


@pytest.mark.parametrize("precision", ["fp32_refined", "fp32_plain"])
def test_persistent_iteration_is_bitwise_the_tick_graph(precision):
    import paper_1905_07622_gb300 as hg
    p = _problem()
    if precision == "fp32_plain":
        p.rtol = 1e-6  # what FP32 arithmetic alone reaches
    ref = pins.oracle_steps(p)
    vs = _loop_variants()
    assert vs
    for v in vs:
        for quads in (1, 2, 4):
            _set(precision, v, quads, 0)
            tick, tick_its = _solve(p, precision)
            _set(precision, v, quads, 1)
            assert hg.heat_tuning_get()["loop"][hg.PRECISIONS[precision]] == 1
            loop, loop_its = _solve(p, precision)
            assert loop_its == tick_its, (v, quads)
            for n in range(p.nsteps):
                assert np.array_equal(loop[n], tick[n]), (v, quads, n)
            if precision == "fp32_refined":
                for n in range(p.nsteps):
                    err = np.linalg.norm(loop[n] - ref.u[n + 1]) / np.linalg.norm(ref.u[n + 1])
                    assert err <= 1e-8, (v, quads, n, err)


def test_persistent_iteration_in_a_batch_is_bitwise_alone_and_tick():
    """Members of different sizes converge at different rounds: the loop goes
    on while any member iterates, and each member's results stay its own."""
    import paper_1905_07622_gb300 as hg
    ps = [_problem(), W.random_box(9, 30, 5, seed=22, flux={0: 1.0}, nsteps=2, rtol=1e-11),
          W.lognormal_cube(1, n=24, nsteps=2)]
    v = _loop_variants()[0]

    def batch():
        sims = [hg.Simulation.from_problem(p, precision="fp32_refined") for p in ps]
        try:
            b = hg.heat_batch_create([s.sim for s in sims])
            try:
                got = [[] for _ in ps]
                for _ in range(2):
                    rc, stats = hg.heat_batch_step(b, 1, len(ps))
                    assert rc == 0, hg.heat_last_error()
                    for k, s in enumerate(sims):
                        got[k].append(s.state())
                return got, [(st["iters"], st["outer"]) for st in stats]
            finally:
                hg.heat_destroy_batch(b)
        finally:
            for s in sims:
                s.close()

    _set("fp32_refined", v, 2, 0)
    tick, tick_its = batch()
    _set("fp32_refined", v, 2, 1)
    loop, loop_its = batch()
    assert loop_its == tick_its
    for k, p in enumerate(ps):
        alone, _ = _solve(p, "fp32_refined")
        for step in range(2):
            assert np.array_equal(loop[k][step], tick[k][step]), (k, step)
            assert np.array_equal(loop[k][step], alone[step]), (k, step)


def test_persistent_iteration_launches_two_kernels_per_tick():
    import paper_1905_07622_gb300 as hg
    p = _problem()
    v = _loop_variants()[0]
    counts = {}
    for loop in (0, 1):
        _set("fp32_refined", v, 2, loop)
        with hg.Simulation.from_problem(p, precision="fp32_refined") as s:
            st = s.step(3)
            assert st["status"] == 0
            counts[loop] = (st["kernel_launches"], st["iters"])
    # the tick form launches two kernels per iteration, the persistent form
    # two per tick (k_open and the loop) and polls alike
    assert counts[1][1] == counts[0][1]
    assert counts[1][0] < counts[0][0] / 2, counts


def test_a_barrier_wait_that_runs_out_fails_the_step_and_the_gpu_stays_usable():
    """The hook makes every barrier expect one arrival more than the grid
    has, so no wait can end by the barrier: each must end by its 20 ms bound,
    and the step must report HEAT_ERR_TIMEOUT. With the hook cleared the
    same simulation, restarted, solves correctly."""
    import paper_1905_07622_gb300 as hg
    p = _problem()
    v = _loop_variants()[0]
    _set("fp32_refined", v, 2, 1)
    hg.heat_debug_loop_wait(1, 0.02)
    with hg.Simulation.from_problem(p, precision="fp32_refined") as s:
        rc, st = hg.heat_step_nocheck(s.sim, 1)
        assert rc == hg.HEAT_ERR_TIMEOUT, (rc, hg.heat_last_error())
        assert st["status"] == hg.HEAT_ERR_TIMEOUT
        hg.heat_debug_loop_wait(0, 0.0)
        hg.heat_set_history(s.sim, p.u0, None, 0, p.n_nodes)
        us = []
        for _ in range(p.nsteps):
            assert s.step(1)["status"] == 0
            us.append(s.state())
    ref = pins.oracle_steps(p)
    for n in range(p.nsteps):
        err = np.linalg.norm(us[n] - ref.u[n + 1]) / np.linalg.norm(ref.u[n + 1])
        assert err <= 1e-8, (n, err)
