"""The request server: continuous batching, footprint admission, bounded waits.

Requests are submitted while others are running; each result must be bitwise
identical to the same simulation stepped alone (its reductions do not depend
on what shares the launches) and match the oracle within the refined path's
1e-8 tolerance. The stopping rule bounds the preconditioned residual, and the
field error can exceed it by up to the condition number, so the parity
requests are solved to rtol 1e-10 (the serving workload's own 1e-8 is a
residual tolerance, not a field one).
"""
import time

import numpy as np
import pytest

import pins
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GB = 1 << 30


def _alone(p, precision="fp32_refined"):
    import paper_1905_07622_gb300 as hg
    with hg.Simulation.from_problem(p, precision=precision) as s:
        s.step(p.nsteps)
        return s.state()


def _requests():
    ps = [W.serving_request(r, n_min=8, n_max=24) for r in range(6)]
    for p in ps:
        p.rtol = 1e-10
    return ps


def test_staggered_requests_equal_alone_and_oracle():
    import paper_1905_07622_gb300 as hg
    ps = _requests()
    for p in ps:
        p.nsteps = min(p.nsteps, 12)
    srv = hg.heat_server_create(4 * GB, 8)
    try:
        tickets = []
        for i, p in enumerate(ps):
            req, keep = hg.make_request(p)
            tickets.append(hg.heat_submit(srv, req))
            if i == 2:
                time.sleep(0.05)  # the rest arrive while the first ones run
        results = [hg.heat_wait(srv, t, p.n_nodes, timeout_s=300.0) for t, p in zip(tickets, ps)]
        stats = hg.heat_server_get_stats(srv)
    finally:
        hg.heat_destroy_server(srv)
    assert stats["completed"] == len(ps) and stats["failed"] == 0
    assert stats["kernel_launches"] > 0
    for p, (u, st, lat) in zip(ps, results):
        assert st["steps"] == p.nsteps and lat > 0.0
        assert np.array_equal(u, _alone(p))
        ref = pins.oracle_steps(p)
        assert np.linalg.norm(u - ref.u[-1]) <= 1e-8 * np.linalg.norm(ref.u[-1])


def test_small_budget_admits_few_at_a_time():
    import paper_1905_07622_gb300 as hg
    ps = [W.random_box(10, 10, 10, seed=s, flux={5: 1.0}, nsteps=5, rtol=1e-10) for s in range(4)]
    # a 10^3 simulation holds ~205 KB (120 B per node, 24 B per element, work
    # lists): room for two at a time, not three
    budget = 450_000
    srv = hg.heat_server_create(budget, 8)
    try:
        reqs = [hg.make_request(p) for p in ps]
        tickets = [hg.heat_submit(srv, r) for r, _ in reqs]
        peak = 0
        while not all(hg.heat_poll(srv, t) for t in tickets):
            st = hg.heat_server_get_stats(srv)
            assert st["hbm_in_use"] <= st["hbm_budget"]
            peak = max(peak, st["active"])
            time.sleep(0.001)
        assert 1 <= peak <= 2
        for t, p in zip(tickets, ps):
            u, _, _ = hg.heat_wait(srv, t, p.n_nodes, timeout_s=60.0)
            assert np.array_equal(u, _alone(p))
    finally:
        hg.heat_destroy_server(srv)


def test_rejections_and_bounded_wait():
    import paper_1905_07622_gb300 as hg
    srv = hg.heat_server_create(64 << 20, 2)
    try:
        big = W.random_box(100, 100, 100, seed=1, nsteps=1)  # ~150 MB > 64 MB budget
        req, keep = hg.make_request(big)
        with pytest.raises(hg.HeatError) as e:
            hg.heat_submit(srv, req)
        assert e.value.status == hg.HEAT_ERR_NOMEM
        bad = W.random_box(4, 4, 4, seed=2, nsteps=1)
        bad.k[3] = np.inf
        req, keep = hg.make_request(bad)
        with pytest.raises(hg.HeatError) as e:
            hg.heat_submit(srv, req)
        assert e.value.status == hg.HEAT_ERR_NONFINITE
        slow = W.random_box(30, 30, 30, seed=3, flux={5: 1.0}, nsteps=200, rtol=1e-10)
        req, keep = hg.make_request(slow)
        t = hg.heat_submit(srv, req)
        with pytest.raises(hg.HeatError) as e:
            hg.heat_wait(srv, t, slow.n_nodes, timeout_s=0.0)
        assert e.value.status == hg.HEAT_ERR_TIMEOUT
    finally:
        hg.heat_destroy_server(srv)  # abandons the running request without hanging


def test_admission_that_cannot_be_built_leaves_running_requests_unchanged():
    """A request admitted while another runs, whose member set cannot be
    built (a failed device allocation, injected on the host), is refused;
    the running request finishes bitwise as it would alone, and the next
    request is served normally."""
    import paper_1905_07622_gb300 as hg
    p_long = W.random_box(16, 16, 16, seed=31, flux={5: 1.0}, nsteps=600, rtol=1e-10)
    p_new = W.random_box(10, 10, 10, seed=32, flux={5: 1.0}, nsteps=5, rtol=1e-10)
    srv = hg.heat_server_create(4 * GB, 8)
    try:
        r1, k1 = hg.make_request(p_long, precision="fp32_refined")
        t1 = hg.heat_submit(srv, r1)
        t0 = time.time()
        while hg.heat_server_get_stats(srv)["active"] < 1:
            assert time.time() - t0 < 60
            time.sleep(0.001)
        hg.heat_debug_fail_engine_builds(1)
        r2, k2 = hg.make_request(p_new, precision="fp32_refined")
        t2 = hg.heat_submit(srv, r2)
        with pytest.raises(hg.HeatError) as e:
            hg.heat_wait(srv, t2, p_new.n_nodes, timeout_s=120.0)
        assert e.value.status == hg.HEAT_ERR_NOMEM
        still_running = not hg.heat_poll(srv, t1)
        u1, st1, _ = hg.heat_wait(srv, t1, p_long.n_nodes, timeout_s=300.0)
        r3, k3 = hg.make_request(p_new, precision="fp32_refined")
        t3 = hg.heat_submit(srv, r3)
        u3, _, _ = hg.heat_wait(srv, t3, p_new.n_nodes, timeout_s=120.0)
        stats = hg.heat_server_get_stats(srv)
    finally:
        hg.heat_debug_fail_engine_builds(0)
        hg.heat_destroy_server(srv)
    assert still_running  # the refusal happened while the long request ran
    assert st1["steps"] == p_long.nsteps
    assert np.array_equal(u1, _alone(p_long))
    assert np.array_equal(u3, _alone(p_new))
    assert stats["failed"] == 1 and stats["completed"] == 2
