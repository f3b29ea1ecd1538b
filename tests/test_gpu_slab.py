"""One simulation split into z-slabs (heat_slab_*, the partitioned form of
§4.4's dual-GPU split) against the oracle and against the unsplit solve.

The slab form solves the same step systems (§3.1) with the same stopping rule
(Algorithm 1 with the relative reading), so each step's field must match the
oracle's exact step solution within the FP64 parity bar of the transient
tests (1e-9 relative L2 at rtol 1e-12), for every slab count from one slab to
one owned node layer per slab, in both iteration forms. Slab counts that leave
ragged tiles and single-layer slabs are included.
"""
import numpy as np
import pytest

import workloads as W
from oracle import transient

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _run_slab(p, nslabs, merged, nsteps=None, **kw):
    import paper_1905_07622_gb300 as hg
    us, stats, its = [], [], []
    with hg.SlabSimulation.from_problem(p, nslabs, merged=merged, **kw) as s:
        us.append(s.state())
        for _ in range(nsteps or p.nsteps):
            stats.append(s.step(1))
            its += s.iterations()
            us.append(s.state())
    return us, stats, its


CASES = [
    ((6, 5, 7), {0: 0.5}, {5: 1.0}, 0.5),
    ((9, 4, 12), {4: 1.0, 3: -0.25}, {2: 0.7}, 1.0),
    ((17, 16, 5), {}, {5: 1.0, 0: -0.3}, 0.5),
    ((3, 3, 2), {5: 2.0}, {1: 1.0}, 0.7),
]


@pytest.mark.parametrize("case", range(len(CASES)))
@pytest.mark.parametrize("merged", [True, False])
def test_slab_steps_match_oracle_for_every_slab_count(case, merged):
    dims, dirichlet, flux, theta = CASES[case]
    p = W.random_box(*dims, seed=11 + case, dirichlet=dirichlet, flux=flux, theta=theta, dt=0.01,
                     nsteps=3, flux_steps=2, rtol=1e-12, contrast=(0.2, 5.0))
    ref = transient.run(p, solver="direct")
    nz = dims[2]
    counts = sorted({1, 2, 3, nz, nz + 1})
    for ns in counts:
        us, stats, _ = _run_slab(p, ns, merged)
        for n in range(1, p.nsteps + 1):
            err = _rel(us[n], ref.u[n])
            assert err <= 1e-9, (dims, ns, merged, n, err)
        assert all(st["status"] == 0 for st in stats)


def test_slab_matches_unsplit_gpu_solve_and_iteration_counts():
    import paper_1905_07622_gb300 as hg
    p = W.random_box(20, 18, 24, seed=5, dirichlet={4: 1.0}, flux={5: 1.0}, theta=0.5, dt=0.005,
                     nsteps=4, rtol=1e-10, contrast=(0.1, 10.0))
    with hg.Simulation.from_problem(p, precision="fp64") as s:
        whole = []
        its_whole = []
        for _ in range(p.nsteps):
            st = s.step(1)
            its_whole.append(st["iters"])
            whole.append(s.state())
    for merged in (True, False):
        for ns in (1, 4, 7):
            us, _, its = _run_slab(p, ns, merged)
            for n in range(p.nsteps):
                assert _rel(us[n + 1], whole[n]) <= 1e-9, (merged, ns, n)
            # Algorithm 1 is the unsplit path's iteration; the merged form is the
            # same method in exact arithmetic
            assert all(abs(a - b) <= 3 for a, b in zip(its, its_whole)), (merged, ns, its, its_whole)


def test_slab_on_layered_contrast_matches_oracle():
    """The 1:1000 layers and k = 0.01 pockets of the 200^3 workload at 32^3,
    split in 4 slabs."""
    p = W.layered_cube(n=32, nsteps=3)
    ref = transient.run(p, solver="pcg", rtol=1e-13)
    for merged in (True, False):
        us, stats, _ = _run_slab(p, 4, merged)
        errs = [_rel(us[n], ref.u[n]) for n in range(1, p.nsteps + 1)]
        assert max(errs) <= 1e-9, (merged, errs)


def test_slab_results_are_deterministic():
    p = W.random_box(12, 11, 19, seed=8, dirichlet={0: 0.0}, flux={5: 1.0}, nsteps=3, rtol=1e-11)
    a, _, ia = _run_slab(p, 5, True)
    b, _, ib = _run_slab(p, 5, True)
    assert ia == ib
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


def test_slab_failure_keeps_last_good_step():
    import paper_1905_07622_gb300 as hg
    p = W.random_box(10, 10, 10, seed=3, flux={5: 1.0}, nsteps=2, rtol=1e-12)
    with hg.SlabSimulation.from_problem(p, 3, max_iter=2) as s:
        u0 = s.state()
        with pytest.raises(hg.HeatError) as e:
            s.step(1)
        assert e.value.status == hg.HEAT_ERR_NOT_CONVERGED
        assert np.array_equal(s.state(), u0)


def test_slab_rejects_unsupported_settings():
    import paper_1905_07622_gb300 as hg
    p = W.random_box(4, 4, 4, seed=1)
    for kw in ({"precision": "fp32_refined"}, {"cheb_degree": 2}):
        with pytest.raises(hg.HeatError) as e:
            hg.SlabSimulation.from_problem(p, 2, **kw)
        assert e.value.status == hg.HEAT_ERR_ARG
    with pytest.raises(hg.HeatError):
        hg.SlabSimulation.from_problem(p, 6)  # more slabs than node layers
