"""Kernel tuning: every apply variant and segment size against the oracle
(trilinear and six-tetrahedra boxes), bitwise batch equality under a
non-default table, and the autotuner.

The tuning table picks which warp-segment apply kernel runs and how large
its tiles are; every choice must give the same step solutions (within the
path's tolerance) as the oracle, and a member of a batch must still match
itself run alone when both are built under the same table.
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
    hg.heat_tuning_set(old["variant"], old["seg_nodes"], old["pw_quads"], old["open_w"], old["loop"])


def _problem():
    # ragged in every direction against 16- and 32-wide segments
    return W.random_box(37, 11, 19, seed=21, dirichlet={2: 0.5}, flux={5: 1.0}, theta=0.5, dt=0.01, nsteps=2,
                        rtol=1e-11, contrast=(0.1, 10.0))


def _solve(p, precision):
    import paper_1905_07622_gb300 as hg
    with hg.Simulation.from_problem(p, precision=precision) as s:
        out = []
        for _ in range(p.nsteps):
            s.step(1)
            out.append(s.state())
        return out


def _variants(fp64):
    import paper_1905_07622_gb300 as hg
    vs = [-1]
    for v in range(hg.heat_tuning_num_variants()):
        if not fp64 or hg.heat_tuning_variant(v)["has_fp64"]:
            vs.append(v)
    return vs


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32_refined", 1e-8)])
def test_every_variant_and_segment_size_matches_oracle(precision, tol):
    import paper_1905_07622_gb300 as hg
    p = _problem()
    ref = pins.oracle_steps(p)
    pid = hg.PRECISIONS[precision]
    cases = [(v, seg, None) for v in _variants(precision == "fp64") for seg in ([512] if v < 0 else [64, 256, 2048])]
    cases += [(-1, 512, 1), (-1, 512, 2), (-1, 512, 4)]  # every pointwise item size
    for v, seg, quads in cases:
        table = hg.heat_tuning_get()
        table["variant"][pid] = v
        table["seg_nodes"][0] = seg
        if quads:
            table["pw_quads"][pid] = quads
        hg.heat_tuning_set(table["variant"], table["seg_nodes"], table["pw_quads"])
        us = _solve(p, precision)
        for n in range(1, p.nsteps + 1):
            err = np.linalg.norm(us[n - 1] - ref.u[n]) / np.linalg.norm(ref.u[n])
            assert err <= tol, (v, seg, quads, n, err)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32_refined", 1e-8)])
def test_every_variant_on_six_tetrahedra_boxes(precision, tol):
    """The box-centred P1 march under every load policy (register prefetch,
    cp.async ring, the fused iteration) and the P1 block tiles."""
    import paper_1905_07622_gb300 as hg
    p = _problem()
    p.element = "p1"
    ref = pins.oracle_steps(p)
    pid = hg.PRECISIONS[precision]
    for v in _variants(precision == "fp64"):
        for seg in ([512] if v < 0 else [64, 2048]):
            table = hg.heat_tuning_get()
            table["variant"][pid] = v
            table["seg_nodes"][0] = seg
            hg.heat_tuning_set(table["variant"], table["seg_nodes"], table["pw_quads"])
            us = _solve(p, precision)
            for n in range(1, p.nsteps + 1):
                err = np.linalg.norm(us[n - 1] - ref.u[n]) / np.linalg.norm(ref.u[n])
                assert err <= tol, (v, seg, n, err)


def test_batch_bitwise_equal_to_alone_under_a_tuned_table():
    import paper_1905_07622_gb300 as hg
    n = hg.heat_tuning_num_variants()
    info = [hg.heat_tuning_variant(v) for v in range(n)]
    v64 = max(v for v in range(n) if info[v]["has_fp64"])
    v32 = next((v for v in range(n) if info[v]["stages"] > 0), n - 1)  # a cp.async-staged kernel if any
    hg.heat_tuning_set([v64, v32, 0], [256, 1024, 512])
    ps = [_problem(), W.random_box(9, 30, 5, seed=22, flux={0: 1.0}, nsteps=2, rtol=1e-11),
          W.lognormal_cube(1, n=24, nsteps=2)]
    for precision in ("fp64", "fp32_refined"):
        sims = [hg.Simulation.from_problem(p, precision=precision) for p in ps]
        try:
            b = hg.heat_batch_create([s.sim for s in sims])
            try:
                got = [[] for _ in ps]
                for _ in range(2):
                    rc, stats = hg.heat_batch_step(b, 1, len(ps))
                    assert rc == 0, hg.heat_last_error()
                    for k, s in enumerate(sims):
                        got[k].append(s.state())
            finally:
                hg.heat_destroy_batch(b)
        finally:
            for s in sims:
                s.close()
        for k, p in enumerate(ps):
            alone = _solve(p, precision)
            for step in range(2):
                assert np.array_equal(got[k][step], alone[step]), (precision, k, step)


@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_autotune_picks_a_valid_entry_and_keeps_parity(precision):
    import paper_1905_07622_gb300 as hg
    p = W.lognormal_cube(2, n=32, nsteps=2)
    p.rtol = 1e-11
    pid = hg.PRECISIONS[precision]
    before = hg.heat_tuning_get()
    with hg.Simulation.from_problem(p, precision=precision) as s:
        s.step(1)
        table, ms = hg.heat_autotune(s.sim, 5)
        assert ms > 0.0
        assert table == hg.heat_tuning_get()
        v = table["variant"][pid]
        assert v == -1 or (0 <= v < hg.heat_tuning_num_variants())
        if v >= 0 and precision == "fp64":
            assert hg.heat_tuning_variant(v)["has_fp64"]
        seg = table["seg_nodes"][0]
        if seg not in (256, 512, 1024, 2048):  # a wave-aligned size: whole levels of the chosen segment tile
            assert v >= 0, seg
            shape = hg.heat_tuning_variant(v)
            assert seg % ((shape["seg_width"] - 2) * shape["rows"]) == 0, (v, seg)
        # entries of the other precisions and size buckets are untouched
        for q in range(3):
            if q != pid:
                assert table["variant"][q] == before["variant"][q]
        assert table["seg_nodes"][1:] == before["seg_nodes"][1:]
        # the solver state is undefined after tuning: restart from u0
        hg.heat_set_history(s.sim, p.u0, None, 0, p.n_nodes)
        s.step(2)
        got = s.state()
    ref = pins.oracle_steps(p)
    err = np.linalg.norm(got - ref.u[2]) / np.linalg.norm(ref.u[2])
    assert err <= (1e-9 if precision == "fp64" else 1e-8), err


def test_batch_autotune_rebuilds_and_keeps_parity():
    import paper_1905_07622_gb300 as hg
    ps = [W.lognormal_cube(s, n=16, nsteps=2) for s in range(3)]
    for p in ps:
        p.rtol = 1e-11
    sims = [hg.Simulation.from_problem(p, precision="fp32_refined") for p in ps]
    try:
        b = hg.heat_batch_create([s.sim for s in sims])
        try:
            rc, _ = hg.heat_batch_step(b, 1, len(ps))
            assert rc == 0
            table, ms = hg.heat_batch_autotune(b, 8)
            assert ms > 0.0 and table == hg.heat_tuning_get()
            for s, p in zip(sims, ps):
                hg.heat_set_history(s.sim, p.u0, None, 0, p.n_nodes)
            rc, stats = hg.heat_batch_step(b, 2, len(ps))
            assert rc == 0, hg.heat_last_error()
            got = [s.state() for s in sims]
        finally:
            hg.heat_destroy_batch(b)
    finally:
        for s in sims:
            s.close()
    for g, p in zip(got, ps):
        ref = pins.oracle_steps(p)
        assert np.linalg.norm(g - ref.u[2]) <= 1e-8 * np.linalg.norm(ref.u[2])


@pytest.mark.parametrize("shape", [1, 2])
@pytest.mark.parametrize("precision", ["fp64", "fp32_refined"])
def test_warp_segment_open_passes_match_block_tiles_and_oracle(precision, shape):
    """The step-start and refinement passes in the warp-segment march
    (tuning open_w = 1) give the block-tile passes' fields and the oracle's."""
    import paper_1905_07622_gb300 as hg
    from oracle import transient
    p = W.random_box(37, 9, 14, seed=19, dirichlet={4: 1.0, 1: -0.5}, flux={5: 1.0}, theta=0.5, dt=0.01,
                     nsteps=4, flux_steps=2, rtol=1e-12, contrast=(0.1, 10.0))
    ref = transient.run(p, solver="direct")
    old = hg.heat_tuning_get()
    fields = {}
    try:
        for ow in (0, shape):
            hg.heat_tuning_set(old["variant"], old["seg_nodes"], old["pw_quads"], [ow, ow, ow])
            with hg.Simulation.from_problem(p, precision=precision) as s:
                us = []
                for _ in range(p.nsteps):
                    assert s.step(1)["status"] == 0
                    us.append(s.state())
            fields[ow] = us
    finally:
        hg.heat_tuning_set(old["variant"], old["seg_nodes"], old["pw_quads"], old["open_w"])
    tol = 1e-9 if precision == "fp64" else 1e-8
    for n in range(p.nsteps):
        a, b = fields[0][n], fields[shape][n]
        assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a), n
        assert np.linalg.norm(b - ref.u[n + 1]) <= tol * np.linalg.norm(ref.u[n + 1]), n
