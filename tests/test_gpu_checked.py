"""The index-checked build (HEAT_CHECK) on the parity cases, and determinism.

No GPU sanitizer is available on the target machines; instead the library
is built a second time with every node and element index of the operator
kernels tested against the simulation's bounds (an out-of-range access is
skipped and counted). A child process loads that build and runs ragged,
tiny and Dirichlet meshes through every precision, every apply variant, a
batch and the inverse-problem driver; each simulation must end with zero
violations. The same runs repeated must give bitwise the same states.
"""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import numpy as np
    import paper_1905_07622_gb300 as hg
    import workloads as W
    assert hg.heat_checks_compiled()
    cases = [W.random_box(1, 1, 1, seed=1, nsteps=2, flux={5: 1.0}),
             W.random_box(33, 9, 17, seed=2, nsteps=2, dirichlet={0: 0.5, 5: 1.0}, flux={2: 1.0}),
             W.random_box(17, 31, 5, seed=3, nsteps=2, dirichlet={2: 0.0, 4: 1.0}),
             W.random_box(40, 6, 9, seed=4, nsteps=2, dirichlet={f: 0.1 * f for f in range(6)})]
    nv = hg.heat_tuning_num_variants()
    fails = []

    def run(p, precision):
        with hg.Simulation.from_problem(p, precision=precision) as s:
            s.step(p.nsteps)
            return s.state(), hg.heat_check_violations(s.sim)

    for p in cases:
        for precision in ("fp64", "fp32_refined", "fp32_plain"):
            pid = hg.PRECISIONS[precision]
            for v in [-1] + list(range(nv)):
                info = hg.heat_tuning_variant(v) if v >= 0 else None
                if info and precision == "fp64" and not info["has_fp64"]:
                    continue
                t = hg.heat_tuning_get()
                t["variant"][pid] = v
                t["seg_nodes"] = [256, 256, 256]
                hg.heat_tuning_set(t["variant"], t["seg_nodes"], t["pw_quads"])
                u1, c1 = run(p, precision)
                u2, c2 = run(p, precision)
                if c1 or c2:
                    fails.append(("violations", p.name, precision, v, c1, c2))
                if not np.array_equal(u1, u2):
                    fails.append(("nondeterministic", p.name, precision, v))
    # a batch of mixed sizes
    sims = [hg.Simulation.from_problem(p, precision="fp32_refined") for p in cases]
    b = hg.heat_batch_create([s.sim for s in sims])
    rc, _ = hg.heat_batch_step(b, 2, len(sims))
    hg.heat_destroy_batch(b)
    for s in sims:
        if hg.heat_check_violations(s.sim):
            fails.append(("batch violations", hg.heat_check_violations(s.sim)))
        s.close()
    assert rc == 0
    assert not fails, fails
    print("checked ok")
""")


def test_index_checked_build_has_no_violations_and_is_deterministic():
    import __graft_entry__
    b = __graft_entry__._build_module()
    lib = b.build(checked=True)
    env = dict(os.environ, HEATGB_LIBRARY=lib, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "checked ok" in r.stdout
