"""The highest-contrast workload, reduced to a size the oracle solves: the
layered cube's recipe (20 layers with k alternating 1 / 1000, 30 ellipsoidal
pockets with k = 0.01 and rho_c = 0.5, Dirichlet u = 1 on z = 0, dt = 5e-4,
theta = 0.5, rtol 1e-10) on 40^3 elements, every step compared with the
oracle's exact step solution.

The exact solution is the oracle's Algorithm 1 run to rtol 1e-13 (pinned
against sparse LU on this recipe at 24^3 by the oracle tests; LU itself takes
over a minute at 40^3). The bars are the parity bars of the transient tests:
relative L2 field error per step <= 1e-9 on the FP64 path and <= 1e-8 on the
refined path, whose outer residual is formed in double-float arithmetic.
The field error may exceed the residual tolerance by up to kappa(P^-1 A);
the test reports the Lanczos estimate of kappa from the oracle's own CG
coefficients beside each error.
"""
import numpy as np
import pytest

import workloads as W
from oracle import pcg, transient

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NSTEPS = 4


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def layered40():
    p = W.layered_cube(n=40, nsteps=NSTEPS)
    S = transient.build_system(p)
    ref = transient.run(p, solver="pcg", rtol=1e-13, system=S)
    # kappa(P^-1 A) of the step matrix (the same every step), from one solve
    b = transient.step_rhs(p, S, ref.u[0], 1)
    rec = []
    pcg.pcg(S.A_ff, b, np.zeros_like(b), S.pinv_f, 1e-13, record=rec)
    lo, hi = pcg.lanczos_extremes(rec)
    return p, ref, hi / lo


def _run_gpu(p, precision, **kw):
    import paper_1905_07622_gb300 as hg
    us, stats = [], []
    with hg.Simulation.from_problem(p, precision=precision, **kw) as s:
        us.append(s.state())
        for _ in range(p.nsteps):
            st = s.step(1)
            assert st["status"] == 0, st
            stats.append(st)
            us.append(s.state())
    return us, stats


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32_refined", 1e-8)])
def test_layered_40_every_step_matches_oracle(layered40, precision, tol):
    p, ref, kappa = layered40
    us, stats = _run_gpu(p, precision)
    errs = [_rel(us[n], ref.u[n]) for n in range(1, p.nsteps + 1)]
    print(f"layered 40^3 {precision}: kappa(P^-1 A) ~ {kappa:.3e}; per-step field error "
          + ", ".join(f"{e:.2e}" for e in errs) + "; iterations " + str([st["iters"] for st in stats]))
    assert max(errs) <= tol, errs
    # Dirichlet face exactly at 1
    dn = np.arange((p.nx + 1) * (p.ny + 1))
    assert np.all(us[-1][dn] == 1.0)


def test_layered_40_chebyshev_refined_matches_oracle(layered40):
    p, ref, _ = layered40
    us, _ = _run_gpu(p, "fp32_refined", cheb_degree=2)
    errs = [_rel(us[n], ref.u[n]) for n in range(1, p.nsteps + 1)]
    assert max(errs) <= 1e-8, errs
