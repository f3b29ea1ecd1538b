"""The allocation-free operator call (heat_apply_dot_noalloc) against heat_apply.

heat_apply_dot_noalloc serves callers that cannot allocate device memory
(during CUDA graph capture, in allocation-free real-time loops, or under a
host memory manager that owns the device): its reduction scratch is a fixed
device array inside the library. This test calls it through the C ABI twice
in a row (the second call reuses the scratch the first left behind) and
compares its y = A' x with heat_apply's, and its x.A'x with the dot product
of x and heat_apply's y, at the 1e-12 relative tolerance of the FP64
operator tests. The file is named to run last so that a failing run stops
after every other test has run.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_noalloc_apply_dot_matches_heat_apply_on_two_calls():
    import paper_1905_07622_gb300 as hg
    p = W.random_box(33, 9, 17, seed=41, extent=(1.0, 0.7, 1.3), dirichlet={4: 1.0, 1: -0.5},
                     theta=0.5, dt=0.003, contrast=(0.1, 10.0))
    faces = sum(1 << f for f in p.dirichlet)
    rng = np.random.default_rng(5)
    coef = torch.tensor(np.stack([p.rho_c, p.k], axis=1).ravel(), device="cuda")
    with hg.Simulation.from_problem(p) as s:
        for call in range(2):
            x = torch.tensor(rng.standard_normal(p.n_nodes), device="cuda")
            y_ref = torch.empty_like(x)
            hg.heat_apply(s.sim, x, y_ref)
            y = torch.full_like(x, np.nan)
            xdoty = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
            hg.heat_apply_dot_noalloc(p.nx, p.ny, p.nz, p.extent, p.dt, p.theta, faces, coef, x, y, xdoty)
            torch.cuda.synchronize()
            ref = y_ref.cpu().numpy()
            got = y.cpu().numpy()
            assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref), call
            dot_ref = float(np.dot(x.cpu().numpy(), ref))
            assert abs(float(xdoty.item()) - dot_ref) <= 1e-12 * abs(dot_ref), call


def test_noalloc_rejects_meshes_beyond_its_scratch():
    import paper_1905_07622_gb300 as hg
    dummy = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(hg.HeatError) as e:
        hg.heat_apply_dot_noalloc(200, 200, 200, (1.0, 1.0, 1.0), 1e-3, 0.5, 0, dummy, dummy, dummy, dummy)
    assert e.value.status == hg.HEAT_ERR_ARG
    assert "static" in str(e.value)
