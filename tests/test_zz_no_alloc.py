"""The allocation-free operator call (heat_apply_dot_noalloc) against heat_apply.

heat_apply_dot_noalloc serves callers that cannot allocate device memory
(allocation-free real-time loops, or a host memory manager that owns the
device and hands out only the buffers it was given): its reduction scratch is
a fixed device array inside the library. This test calls it through the C ABI twice
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


def _compare_two_calls(p, seed):
    import paper_1905_07622_gb300 as hg
    faces = sum(1 << f for f in p.dirichlet)
    rng = np.random.default_rng(seed)
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


def _tiles(nx, ny, nz):
    return -(-(nx + 1) // 32) * -(-(ny + 1) // 4) * -(-(nz + 1) // 8)


def test_noalloc_apply_dot_matches_heat_apply_on_two_calls():
    p = W.random_box(33, 9, 17, seed=41, extent=(1.0, 0.7, 1.3), dirichlet={4: 1.0, 1: -0.5},
                     theta=0.5, dt=0.003, contrast=(0.1, 10.0))
    _compare_two_calls(p, 5)


def test_noalloc_grid_stride_and_largest_mesh():
    """More tiles than blocks (each block loops over several tiles and reuses
    its shared state), and a mesh of exactly HEAT_NOALLOC_MAX_TILES tiles."""
    assert _tiles(159, 159, 159) == 4000 and _tiles(31, 255, 511) == 4096
    _compare_two_calls(W.random_box(159, 159, 159, seed=42, dirichlet={0: 0.5}, theta=0.5, dt=0.01), 6)
    _compare_two_calls(W.random_box(31, 255, 511, seed=43, flux={5: 1.0}, theta=1.0, dt=0.02), 7)


def test_noalloc_rejects_meshes_beyond_its_scratch():
    import paper_1905_07622_gb300 as hg
    nx, ny, nz = 543, 963, 7
    assert _tiles(nx, ny, nz) == 4097
    nn = (nx + 1) * (ny + 1) * (nz + 1)
    coef = torch.zeros(2 * nx * ny * nz, dtype=torch.float64, device="cuda")
    x = torch.zeros(nn, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    dot = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(hg.HeatError) as e:
        hg.heat_apply_dot_noalloc(nx, ny, nz, (1.0, 1.0, 1.0), 1e-3, 0.5, 0, coef, x, y, dot)
    assert e.value.status == hg.HEAT_ERR_ARG
    assert "static" in str(e.value)
