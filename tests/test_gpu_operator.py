"""GPU operator-level parity with the CPU oracle, through the C ABI.

Operator apply (FP64) must match the oracle's assembled CSR product to 1e-12
relative L2; the FP32 apply is reported against a looser bound; diagonal,
flux vector and step right-hand side match the oracle's assembled pieces.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, transient

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [
    ((1, 1, 1), {}),
    ((1, 7, 3), {2: 1.0}),
    ((17, 1, 5), {}),
    ((7, 5, 3), {0: 0.5, 5: -1.0}),
    ((33, 9, 17), {4: 1.0}),           # crosses the 32-wide tile, ragged in y and z
    ((40, 6, 9), {f: 0.1 * f for f in range(6)}),
]


def _sim(p, precision="fp64"):
    import paper_1905_07622_gb300 as hg
    return hg.Simulation.from_problem(p, precision=precision)


def _eliminated_apply(S, x):
    xf = np.zeros_like(x)
    xf[S.free] = x[S.free]
    y = S.A @ xf
    y[S.dir_ids] = x[S.dir_ids]
    return y


@pytest.mark.parametrize("dims,dirichlet", SHAPES)
def test_apply_fp64_matches_oracle_csr(dims, dirichlet):
    import paper_1905_07622_gb300 as hg
    p = W.random_box(*dims, seed=sum(dims), extent=(1.0, 0.7, 1.3), dirichlet=dirichlet,
                     theta=0.5, dt=0.003, contrast=(0.1, 10.0))
    S = transient.build_system(p)
    x = np.random.default_rng(1).standard_normal(p.n_nodes)
    ref = _eliminated_apply(S, x)
    with _sim(p) as s:
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        hg.heat_apply(s.sim, xd, yd)
        got = yd.cpu().numpy()
        # general (non-eliminated) products: M, K and L
        for sa, sb, mat in ((1.0, 0.0, S.M), (0.0, 1.0, S.K), (1 / p.dt, p.theta - 1, S.L)):
            hg.heat_apply_general(s.sim, sa, sb, xd, yd)
            g2 = yd.cpu().numpy()
            r2 = mat @ x
            assert np.linalg.norm(g2 - r2) <= 1e-12 * np.linalg.norm(r2)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("dims,dirichlet", SHAPES[2:5])
def test_apply_fp32_close_to_oracle(dims, dirichlet):
    import paper_1905_07622_gb300 as hg
    p = W.random_box(*dims, seed=7, dirichlet=dirichlet, theta=1.0, dt=0.01)
    S = transient.build_system(p)
    x = np.random.default_rng(2).standard_normal(p.n_nodes).astype(np.float32).astype(np.float64)
    ref = _eliminated_apply(S, x)
    with _sim(p) as s:
        xd = torch.tensor(x, device="cuda", dtype=torch.float32)
        yd = torch.empty_like(xd)
        hg.heat_apply_f32(s.sim, xd, yd)
        got = yd.double().cpu().numpy()
    # FP32 operator: error bounded by a few ulp of the largest partial sums
    assert np.linalg.norm(got - ref) <= 2e-6 * np.linalg.norm(ref)


@pytest.mark.parametrize("dims,dirichlet", SHAPES)
def test_diagonal_flux_and_rhs_match_oracle(dims, dirichlet):
    import paper_1905_07622_gb300 as hg
    p = W.random_box(*dims, seed=11, dirichlet=dirichlet, flux={5: 2.0, 2: -0.5, 0: 1.0},
                     flux_steps=1, theta=0.5, dt=0.02)
    S = transient.build_system(p)
    with _sim(p) as s:
        d = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
        hg.heat_diagonal(s.sim, d)
        diag = d.cpu().numpy()
        hg.heat_flux_vector(s.sim, d)
        flux = d.cpu().numpy()
        u = torch.tensor(p.u0, device="cuda")
        hg.heat_rhs(s.sim, 1, u, d)
        rhs1 = d.cpu().numpy()
        hg.heat_rhs(s.sim, 2, u, d)  # flux off after step 1
        rhs2 = d.cpu().numpy()
    ref_diag = np.ones(p.n_nodes)
    ref_diag[S.free] = S.A_ff.diagonal()
    assert np.abs(diag - ref_diag).max() <= 1e-13 * np.abs(ref_diag).max()
    Ff = S.F.copy()
    Ff[S.dir_ids] = 0.0
    assert np.abs(flux - Ff).max() <= 1e-14 * max(1.0, np.abs(S.F).max())
    for n, got in ((1, rhs1), (2, rhs2)):
        ref = np.empty(p.n_nodes)
        ref[S.free] = transient.step_rhs(p, S, p.u0, n)
        ref[S.dir_ids] = S.dir_vals
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_apply_symmetry_and_constant_vector():
    """x^T A y = y^T A x and A 1 = M 1 / dt (K 1 = 0) without Dirichlet faces."""
    import paper_1905_07622_gb300 as hg
    p = W.random_box(20, 13, 9, seed=5, theta=0.5, dt=0.004, contrast=(0.01, 100.0))
    S = transient.build_system(p)
    rng = np.random.default_rng(3)
    with _sim(p) as s:
        x = torch.tensor(rng.standard_normal(p.n_nodes), device="cuda")
        y = torch.tensor(rng.standard_normal(p.n_nodes), device="cuda")
        ax, ay = torch.empty_like(x), torch.empty_like(y)
        hg.heat_apply(s.sim, x, ax)
        hg.heat_apply(s.sim, y, ay)
        a = float(torch.dot(y, ax))
        b = float(torch.dot(x, ay))
        one = torch.ones_like(x)
        hg.heat_apply(s.sim, one, ax)
        got1 = ax.cpu().numpy()
    assert abs(a - b) <= 1e-12 * (abs(a) + abs(b))
    lumped = (S.M @ np.ones(p.n_nodes)) / p.dt
    assert np.abs(got1 - lumped).max() <= 1e-12 * np.abs(lumped).max()


@pytest.mark.parametrize("n", [100, 200])
def test_full_size_apply_sampled_rows(n):
    """Full-size meshes (1,030,301 and 8,120,601 nodes): sampled rows vs the oracle's row apply."""
    import paper_1905_07622_gb300 as hg
    p = W.inclusions_cube(n=100) if n == 100 else W.layered_cube(n=200)
    rng = np.random.default_rng(n)
    x = rng.standard_normal(p.n_nodes)
    rows = np.concatenate([rng.integers(0, p.n_nodes, 300), [0, p.n_nodes - 1, n, (n + 1) ** 2 * n // 2]])
    ref = fem.apply_rows(p, x, rows, 1.0 / p.dt, p.theta)
    with _sim(p) as s:
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        hg.heat_apply(s.sim, xd, yd)
        got = yd.cpu().numpy()[rows]
        x32 = xd.float()
        y32 = torch.empty_like(x32)
        hg.heat_apply_f32(s.sim, x32, y32)
        got32 = y32.double().cpu().numpy()[rows]
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(got32 - ref).max() <= 1e-5 * np.abs(ref).max()


def test_bad_coefficients_rejected_and_state_kept():
    import paper_1905_07622_gb300 as hg
    p = W.random_box(4, 4, 4, seed=1)
    with _sim(p) as s:
        d = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
        hg.heat_diagonal(s.sim, d)
        before = d.cpu().numpy()
        bad = p.k.copy()
        bad[5] = np.nan
        with pytest.raises(hg.HeatError) as e:
            hg.heat_set_coeffs(s.sim, p.rho_c, bad, p.n_elems)
        assert e.value.status == hg.HEAT_ERR_NONFINITE
        bad_dev = torch.tensor(p.k, device="cuda")
        bad_dev[3] = -1.0
        with pytest.raises(hg.HeatError):
            hg.heat_set_coeffs(s.sim, torch.tensor(p.rho_c, device="cuda"), bad_dev, p.n_elems)
        hg.heat_diagonal(s.sim, d)
        assert np.array_equal(before, d.cpu().numpy())
