"""Pins of the oracle's whole-mesh operator, diagonal and condition estimate (no GPU).

* fem.apply_all (Eq. 1 as an element-by-element product) equals the assembled
  CSR operator of transient.build_system, which the closed-form pins fix, on
  anisotropic boxes with and without Dirichlet elimination; A.1 = M.1/dt is
  the closed form 1^T K = 0 on its own.
* fem.diagonal_all equals the assembled diagonal and the closed form
  P_i = sum_{e ni i} (rho_c_e h^3/(27 dt) + theta k_e h/3) on cubes.
* pcg.lanczos_extremes reproduces the extreme eigenvalues of P^-1/2 A P^-1/2
  computed densely.
* Oracle PCG at rtol 1e-13 equals sparse LU on a layered cube with the
  1:1000 layers and k = 0.01 pockets of the 200^3 workload, so the GPU tests
  may use it as the exact step solution where LU is too slow.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem, pcg, transient


@pytest.mark.parametrize("dims,extent,dirichlet", [
    ((5, 4, 6), (1.0, 0.5, 2.0), {0: 1.0, 5: -0.5}),
    ((3, 7, 2), (0.3, 1.0, 1.0), {}),
    ((6, 2, 9), (1.0, 1.0, 1.0), {2: 0.25, 3: 1.0, 4: 2.0}),
])
def test_apply_all_equals_assembled_operator(dims, extent, dirichlet):
    p = W.random_box(*dims, seed=7, extent=extent, dirichlet=dirichlet, theta=0.7, dt=0.03)
    S = transient.build_system(p)
    x = np.random.default_rng(11).standard_normal(p.n_nodes)
    for sa, sb, Mx in ((1 / p.dt, p.theta, S.A), (1 / p.dt, p.theta - 1.0, S.L)):
        y = fem.apply_all(p, x, sa, sb, eliminate=False, layers=2)
        ref = Mx @ x
        assert np.linalg.norm(y - ref) <= 1e-14 * np.linalg.norm(ref)
    y = fem.apply_all(p, x, 1 / p.dt, p.theta, eliminate=True, layers=3)
    ref = np.array(x)
    ref[S.free] = S.A_ff @ x[S.free]
    assert np.linalg.norm(y - ref) <= 1e-14 * np.linalg.norm(ref)


def test_apply_all_of_ones_is_the_lumped_mass():
    p = W.random_box(4, 5, 3, seed=2, extent=(2.0, 1.0, 0.5))
    y = fem.apply_all(p, np.ones(p.n_nodes), 1.0, 123.0, eliminate=False)
    vol = np.prod(p.extent) / p.n_elems
    conn = fem.connectivity(p.nx, p.ny, p.nz)
    lumped = np.bincount(conn.ravel(), weights=np.repeat(p.rho_c * vol / 8.0, 8), minlength=p.n_nodes)
    # rounding of the K part (weight 123): its row entries are summed to zero
    assert np.abs(y - lumped).max() <= 1e-13 * 123.0 * p.k.max()


def test_diagonal_all_matches_assembly_and_closed_form():
    p = W.random_box(6, 6, 6, seed=5, dirichlet={1: 0.0}, theta=0.5, dt=0.02)
    S = transient.build_system(p)
    d = fem.diagonal_all(p, 1 / p.dt, p.theta)
    assert np.abs(d[S.free] * S.pinv_f - 1.0).max() <= 1e-14
    assert np.all(d[S.dir_ids] == 1.0)
    h = 1.0 / 6
    conn = fem.connectivity(6, 6, 6)
    per = p.rho_c * h ** 3 / (27 * p.dt) + p.theta * p.k * h / 3
    closed = np.bincount(conn.ravel(), weights=np.repeat(per, 8), minlength=p.n_nodes)
    assert np.abs(d[S.free] - closed[S.free]).max() <= 1e-13 * closed.max()


def test_lanczos_extremes_match_dense_eigenvalues():
    p = W.random_box(4, 3, 5, seed=9, dirichlet={4: 0.0}, contrast=(0.1, 10.0), dt=0.05)
    S = transient.build_system(p)
    b = np.random.default_rng(3).standard_normal(S.free.size)
    rec = []
    pcg.pcg(S.A_ff, b, np.zeros_like(b), S.pinv_f, 1e-14, record=rec)
    lo, hi = pcg.lanczos_extremes(rec)
    sq = np.sqrt(S.pinv_f)
    ev = np.linalg.eigvalsh(S.A_ff.toarray() * sq[:, None] * sq[None, :])
    # the smallest Ritz value converges last (29 iterations here)
    assert abs(lo - ev[0]) <= 1e-4 * ev[0]
    assert abs(hi - ev[-1]) <= 1e-9 * ev[-1]
    # Ritz values lie inside the spectrum
    assert lo >= ev[0] * (1 - 1e-12) and hi <= ev[-1] * (1 + 1e-12)


def test_tight_pcg_equals_lu_on_high_contrast_layers():
    p = W.layered_cube(n=24, nsteps=2)
    S = transient.build_system(p)
    lu = transient.run(p, solver="direct", system=S)
    it = transient.run(p, solver="pcg", rtol=1e-13, system=S)
    for n in (1, 2):
        err = np.linalg.norm(it.u[n] - lu.u[n]) / np.linalg.norm(lu.u[n])
        assert err <= 1e-11, (n, err)


def test_pins_catch_planted_mistakes():
    """A dropped beta/alpha term in the Lanczos diagonal, or an apply that
    skips the last element layer of a chunk, fails the pins above."""
    import scipy.linalg as sla
    p = W.random_box(4, 3, 5, seed=9, dirichlet={4: 0.0}, contrast=(0.1, 10.0), dt=0.05)
    S = transient.build_system(p)
    b = np.random.default_rng(3).standard_normal(S.free.size)
    rec = []
    pcg.pcg(S.A_ff, b, np.zeros_like(b), S.pinv_f, 1e-14, record=rec)
    al = np.array([c[0] for c in rec])
    be = np.array([c[1] for c in rec])
    ev_bad = sla.eigh_tridiagonal(1.0 / al, np.sqrt(be[:-1]) / al[:-1], eigvals_only=True)
    sq = np.sqrt(S.pinv_f)
    ev = np.linalg.eigvalsh(S.A_ff.toarray() * sq[:, None] * sq[None, :])
    assert abs(ev_bad[-1] - ev[-1]) > 1e-3 * ev[-1]

    x = np.random.default_rng(2).standard_normal(p.n_nodes)
    orig = fem._layer_connectivity
    try:
        fem._layer_connectivity = lambda nx, ny, k0, k1: orig(nx, ny, k0, max(k0 + 1, k1 - 1))
        with pytest.raises(Exception):
            bad = fem.apply_all(p, x, 1 / p.dt, p.theta, eliminate=False, layers=2)
            ref = S.A @ x
            assert np.linalg.norm(bad - ref) <= 1e-14 * np.linalg.norm(ref)
    finally:
        fem._layer_connectivity = orig


@pytest.mark.parametrize("dims,extent", [((5, 4, 6), (1.0, 0.5, 2.0)), ((3, 7, 2), (0.3, 1.0, 1.0)),
                                         ((8, 8, 8), (1.0, 1.0, 1.0))])
def test_stencil_assembly_equals_coo_assembly(dims, extent):
    p = W.random_box(*dims, seed=13, extent=extent, contrast=(0.01, 100.0))
    M = fem.assemble(p.nx, p.ny, p.nz, p.extent, p.rho_c, "M")
    K = fem.assemble(p.nx, p.ny, p.nz, p.extent, p.k, "K")
    for sa, sb in ((1.0, 0.0), (0.0, 1.0), (1 / 0.003, 0.5), (1 / 0.003, -0.5)):
        A = (sa * M + sb * K).tocsr()
        B = fem.assemble_stencil(p, sa, sb, layers=3)
        assert abs(A - B).max() <= 1e-14 * abs(A).max()
