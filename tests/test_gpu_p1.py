"""Six-tetrahedra boxes (§4.1's element) on the GPU against the oracle.

- operator entry points: the eliminated apply and the general products
  (M, K, L) match the oracle's tetrahedron-by-tetrahedron CSR assembly to
  1e-12, the FP32 apply to 2e-6; diagonal, face loads (uniform and per
  element face) and step right-hand sides match the assembled pieces;
- transient steps through the engine's tile kernels: FP64 within 1e-9 and
  FP32-refined within 1e-8 of the exact step solution on meshes that cross
  tile boundaries in every direction, with and without Dirichlet faces; FP64
  iteration counts within 2 of the oracle's Algorithm 1, and of its
  Chebyshev PCG on the P1 spectral bound;
- a batch is bitwise its members alone, a batch mixing element types is
  refused, a switch of element between steps and a served request agree
  with the oracle; the 100^3 inclusions workload's first steps at full size.
"""
import numpy as np
import pytest

import workloads as W
from oracle import p1, precond, transient

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [
    ((1, 1, 1), {}),
    ((1, 7, 3), {2: 1.0}),
    ((17, 1, 5), {}),
    ((7, 5, 3), {0: 0.5, 5: -1.0}),
    ((33, 19, 21), {4: 1.0}),          # crosses the 15-column tile in x and y, ragged
    ((40, 6, 9), {f: 0.1 * f for f in range(6)}),
]


def _p1(p):
    p.element = "p1"
    return p


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _run(p, precision, **kw):
    import paper_1905_07622_gb300 as hg
    us, stats = [], []
    with hg.Simulation.from_problem(p, precision=precision, **kw) as s:
        us.append(s.state())
        for _ in range(p.nsteps):
            stats.append(s.step(1))
            us.append(s.state())
    return us, stats


def _eliminated_apply(S, x):
    xf = np.zeros_like(x)
    xf[S.free] = x[S.free]
    y = S.A @ xf
    y[S.dir_ids] = x[S.dir_ids]
    return y


@pytest.mark.parametrize("dims,dirichlet", SHAPES)
def test_apply_matches_oracle_assembly(dims, dirichlet):
    import paper_1905_07622_gb300 as hg
    p = _p1(W.random_box(*dims, seed=sum(dims), extent=(1.0, 0.7, 1.3), dirichlet=dirichlet, theta=0.5,
                         dt=0.003, contrast=(0.1, 10.0)))
    S = transient.build_system(p)
    x = np.random.default_rng(1).standard_normal(p.n_nodes)
    ref = _eliminated_apply(S, x)
    with hg.Simulation.from_problem(p) as s:
        xd = torch.tensor(x, device="cuda")
        yd = torch.empty_like(xd)
        hg.heat_apply(s.sim, xd, yd)
        got = yd.cpu().numpy()
        for sa, sb, mat in ((1.0, 0.0, S.M), (0.0, 1.0, S.K), (1 / p.dt, p.theta - 1, S.L)):
            hg.heat_apply_general(s.sim, sa, sb, xd, yd)
            r2 = mat @ x
            assert np.linalg.norm(yd.cpu().numpy() - r2) <= 1e-12 * np.linalg.norm(r2)
        x32 = torch.tensor(x, device="cuda", dtype=torch.float32)
        y32 = torch.empty_like(x32)
        hg.heat_apply_f32(s.sim, x32, y32)
        ref32 = _eliminated_apply(S, x32.double().cpu().numpy())
        assert np.linalg.norm(y32.double().cpu().numpy() - ref32) <= 2e-6 * np.linalg.norm(ref32)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


@pytest.mark.parametrize("dims,dirichlet", SHAPES)
def test_diagonal_face_loads_and_rhs(dims, dirichlet):
    import paper_1905_07622_gb300 as hg
    p = _p1(W.random_box(*dims, seed=11, dirichlet=dirichlet, flux={5: 2.0, 2: -0.5, 0: 1.0}, flux_steps=1,
                         theta=0.5, dt=0.02))
    S = transient.build_system(p)
    with hg.Simulation.from_problem(p) as s:
        d = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
        hg.heat_diagonal(s.sim, d)
        diag = d.cpu().numpy()
        hg.heat_flux_vector(s.sim, d)
        flux = d.cpu().numpy()
        u = torch.tensor(p.u0, device="cuda")
        hg.heat_rhs(s.sim, 1, u, d)
        rhs1 = d.cpu().numpy()
        # per-element face flux on face 3
        na, nb = p.nx, p.nz
        q = np.random.default_rng(5).uniform(-1, 2, na * nb)
        hg.heat_set_face_flux(s.sim, 3, q)
        hg.heat_flux_vector(s.sim, d)
        flux_q = d.cpu().numpy()
    ref_diag = np.ones(p.n_nodes)
    ref_diag[S.free] = S.A_ff.diagonal()
    assert np.abs(diag - ref_diag).max() <= 1e-13 * np.abs(ref_diag).max()
    Ff = S.F.copy()
    Ff[S.dir_ids] = 0.0
    assert np.abs(flux - Ff).max() <= 1e-14 * max(1.0, np.abs(S.F).max())
    ref_rhs = np.zeros(p.n_nodes)
    ref_rhs[S.free] = transient.step_rhs(p, S, p.u0, 1)
    ref_rhs[S.dir_ids] = S.dir_vals
    assert np.abs(rhs1 - ref_rhs).max() <= 1e-12 * np.abs(ref_rhs).max()
    Fq = S.F + p1.face_load_elements(p.nx, p.ny, p.nz, p.extent, 3, q)  # face 3 had no uniform flux
    Fq[S.dir_ids] = 0.0
    assert np.abs(flux_q - Fq).max() <= 1e-14 * max(1.0, np.abs(Fq).max())


@pytest.mark.parametrize("dims,dirichlet", [((33, 19, 21), {4: 1.0}), ((17, 31, 6), {}),
                                            ((5, 4, 40), {0: 1.0, 3: -0.5}), ((1, 1, 1), {f: 0.3 for f in range(6)})])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32_refined", 1e-8)])
def test_transient_steps(dims, dirichlet, precision, tol):
    p = _p1(W.random_box(*dims, seed=4, dirichlet=dirichlet, flux={2: 1.0}, theta=0.5, dt=0.01, nsteps=3,
                         rtol=1e-12, contrast=(0.1, 10.0)))
    exact = transient.run(p, solver="direct")
    us, stats = _run(p, precision)
    assert all(st["status"] == 0 for st in stats)
    errs = [_rel(us[n], exact.u[n]) for n in range(1, p.nsteps + 1)]
    assert max(errs) <= tol, errs


def test_fp64_iterations_match_oracle_pcg_jacobi_and_chebyshev():
    p = _p1(W.random_box(14, 12, 16, seed=4, dt=10.0, contrast=(0.01, 100.0), dirichlet={4: 1.0}, flux={3: 0.5},
                         nsteps=3, rtol=1e-10))
    S = transient.build_system(p)
    ref = transient.run(p, solver="pcg", system=S)
    _, stats = _run(p, "fp64")
    got = [st["iters"] for st in stats]
    assert all(abs(a - b) <= 2 for a, b in zip(got, ref.iters)), (got, ref.iters)
    refc = transient.run(p, solver="pcg", system=S, cheb=(3, 10.0))
    us, stats = _run(p, "fp64", cheb_degree=3)
    got = [st["iters"] for st in stats]
    assert all(abs(a - b) <= 2 for a, b in zip(got, refc.iters)), (got, refc.iters)
    import paper_1905_07622_gb300 as hg
    with hg.Simulation.from_problem(p, cheb_degree=3) as s:
        _, hi = hg.heat_cheb_interval(s.sim)
    ref_hi = precond.element_lam_max(p)
    assert abs(hi - ref_hi) <= 1e-13 * ref_hi


def test_batch_bitwise_alone_and_mixed_elements_refused():
    import paper_1905_07622_gb300 as hg
    probs = [_p1(W.random_box(*d, seed=s, dt=0.5, contrast=(0.1, 10.0), dirichlet={4: 1.0}, nsteps=3))
             for s, d in ((1, (12, 10, 14)), (2, (9, 17, 6)), (3, (20, 8, 11)))]
    for precision in ("fp32_refined", "fp64"):
        alone = [_run(p, precision)[0][-1] for p in probs]
        sims = [hg.Simulation.from_problem(p, precision=precision) for p in probs]
        try:
            b = hg.heat_batch_create([s.sim for s in sims])
            try:
                rc, _ = hg.heat_batch_step(b, probs[0].nsteps, len(sims))
                assert rc == 0
            finally:
                hg.heat_destroy_batch(b)
            for s, a in zip(sims, alone):
                assert np.array_equal(s.state(), a)
        finally:
            for s in sims:
                s.close()
    q1 = W.random_box(5, 5, 5, seed=9)
    sims = [hg.Simulation.from_problem(probs[0]), hg.Simulation.from_problem(q1)]
    try:
        with pytest.raises(hg.HeatError):
            hg.heat_batch_create([s.sim for s in sims])
    finally:
        for s in sims:
            s.close()


def test_switching_element_between_steps():
    import paper_1905_07622_gb300 as hg
    p = W.random_box(9, 8, 7, seed=3, dt=0.05, dirichlet={4: 1.0}, flux={5: 0.7}, nsteps=2, rtol=1e-12)
    exact_q1 = transient.run(p, solver="direct")
    pp = _p1(W.random_box(9, 8, 7, seed=3, dt=0.05, dirichlet={4: 1.0}, flux={5: 0.7}, nsteps=2, rtol=1e-12))
    kw = dict(theta=p.theta, dt=p.dt, rtol=p.rtol, precision="fp32_refined")
    with hg.Simulation.from_problem(p, precision="fp32_refined") as s:
        s.step(1)
        assert _rel(s.state(), exact_q1.u[1]) <= 1e-8
        s.set_params(element="p1", **kw)
        s.step(1)
        u = s.state()
    # the second step is a P1 step from the Q1 state (the history restarts at U^1 only if set_state is called)
    S = transient.build_system(pp)
    b = transient.step_rhs(pp, S, exact_q1.u[1], 2)
    import scipy.sparse.linalg as spla
    ref = np.empty(pp.n_nodes)
    ref[S.free] = spla.spsolve(S.A_ff.tocsc(), b)
    ref[S.dir_ids] = S.dir_vals
    assert _rel(u, ref) <= 1e-8


def test_served_request_matches_oracle():
    import paper_1905_07622_gb300 as hg
    p = _p1(W.random_box(11, 9, 13, seed=21, dt=0.05, dirichlet={0: 0.2}, flux={5: 1.0}, nsteps=3, rtol=1e-12))
    exact = transient.run(p, solver="direct")
    srv = hg.heat_server_create(1 << 30, 4)
    try:
        req, keep = hg.make_request(p, rtol=1e-12)
        t = hg.heat_submit(srv, req)
        u, st, _ = hg.heat_wait(srv, t, p.n_nodes)
    finally:
        hg.heat_destroy_server(srv)
    assert _rel(u, exact.u[-1]) <= 1e-8


def test_inclusions_cube_100_first_steps():
    """Full size (1,030,301 nodes, 6 million tetrahedra): first 2 steps vs the oracle."""
    p = _p1(W.inclusions_cube().truncated(2))
    S = transient.build_system(p)
    ref = transient.run(p, solver="pcg", rtol=1e-13, system=S)
    for prec, tol in (("fp64", 1e-9), ("fp32_refined", 1e-8)):
        us, stats = _run(p, prec)
        assert all(st["status"] == 0 for st in stats)
        assert max(_rel(us[n], ref.u[n]) for n in (1, 2)) <= tol
