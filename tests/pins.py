"""Pin checks for the oracle: closed forms and invariants the paper's equations fix.

Each check returns an error measure so that the mutation tests can plant a
mistake in the oracle (on the CPU) and show that some check catches it.
"""
from __future__ import annotations

import os
from fractions import Fraction

import numpy as np

from oracle import fem, pcg, transient
import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_q1_unit_cube():
    """(M, K) 8x8 from tests/golden/q1_unit_cube.txt (exact textbook values)."""
    table = {}
    with open(os.path.join(GOLDEN, "q1_unit_cube.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            d, mn, md, kn, kd = (int(t) for t in line.split())
            table[d] = (Fraction(mn, md), Fraction(kn, kd))
    M = np.zeros((8, 8))
    K = np.zeros((8, 8))
    for a in range(8):
        for b in range(8):
            d = bin(a ^ b).count("1")
            M[a, b] = float(table[d][0])
            K[a, b] = float(table[d][1])
    return M, K


def lambda_1d(omega: float, h: float) -> float:
    """Generalised eigenvalue of the 1-D linear-element pencil (K, M) for the
    nodal interpolant of sin/cos(omega x) on a uniform grid of spacing h:
    (6/h^2) (1 - cos(omega h)) / (2 + cos(omega h)).
    """
    c = np.cos(omega * h)
    return 6.0 / h ** 2 * (1.0 - c) / (2.0 + c)


def amplification(lam: float, kappa: float, dt: float, theta: float) -> float:
    """One theta-scheme step of the scalar mode equation u' = -kappa*lam*u."""
    return (1.0 / dt - (1.0 - theta) * kappa * lam) / (1.0 / dt + theta * kappa * lam)


def check_element_golden() -> float:
    Me, Ke = fem.element_matrices(1.0, 1.0, 1.0)
    Mg, Kg = golden_q1_unit_cube()
    return max(np.abs(Me - Mg).max(), np.abs(Ke - Kg).max())


def check_element_box_closed_form(h=(0.7, 1.9, 0.35)) -> float:
    """Anisotropic box vs Kronecker products of the exact 1-D element matrices.

    Corner c has x-bit 1, y-bit 2, z-bit 4, so the z factor is the outermost
    Kronecker factor.
    """
    hx, hy, hz = h
    m1 = lambda s: s / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
    k1 = lambda s: 1.0 / s * np.array([[1.0, -1.0], [-1.0, 1.0]])
    Mx, My, Mz = m1(hx), m1(hy), m1(hz)
    Kx, Ky, Kz = k1(hx), k1(hy), k1(hz)
    M_ref = np.kron(Mz, np.kron(My, Mx))
    K_ref = np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) + np.kron(Kz, np.kron(My, Mx))
    Me, Ke = fem.element_matrices(hx, hy, hz)
    return max(np.abs(Me - M_ref).max() / np.abs(M_ref).max(),
               np.abs(Ke - K_ref).max() / np.abs(K_ref).max())


def mode_problem(kind: str):
    """Homogeneous anisotropic box with an exact discrete eigenmode as u0."""
    nx, ny, nz = 6, 5, 4
    ext = (1.3, 0.8, 0.6)
    rho_c, k = 2.0, 0.7
    X, Y, Z = W.node_coords(nx, ny, nz, extent=ext)
    hx, hy, hz = ext[0] / nx, ext[1] / ny, ext[2] / nz
    if kind == "dirichlet":  # all six faces u = 0
        wx, wy, wz = np.pi / ext[0], 2 * np.pi / ext[1], np.pi / ext[2]
        u0 = np.sin(wx * X) * np.sin(wy * Y) * np.sin(wz * Z)
        dirichlet = {f: 0.0 for f in range(6)}
        theta, dt = 0.5, 2e-3
    elif kind == "mixed":  # u = 0 on x=0, zero flux elsewhere (two_phase_cube's BC set)
        wx, wy, wz = np.pi / (2 * ext[0]), np.pi / ext[1], 2 * np.pi / ext[2]
        u0 = np.sin(wx * X) * np.cos(wy * Y) * np.cos(wz * Z)
        dirichlet = {0: 0.0}
        theta, dt = 1.0, 3e-3
    else:  # pure Neumann cosine mode
        wx, wy, wz = 2 * np.pi / ext[0], 0.0, np.pi / ext[2]
        u0 = np.cos(wx * X) * np.cos(wy * Y) * np.cos(wz * Z)
        dirichlet = {}
        theta, dt = 0.7, 1e-3
    lam = lambda_1d(wx, hx) + lambda_1d(wy, hy) + lambda_1d(wz, hz)
    ne = nx * ny * nz
    p = W.Problem(f"mode_{kind}", nx, ny, nz, extent=ext, rho_c=np.full(ne, rho_c),
                  k=np.full(ne, k), u0=u0, dirichlet=dirichlet, theta=theta, dt=dt,
                  nsteps=4, rtol=1e-13)
    p.u0 = W.apply_dirichlet_values(p, p.u0)
    g = amplification(lam, k / rho_c, dt, theta)
    return p, g


def check_eigenmode(kind: str, solver: str = "direct") -> float:
    """max_n ||U^n - g^n U^0|| / ||U^0|| for an exact discrete eigenmode."""
    p, g = mode_problem(kind)
    res = transient.run(p, solver=solver, rtol=1e-13)
    err = 0.0
    for n, u in enumerate(res.u):
        err = max(err, np.linalg.norm(u - g ** n * res.u[0]) / np.linalg.norm(res.u[0]))
    return err


def check_energy_balance(seed: int = 7) -> float:
    """Zero-flux elsewhere, no Dirichlet: 1^T M (U^n - U^{n-1}) = dt * 1^T F^n."""
    p = W.random_box(4, 3, 5, seed, extent=(1.0, 0.5, 2.0), flux={5: 1.5, 0: -0.4},
                     theta=0.5, dt=0.05, nsteps=4, flux_steps=2)
    S = transient.build_system(p)
    res = transient.run(p, solver="direct", system=S)
    one = np.ones(p.n_nodes)
    ref = abs(one @ (S.M @ res.u[0])) + 1.0
    err = 0.0
    for n in range(1, p.nsteps + 1):
        lhs = one @ (S.M @ (res.u[n] - res.u[n - 1]))
        rhs = p.dt * (one @ S.F) if transient.flux_on(p, n) else 0.0
        err = max(err, abs(lhs - rhs) / ref)
    return err


def check_face_load() -> float:
    """Face load of a constant flux: total q*area; nodal shares q*h_a*h_b*{1,1/2,1/4}."""
    nx, ny, nz, ext, q = 4, 3, 2, (2.0, 1.5, 1.0), 2.5
    err = 0.0
    for face in range(6):
        F = fem.face_load(nx, ny, nz, ext, face, q)
        axis = face // 2
        dims = [d for d in range(3) if d != axis]
        area = ext[dims[0]] * ext[dims[1]]
        err = max(err, abs(F.sum() - q * area) / (q * area))
        n = (nx, ny, nz)
        hA, hB = ext[dims[0]] / n[dims[0]], ext[dims[1]] / n[dims[1]]
        ids = fem.face_nodes(nx, ny, nz, face).reshape(-1)
        share = F[ids] / (q * hA * hB)
        assert set(np.round(share, 12)) <= {1.0, 0.5, 0.25}
    return err


def check_patch_linear(seed: int = 3) -> float:
    """Homogeneous k: K (a + b x + c y + d z) = 0 on interior rows."""
    nx, ny, nz, ext = 5, 4, 6, (1.0, 2.0, 0.7)
    K = fem.assemble(nx, ny, nz, ext, np.full(nx * ny * nz, 1.7), "K")
    X, Y, Z = W.node_coords(nx, ny, nz, extent=ext)
    u = 0.3 + 1.1 * X - 0.7 * Y + 2.0 * Z
    r = (K @ u).reshape(nz + 1, ny + 1, nx + 1)[1:-1, 1:-1, 1:-1]
    return float(np.abs(r).max())


def check_steady_dirichlet() -> float:
    """Dirichlet u=1 on z=0, zero flux elsewhere, theta=1, dt huge: U^1 = 1."""
    p = W.random_box(3, 4, 5, 11, dirichlet={4: 1.0}, theta=1.0, dt=1e13, nsteps=1,
                     contrast=(0.01, 100.0))
    p.u0 = W.apply_dirichlet_values(p, np.zeros(p.n_nodes))
    res = transient.run(p, solver="direct")
    return float(np.abs(res.u[1] - 1.0).max())


def check_pcg_vs_dense(cases=None) -> float:
    """Algorithm 1 PCG (rtol 1e-14) vs dense Cholesky on tiny meshes."""
    cases = cases or [((1, 1, 1), {}), ((2, 2, 2), {4: 0.5}), ((3, 4, 5), {}),
                      ((3, 4, 5), {0: 1.0, 5: -2.0})]
    err = 0.0
    for t, (dims, dirichlet) in enumerate(cases):
        p = W.random_box(*dims, seed=100 + t, dirichlet=dirichlet, flux={2: 1.0},
                         theta=0.5, dt=0.01, nsteps=1, contrast=(0.1, 10.0))
        S = transient.build_system(p)
        b = transient.step_rhs(p, S, p.u0, 1)
        xd = pcg.solve_dense(S.A_ff, b)
        xp, it, _, _ = pcg.pcg(S.A_ff, b, p.u0[S.free], S.pinv_f, 1e-14, 5000)
        err = max(err, np.linalg.norm(xp - xd) / max(np.linalg.norm(xd), 1e-300))
    return err


def check_continuum_decay() -> float:
    """All-Dirichlet unit cube, u0 = sin sin sin: U(center, t) vs exp(-3 pi^2 t)."""
    n = 16
    X, Y, Z = W.node_coords(n, n, n)
    u0 = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    ne = n ** 3
    p = W.Problem("decay", n, n, n, rho_c=np.ones(ne), k=np.ones(ne), u0=u0,
                  dirichlet={f: 0.0 for f in range(6)}, theta=0.5, dt=1e-3, nsteps=10)
    p.u0 = W.apply_dirichlet_values(p, p.u0)
    res = transient.run(p, solver="direct")
    c = fem.node_id(n, n, n // 2, n // 2, n // 2)
    t = p.dt * p.nsteps
    return abs(res.u[-1][c] - np.exp(-3 * np.pi ** 2 * t)) / np.exp(-3 * np.pi ** 2 * t)


def check_pcg_finite_termination() -> float:
    """CG on an n x n SPD system terminates in at most n iterations in exact
    arithmetic. Returns iterations / n on a small system (<= ~1 expected)."""
    p = W.random_box(3, 2, 2, seed=9, theta=1.0, dt=0.1, contrast=(0.2, 5.0))
    S = transient.build_system(p)
    b = transient.step_rhs(p, S, p.u0, 1)
    x, it, delta, delta_b = pcg.pcg(S.A_ff, b, np.zeros_like(b), S.pinv_f, 1e-12, 10000)
    if delta > 1e-24 * delta_b:
        return np.inf
    return it / S.A_ff.shape[0]


def oracle_steps(p, tight_rtol: float = 1e-13, direct_limit: int = 20000):
    """Oracle step solutions for parity tests: sparse LU on small meshes, the
    oracle's Algorithm 1 PCG at a tight tolerance on larger ones (the LU
    fill-in of a 3-D 27-point stencil makes it slow beyond ~20K nodes)."""
    if p.n_nodes <= direct_limit:
        return transient.run(p, solver="direct")
    return transient.run(p, solver="pcg", rtol=tight_rtol)
