"""Theta-scheme transient driver of the oracle (test infrastructure only).

Each step solves the system of §3.1 divided by dt (trilinear boxes, or the
six-tetrahedra split of §4.1 when the problem's element is "p1"):
    A U^n = L U^{n-1} + F^n,  A = M/dt + theta K,  L = M/dt - (1-theta) K,
with M, K assembled explicitly (the definition the assembly-free method must
reproduce). Dirichlet nodes (a reading: the paper only has flux faces) are
eliminated symmetrically: the free rows solve
    A_ff U_f = (L U^{n-1} + F^n)_f - A_fD g,  U_D = g.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List

import numpy as np

from . import fem, p1 as _p1, pcg as _pcg, precond as _precond


@dataclass
class System:
    """Assembled matrices and index sets of one Problem."""

    M: object
    K: object
    A: object
    L: object
    F: np.ndarray
    free: np.ndarray
    dir_ids: np.ndarray
    dir_vals: np.ndarray
    A_ff: object
    A_fD: object
    pinv_f: np.ndarray


def build_system(p) -> System:
    asm = _p1 if getattr(p, "element", "q1") == "p1" else fem
    M = asm.assemble(p.nx, p.ny, p.nz, p.extent, p.rho_c, "M")
    K = asm.assemble(p.nx, p.ny, p.nz, p.extent, p.k, "K")
    A = (M / p.dt + p.theta * K).tocsr()
    L = (M / p.dt - (1.0 - p.theta) * K).tocsr()
    F = asm.flux_vector(p)
    dir_ids, dir_vals = fem.dirichlet_nodes(p)
    mask = np.ones(p.n_nodes, dtype=bool)
    mask[dir_ids] = False
    free = np.nonzero(mask)[0]
    A_f = A[free]
    A_ff = A_f[:, free].tocsr()
    A_fD = A_f[:, dir_ids].tocsr()
    pinv_f = 1.0 / A_ff.diagonal()
    return System(M, K, A, L, F, free, dir_ids, dir_vals, A_ff, A_fD, pinv_f)


def flux_on(p, n: int) -> bool:
    return p.flux_steps < 0 or n <= p.flux_steps


def step_rhs(p, S: System, u_prev: np.ndarray, n: int) -> np.ndarray:
    """Free-row right-hand side of step n."""
    rhs = S.L @ u_prev
    if flux_on(p, n):
        rhs = rhs + S.F
    b_f = rhs[S.free]
    if S.dir_ids.size:
        b_f = b_f - S.A_fD @ S.dir_vals
    return b_f


@dataclass
class Result:
    u: List[np.ndarray] = field(default_factory=list)  # u[0] = U^0 ... u[n] = U^n
    iters: List[int] = field(default_factory=list)


def run(p, solver: str = "direct", rtol: float = None, max_iter: int = 20000,
        nsteps: int = None, system: System = None, callback=None, cheb=None) -> Result:
    """Run the transient; solver is 'direct' (sparse LU), 'dense' or 'pcg'
    (Algorithm 1; with cheb = (degree, ratio) its Chebyshev-preconditioned
    form on the interval [lam_hi / ratio, lam_hi] of the element bound)."""
    S = system or build_system(p)
    rtol = p.rtol if rtol is None else rtol
    nsteps = p.nsteps if nsteps is None else nsteps
    lu = None
    if solver == "direct" and S.free.size:
        import scipy.sparse.linalg as spla
        lu = spla.splu(S.A_ff.tocsc())
    u_prev = np.array(p.u0, dtype=np.float64, copy=True)
    u_prev[S.dir_ids] = S.dir_vals
    u_prev2 = None
    res = Result(u=[u_prev.copy()])
    for n in range(1, nsteps + 1):
        b_f = step_rhs(p, S, u_prev, n)
        if solver == "pcg" and cheb is not None:
            x0 = u_prev if u_prev2 is None else 2.0 * u_prev - u_prev2
            lo, hi = _precond.chebyshev_interval(_precond.element_lam_max(p), cheb[1])
            x, it, _, _ = _precond.pcg_cheb(S.A_ff, b_f, x0[S.free], S.pinv_f, cheb[0], lo, hi, rtol, max_iter)
        elif solver == "pcg":
            x0 = u_prev if u_prev2 is None else 2.0 * u_prev - u_prev2
            x, it, _, _ = _pcg.pcg(S.A_ff, b_f, x0[S.free], S.pinv_f, rtol, max_iter)
        elif solver == "dense":
            x, it = _pcg.solve_dense(S.A_ff, b_f), 0
        else:
            x, it = (lu.solve(b_f) if lu is not None else np.zeros(0)), 0
        u_new = np.empty(p.n_nodes)
        u_new[S.free] = x
        u_new[S.dir_ids] = S.dir_vals
        res.u.append(u_new)
        res.iters.append(int(it))
        if callback is not None:
            callback(n, u_new, it)
        u_prev2, u_prev = u_prev, u_new
    return res
