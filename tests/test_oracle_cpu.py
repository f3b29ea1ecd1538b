"""Pins of the oracle's plain C solvers (oracle/cpcg.c, no GPU).

* oracle.cpu.pcg is Algorithm 1 as oracle.pcg.pcg: the same iteration count
  and solution on one and on several threads.
* oracle.cpu.IC with droptol 0 is the complete Cholesky factor (L L^T = A,
  and L equals numpy's Cholesky factor); with droptol > 0 every kept entry
  satisfies the defining recurrence, so (L L^T)_ij = a_ij on L's pattern
  (diagonal included), and every kept entry passes the drop rule
  |l_ik| >= droptol ||A(k:n, k)||_1.
* oracle.cpu.pcg_ic reaches the sparse-LU solution with fewer iterations
  than Jacobi-PCG under the same stopping rule.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import cpu, pcg, transient


def _system(seed=2, dims=(6, 5, 7), **kw):
    p = W.random_box(*dims, seed=seed, **kw)
    S = transient.build_system(p)
    b = transient.step_rhs(p, S, p.u0, 1)
    return p, S, b, p.u0[S.free]


@pytest.mark.parametrize("seed,dims,kw", [
    (2, (6, 5, 7), dict(dirichlet={0: 1.0}, flux={5: 1.0})),
    (3, (9, 4, 3), dict(flux={2: 0.5}, contrast=(0.1, 10.0))),
    (4, (3, 8, 10), dict(dirichlet={4: 0.0, 3: 2.0}, theta=1.0, dt=0.1)),
])
@pytest.mark.parametrize("threads", [1, 3])
def test_c_pcg_is_algorithm_1_as_the_python_oracle(seed, dims, kw, threads):
    p, S, b, x0 = _system(seed, dims, **kw)
    xa, ia, da, dba = pcg.pcg(S.A_ff, b, x0, S.pinv_f, 1e-12, resid_period=7)
    xb, ib, db, dbb = cpu.pcg(S.A_ff, b, x0, S.pinv_f, 1e-12, resid_period=7, threads=threads)
    assert ia == ib
    assert np.linalg.norm(xa - xb) <= 1e-12 * np.linalg.norm(xa)
    assert abs(dba - dbb) <= 1e-13 * dba


def test_ic_without_dropping_is_the_cholesky_factor():
    p, S, b, x0 = _system(5, (4, 4, 5), dirichlet={1: 0.0})
    L = cpu.IC(S.A_ff, 0.0).matrix().toarray()
    A = S.A_ff.toarray()
    assert np.abs(L @ L.T - A).max() <= 1e-13 * np.abs(A).max()
    assert np.abs(L - np.linalg.cholesky(A)).max() <= 1e-12 * np.abs(L).max()


@pytest.mark.parametrize("droptol", [1e-3, 1e-2, 0.1])
def test_ic_with_dropping_matches_a_on_its_pattern_and_obeys_the_drop_rule(droptol):
    p, S, b, x0 = _system(6, (7, 6, 5), flux={5: 1.0}, contrast=(0.1, 10.0))
    A = S.A_ff.tocsr()
    Lm = cpu.IC(A, droptol).matrix()
    LLt = (Lm @ Lm.T).tocsr()
    Lc = Lm.tocoo()
    rows, cols = Lc.row, Lc.col
    Ad = A.toarray()
    diff = np.abs(np.asarray(LLt[rows, cols]).ravel() - Ad[rows, cols])
    assert diff.max() <= 1e-12 * np.abs(Ad).max()
    colnorm = np.array([np.abs(Ad[k:, k]).sum() for k in range(A.shape[0])])
    off = rows != cols
    assert np.all(np.abs(Lc.data[off]) >= droptol * colnorm[cols[off]] * (1 - 1e-12))
    full = sp.csr_matrix(np.tril(np.linalg.cholesky(Ad)))
    assert Lm.nnz < full.nnz  # something was dropped


def test_ic_pcg_reaches_the_exact_solution_in_fewer_iterations():
    p, S, b, x0 = _system(7, (10, 9, 8), dirichlet={4: 1.0}, flux={5: 1.0}, contrast=(0.2, 5.0))
    exact = pcg.solve_direct(S.A_ff, b)
    F = cpu.IC(S.A_ff, 1e-3)
    x, it_ic, rpr, db = cpu.pcg_ic(S.A_ff, b, x0, S.pinv_f, F, 1e-12)
    _, it_jac, _, _ = cpu.pcg(S.A_ff, b, x0, S.pinv_f, 1e-12)
    assert np.linalg.norm(x - exact) <= 1e-10 * np.linalg.norm(exact)
    assert rpr <= 1e-24 * db
    assert it_ic < it_jac
