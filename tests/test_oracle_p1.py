"""Pins of the oracle's linear-tetrahedron discretisation (§4.1) against facts
outside it.

- the unit-cube box matrices equal the hand-worked fixture (path gradients);
- the split: six tetrahedra per box of volume V/6 that tile the box, faces
  shared by exactly two tetrahedra inside, two boundary triangles per
  boundary box face;
- patch tests of the assembled matrices: K 1 = 0, K u = 0 on interior rows
  for a linear u, u^T K u = |grad u|^2 vol, 1^T M 1 = vol and u^T M v equal
  to the exact integral of two linear functions; interior rows of K equal
  the seven-point finite-difference stencil;
- boundary loads: total q * area, and the A/3, A/6 corner shares of the
  triangle split;
- the transient's energy balance; the element spectral bound above the
  spectrum.
"""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import fem, p1, precond, transient

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "p1_kuhn_unit_cube.txt")


def _golden():
    blocks, cur = {}, None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line in ("6K", "120M"):
            cur = blocks.setdefault(line, [])
            continue
        cur.append([float(v) for v in line.split()])
    return np.array(blocks["6K"]) / 6.0, np.array(blocks["120M"]) / 120.0


def test_unit_cube_matrices_match_hand_worked_fixture():
    K_ref, M_ref = _golden()
    M, K = p1.box_matrices(1.0, 1.0, 1.0)
    assert np.allclose(K, K_ref, rtol=0, atol=1e-14)
    assert np.allclose(M, M_ref, rtol=0, atol=1e-15)


def test_box_matrices_scale_and_keep_the_sparsity_on_any_box():
    h = (0.3, 1.7, 0.8)
    M, K = p1.box_matrices(*h)
    M1, _ = p1.box_matrices(1.0, 1.0, 1.0)
    assert np.allclose(M, M1 * np.prod(h), rtol=1e-13)  # the mass scales with the volume
    for c in range(8):
        for d in range(8):
            diff = bin(c ^ d).count("1")
            if diff > 1:  # the stiffness couples only along box edges
                assert K[c, d] == pytest.approx(0.0, abs=1e-15)
            if (c & d) not in (c, d):  # not a tetrahedron edge: no coupling at all
                assert M[c, d] == 0.0 and K[c, d] == 0.0
    assert np.allclose(K.sum(axis=1), 0.0, atol=1e-13)


def test_split_tiles_the_box_conformingly():
    nx, ny, nz, ext = 3, 2, 4, (1.5, 0.4, 2.0)
    tets, parent = p1.tetrahedra(nx, ny, nz)
    assert tets.shape == (6 * nx * ny * nz, 4)
    X = W.node_coords(nx, ny, nz, extent=ext)
    X = np.stack(X, axis=1) if isinstance(X, tuple) else X
    vols = np.array([p1.tet_matrices(X[t])[2] for t in tets])
    assert np.allclose(vols, np.prod(ext) / (nx * ny * nz) / 6.0, rtol=1e-13)
    faces = np.sort(np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]],
                                    tets[:, [0, 1, 2]]]), axis=1)
    _, cnt = np.unique(faces, axis=0, return_counts=True)
    assert set(cnt.tolist()) <= {1, 2}
    quads = 2 * (nx * ny + ny * nz + nx * nz)
    assert np.count_nonzero(cnt == 1) == 2 * quads
    tri, area, face, _ = p1.boundary_triangles(nx, ny, nz, ext)
    for f, a in enumerate((ext[1] * ext[2],) * 2 + (ext[0] * ext[2],) * 2 + (ext[0] * ext[1],) * 2):
        assert math.isclose(area[face == f].sum(), a, rel_tol=1e-13)


def _linear(nx, ny, nz, ext, g, c0):
    X = W.node_coords(nx, ny, nz, extent=ext)
    X = np.stack(X, axis=1) if isinstance(X, tuple) else X
    return X @ np.asarray(g) + c0, X


def test_patch_tests_of_the_assembled_matrices():
    nx, ny, nz, ext = 4, 3, 5, (1.2, 0.9, 2.1)
    ne = nx * ny * nz
    K = p1.assemble(nx, ny, nz, ext, np.ones(ne), "K")
    M = p1.assemble(nx, ny, nz, ext, np.ones(ne), "M")
    vol = np.prod(ext)
    one = np.ones(K.shape[0])
    assert np.abs(K @ one).max() < 1e-12
    g = np.array([0.7, -1.3, 0.4])
    u, X = _linear(nx, ny, nz, ext, g, 0.25)
    Ku = K @ u
    interior = np.all((X > 1e-12) & (X < np.asarray(ext) - 1e-12), axis=1)
    assert np.abs(Ku[interior]).max() < 1e-12
    assert math.isclose(u @ Ku, (g @ g) * vol, rel_tol=1e-12)
    assert math.isclose(one @ (M @ one), vol, rel_tol=1e-13)
    # int (a x + b)(c y + d) over the box, exact for P1 mass
    a, b, c, d = 0.8, -0.3, 1.9, 0.6
    ux, vy = a * X[:, 0] + b, c * X[:, 1] + d
    Lx, Ly, Lz = ext
    exact = (a * Lx * Lx / 2 + b * Lx) * (c * Ly * Ly / 2 + d * Ly) * Lz
    assert math.isclose(ux @ (M @ vy), exact, rel_tol=1e-12)


@pytest.mark.parametrize("face", range(6))
def test_boundary_loads(face):
    nx, ny, nz, ext = 3, 4, 2, (0.6, 1.0, 0.5)
    h = fem.spacing(nx, ny, nz, ext)
    F = p1.face_load(nx, ny, nz, ext, face, 2.5)
    axis = face // 2
    area = np.prod([ext[d] for d in range(3) if d != axis])
    assert math.isclose(F.sum(), 2.5 * area, rel_tol=1e-13)
    A = np.prod([h[d] for d in range(3) if d != axis])
    ids = fem.face_nodes(nx, ny, nz, face)
    dims = [d for d in range(3) if d != axis]
    na, nb = [(nx, ny, nz)[d] for d in dims]
    grid = ids.reshape(nb + 1, na + 1)  # [b, a]
    assert math.isclose(F[grid[0, 0]], 2.5 * A / 3.0, rel_tol=1e-13)       # lower-left corner of its quad's diagonal
    assert math.isclose(F[grid[0, na]], 2.5 * A / 6.0, rel_tol=1e-13)      # off the diagonal
    assert math.isclose(F[grid[nb, na]], 2.5 * A / 3.0, rel_tol=1e-13)
    assert math.isclose(F[grid[1, 1]], 2.5 * A, rel_tol=1e-13)             # interior: 2 A/3 + 2 A/6


def test_transient_energy_balance_and_spectral_bound():
    p = W.random_box(4, 3, 5, seed=7, extent=(1.0, 0.5, 2.0), flux={1: 0.8, 4: -0.3}, dt=0.05, nsteps=3,
                     contrast=(0.1, 10.0))
    p.element = "p1"
    S = transient.build_system(p)
    res = transient.run(p, solver="direct", system=S)
    one = np.ones(p.n_nodes)
    lhs = one @ (S.M @ res.u[-1])
    rhs = one @ (S.M @ p.u0) + p.nsteps * p.dt * S.F.sum()
    assert math.isclose(lhs, rhs, rel_tol=1e-10)
    D = S.pinv_f
    lam = np.linalg.eigvals(D[:, None] * S.A_ff.toarray()).real
    assert lam.max() <= precond.element_lam_max(p) * (1 + 1e-12)


def test_single_loaded_quad_shares():
    # one loaded boundary quad: its two triangles (split along the lower-to-upper
    # diagonal) give the diagonal's ends q A / 3 and the other corners q A / 6
    nx, ny, nz, ext = 4, 3, 5, (2.0, 3.0, 1.0)
    hx, hy, hz = fem.spacing(nx, ny, nz, ext)
    q = np.zeros(nx * nz)
    q[2 + nx * 3] = 1.5  # face y=0, quad (i=2, k=3)
    F = p1.face_load_elements(nx, ny, nz, ext, 2, q)
    A = hx * hz
    share = {(2, 3): 1 / 3, (3, 4): 1 / 3, (3, 3): 1 / 6, (2, 4): 1 / 6}
    for (i, k), w in share.items():
        assert math.isclose(F[fem.node_id(nx, ny, i, 0, k)], 1.5 * A * w, rel_tol=1e-13)
    assert np.count_nonzero(F) == 4


def test_assembled_stiffness_is_the_seven_point_laplacian():
    # every box edge along axis a is used by 2 + 1 + 1 + 2 = 6 of the tetrahedra
    # around it (V/h_a^2 each, V = hx hy hz / 6), so interior rows of K are the
    # finite-difference stencil (hx hy hz / h_a^2) (-1, 2, -1) summed over axes
    nx, ny, nz, ext = 5, 4, 6, (1.0, 0.6, 1.5)
    h = fem.spacing(nx, ny, nz, ext)
    K = p1.assemble(nx, ny, nz, ext, np.ones(nx * ny * nz), "K").tocsr()
    vol = h[0] * h[1] * h[2]
    for (i, j, k) in [(1, 1, 1), (2, 2, 3), (3, 1, 4)]:
        n = fem.node_id(nx, ny, i, j, k)
        row = K.getrow(n).toarray().ravel()
        want = np.zeros_like(row)
        want[n] = sum(2.0 * vol / h[a] ** 2 for a in range(3))
        for a, (di, dj, dk) in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
            for sgn in (-1, 1):
                want[fem.node_id(nx, ny, i + sgn * di, j + sgn * dj, k + sgn * dk)] = -vol / h[a] ** 2
        assert np.allclose(row, want, rtol=0, atol=1e-13 * want[n])
