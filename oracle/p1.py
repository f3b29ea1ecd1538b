"""Linear tetrahedra on the structured box mesh (test infrastructure only).

§4.1 builds its mesh by splitting every box of the structured grid into six
linear tetrahedra. The split used here is the one in which all six share the
box's main diagonal from local corner 0 to local corner 7: for each ordering
(a, b, c) of the three axes, the tetrahedron with vertices
    corner 0, corner e_a, corner e_a + e_b, corner 7.
Every box is split the same way, so the faces match between neighbours. Each
tetrahedron takes its box's coefficients (the per-element inputs of §3.2).

Element matrices come from the general P1 formulas: with the barycentric
coordinates lambda_i of a tetrahedron of volume V (affine, gradients constant),
    M_ij = V (1 + delta_ij) / 20,   K_ij = V grad(lambda_i) . grad(lambda_j),
the gradients taken from the inverse of the 4x4 matrix [1 x y z] of the
vertices. Boundary loads integrate each boundary triangle's linear functions:
a constant flux q on a triangle of area A gives each vertex q A / 3.
"""
from __future__ import annotations

from itertools import permutations

import numpy as np
import scipy.sparse as sp

from . import fem

# vertex corner lists of the six tetrahedra of a box, in a fixed order
AXIS_BIT = (1, 2, 4)
TETS = [(0, AXIS_BIT[a], AXIS_BIT[a] | AXIS_BIT[b], 7) for a, b, _ in permutations(range(3))]


def tet_matrices(X: np.ndarray):
    """(M, K, V) of one linear tetrahedron with vertex coordinates X (4, 3)."""
    T = np.hstack([np.ones((4, 1)), X])
    V = abs(np.linalg.det(T)) / 6.0
    grads = np.linalg.inv(T)[1:, :].T  # row i: grad lambda_i
    M = V * (np.ones((4, 4)) + np.eye(4)) / 20.0
    K = V * grads @ grads.T
    return M, K, V


def box_corner_coords(hx: float, hy: float, hz: float) -> np.ndarray:
    return np.array([[hx * (c & 1), hy * ((c >> 1) & 1), hz * ((c >> 2) & 1)] for c in range(8)], dtype=np.float64)


def box_matrices(hx: float, hy: float, hz: float):
    """8x8 mass and stiffness of one box: the sum of its six tetrahedra's."""
    X = box_corner_coords(hx, hy, hz)
    M = np.zeros((8, 8))
    K = np.zeros((8, 8))
    for t in TETS:
        Mt, Kt, _ = tet_matrices(X[list(t)])
        idx = np.ix_(t, t)
        M[idx] += Mt
        K[idx] += Kt
    return M, K


def tetrahedra(nx: int, ny: int, nz: int):
    """(Nt, 4) global node ids of every tetrahedron and (Nt,) its box's id."""
    conn = fem.connectivity(nx, ny, nz)
    tets = np.concatenate([conn[:, list(t)] for t in TETS], axis=0)
    parent = np.tile(np.arange(conn.shape[0]), len(TETS))
    return tets, parent


def assemble(nx, ny, nz, extent, coef: np.ndarray, which: str) -> sp.csr_matrix:
    """Global sum over tetrahedra of coef(box) * X_tet, X = M or K, built
    tetrahedron by tetrahedron from its own vertex coordinates."""
    h = fem.spacing(nx, ny, nz, extent)
    Xc = box_corner_coords(*h)
    coef = np.asarray(coef, dtype=np.float64)
    conn = fem.connectivity(nx, ny, nz)
    n = (nx + 1) * (ny + 1) * (nz + 1)
    rows, cols, vals = [], [], []
    for t in TETS:
        Mt, Kt, _ = tet_matrices(Xc[list(t)])  # the same for every box of the mesh
        Xt = Mt if which == "M" else Kt
        ids = conn[:, list(t)]
        rows.append(np.repeat(ids, 4, axis=1).ravel())
        cols.append(np.tile(ids, (1, 4)).ravel())
        vals.append((coef[:, None, None] * Xt[None, :, :]).ravel())
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n)).tocsr()
    A.sum_duplicates()
    return A


def boundary_triangles(nx: int, ny: int, nz: int, extent):
    """Triangles on the box boundary: (ids (Nb, 3), area (Nb,), face (Nb,),
    quad (Nb,)) where quad = a + na*b indexes the boundary box face (lower
    tangential index a) that contains the triangle. Found as the tetrahedron
    faces that belong to one tetrahedron only."""
    tets, _ = tetrahedra(nx, ny, nz)
    faces = np.concatenate([tets[:, [1, 2, 3]], tets[:, [0, 2, 3]], tets[:, [0, 1, 3]], tets[:, [0, 1, 2]]])
    key = np.sort(faces, axis=1)
    uniq, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    tri = uniq[cnt == 1]
    coords = np.stack(np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij"),
                      axis=-1).reshape(-1, 3)[:, ::-1]  # (i, j, k) per node id
    h = np.array(fem.spacing(nx, ny, nz, extent))
    P = coords[tri] * h  # (Nb, 3 vertices, 3)
    area = 0.5 * np.linalg.norm(np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), axis=1)
    ijk = coords[tri]
    counts = np.array([nx, ny, nz])
    face = np.full(len(tri), -1)
    for axis in range(3):
        for side in range(2):
            val = 0 if side == 0 else counts[axis]
            on = np.all(ijk[:, :, axis] == val, axis=1)
            face[on] = 2 * axis + side
    dims = {0: (1, 2), 1: (0, 2), 2: (0, 1)}
    quad = np.empty(len(tri), dtype=np.int64)
    for f in range(6):
        sel = face == f
        d0, d1 = dims[f // 2]
        a = ijk[sel][:, :, d0].min(axis=1)
        b = ijk[sel][:, :, d1].min(axis=1)
        quad[sel] = a + counts[d0] * b
    return tri, area, face, quad


def face_load_elements(nx, ny, nz, extent, face: int, q_elem) -> np.ndarray:
    """F_i = int_face q phi_i ds with q constant on each boundary box face of
    `face` (q_elem indexed as in fem.face_load_elements): q A / 3 to each vertex
    of each boundary triangle."""
    tri, area, fc, quad = boundary_triangles(nx, ny, nz, extent)
    sel = fc == face
    F = np.zeros((nx + 1) * (ny + 1) * (nz + 1))
    w = np.asarray(q_elem, dtype=np.float64)[quad[sel]] * area[sel] / 3.0
    for v in range(3):
        np.add.at(F, tri[sel][:, v], w)
    return F


def face_load(nx, ny, nz, extent, face: int, q: float) -> np.ndarray:
    dims = {0: (ny, nz), 1: (nx, nz), 2: (nx, ny)}[face // 2]
    return face_load_elements(nx, ny, nz, extent, face, np.full(dims[0] * dims[1], float(q)))


def flux_vector(p) -> np.ndarray:
    F = np.zeros(p.n_nodes)
    for face, q in p.flux.items():
        F += face_load(p.nx, p.ny, p.nz, p.extent, int(face), float(q))
    return F
