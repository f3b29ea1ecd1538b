"""Q1 finite-element pieces of the oracle (test infrastructure only).

Follows §3.1 (global matrices M = [int rho C phi_m phi_n], K = [int k grad
phi_m . grad phi_n], flux vector F) and §3.2 (element matrices M_e, K_e on a
fixed grid, coefficients constant per element, assembly operator of Eq. 1).
Element matrices are integrated with 2x2x2 Gauss quadrature, which is exact for
trilinear shape functions on boxes.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

# local corner c of an element: (cx, cy, cz) = bits of c
CORNERS = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], dtype=np.int64)
_GP = np.array([-1.0, 1.0]) / np.sqrt(3.0)


def shape_q1(xi: float, eta: float, zeta: float):
    """Trilinear shape functions on [-1,1]^3 and their reference gradients.

    Returns N (8,) and dN (8, 3) for the corners in CORNERS order.
    """
    s = 2.0 * CORNERS - 1.0  # corner signs
    fx = 1.0 + s[:, 0] * xi
    fy = 1.0 + s[:, 1] * eta
    fz = 1.0 + s[:, 2] * zeta
    N = fx * fy * fz / 8.0
    dN = np.stack([s[:, 0] * fy * fz, fx * s[:, 1] * fz, fx * fy * s[:, 2]], axis=1) / 8.0
    return N, dN


def element_matrices(hx: float, hy: float, hz: float):
    """Element mass and stiffness matrices (8x8) of an hx*hy*hz box (§3.2).

    M_e[a,b] = int N_a N_b dx,  K_e[a,b] = int grad N_a . grad N_b dx,
    by 2x2x2 Gauss quadrature (x = x0 + (xi+1) h/2, so dx = (h/2) dxi).
    """
    detJ = hx * hy * hz / 8.0
    inv_jac = np.array([2.0 / hx, 2.0 / hy, 2.0 / hz])
    Me = np.zeros((8, 8))
    Ke = np.zeros((8, 8))
    for xi in _GP:
        for eta in _GP:
            for zeta in _GP:
                N, dN = shape_q1(xi, eta, zeta)
                G = dN * inv_jac  # physical gradients (8, 3)
                Me += np.outer(N, N) * detJ
                Ke += (G @ G.T) * detJ
    return Me, Ke


def spacing(nx, ny, nz, extent):
    return extent[0] / nx, extent[1] / ny, extent[2] / nz


def node_id(nx, ny, i, j, k):
    return i + (nx + 1) * (j + (ny + 1) * k)


def connectivity(nx: int, ny: int, nz: int) -> np.ndarray:
    """(Ne, 8) global node ids of each element's corners, element order."""
    ek, ej, ei = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    ei, ej, ek = ei.ravel(), ej.ravel(), ek.ravel()
    conn = np.empty((ei.size, 8), dtype=np.int64)
    for c in range(8):
        cx, cy, cz = CORNERS[c]
        conn[:, c] = node_id(nx, ny, ei + cx, ej + cy, ek + cz)
    return conn


def assemble(nx, ny, nz, extent, coef: np.ndarray, which: str, chunk: int = 200_000):
    """Global CSR matrix  sum_e coef_e * X_e  with X = M (mass) or K (stiffness).

    This is the assembly operator of Eq. 1 carried out explicitly (the thing the
    assembly-free method avoids), element by element in chunks.
    """
    Me, Ke = element_matrices(*spacing(nx, ny, nz, extent))
    Xe = Me if which == "M" else Ke
    n = (nx + 1) * (ny + 1) * (nz + 1)
    conn = connectivity(nx, ny, nz)
    coef = np.asarray(coef, dtype=np.float64)
    total = None
    for s in range(0, conn.shape[0], chunk):
        c = conn[s:s + chunk]
        rows = np.repeat(c, 8, axis=1).ravel()
        cols = np.tile(c, (1, 8)).ravel()
        vals = (coef[s:s + chunk, None, None] * Xe[None, :, :]).ravel()
        part = sp.coo_matrix((vals, (rows, cols)), shape=(n, n)).tocsr()
        total = part if total is None else total + part
    total.sum_duplicates()
    return total


def face_nodes(nx, ny, nz, face: int) -> np.ndarray:
    """Node ids on a face (0:x0 1:x1 2:y0 3:y1 4:z0 5:z1)."""
    ids = np.arange((nx + 1) * (ny + 1) * (nz + 1)).reshape(nz + 1, ny + 1, nx + 1)
    return {0: ids[:, :, 0], 1: ids[:, :, nx], 2: ids[:, 0, :], 3: ids[:, ny, :],
            4: ids[0, :, :], 5: ids[nz, :, :]}[face].ravel()


def face_load(nx, ny, nz, extent, face: int, q: float) -> np.ndarray:
    """F_i = int_face q phi_i ds for a constant inward flux q on one face (§3.1).

    Each face quad carries bilinear shape functions; 2x2 Gauss quadrature.
    """
    n = (nx + 1) * (ny + 1) * (nz + 1)
    F = np.zeros(n)
    hx, hy, hz = spacing(nx, ny, nz, extent)
    axis = face // 2
    side = face % 2
    dims = [d for d in range(3) if d != axis]
    counts = (nx, ny, nz)
    h = (hx, hy, hz)
    detJ = h[dims[0]] * h[dims[1]] / 4.0
    # integral of each bilinear corner function over the reference quad
    wq = np.zeros(4)
    for a in _GP:
        for b in _GP:
            for c, (ca, cb) in enumerate([(0, 0), (1, 0), (0, 1), (1, 1)]):
                wq[c] += (1 + (2 * ca - 1) * a) * (1 + (2 * cb - 1) * b) / 4.0 * detJ
    fixed = 0 if side == 0 else counts[axis]
    for p in range(counts[dims[0]]):
        for r in range(counts[dims[1]]):
            for c, (ca, cb) in enumerate([(0, 0), (1, 0), (0, 1), (1, 1)]):
                idx = [0, 0, 0]
                idx[axis] = fixed
                idx[dims[0]] = p + ca
                idx[dims[1]] = r + cb
                F[node_id(nx, ny, *idx)] += q * wq[c]
    return F


def face_load_elements(nx, ny, nz, extent, face: int, q_elem) -> np.ndarray:
    """F_i = int_face q phi_i ds for a flux density that is constant on each
    element face of `face` (§3.1): q_elem[a + na*b] on the quad with lower
    tangential index a and upper index b (na quads along the lower one).

    The same 2x2 Gauss quadrature of the bilinear face functions as face_load.
    """
    n = (nx + 1) * (ny + 1) * (nz + 1)
    F = np.zeros(n)
    h = spacing(nx, ny, nz, extent)
    axis = face // 2
    dims = [d for d in range(3) if d != axis]
    counts = (nx, ny, nz)
    detJ = h[dims[0]] * h[dims[1]] / 4.0
    corners = [(0, 0), (1, 0), (0, 1), (1, 1)]
    fixed = 0 if face % 2 == 0 else counts[axis]
    na = counts[dims[0]]
    q_elem = np.asarray(q_elem, dtype=np.float64)
    for p in range(counts[dims[0]]):
        for r in range(counts[dims[1]]):
            q = q_elem[p + na * r]
            for ca, cb in corners:
                w = 0.0  # int of this corner's bilinear function times q over the quad
                for a in _GP:
                    for b in _GP:
                        w += (1 + (2 * ca - 1) * a) * (1 + (2 * cb - 1) * b) / 4.0 * detJ
                idx = [0, 0, 0]
                idx[axis] = fixed
                idx[dims[0]] = p + ca
                idx[dims[1]] = r + cb
                F[node_id(nx, ny, *idx)] += q * w
    return F


def flux_vector(p) -> np.ndarray:
    """Sum of the face loads of all Neumann flux faces of a Problem."""
    F = np.zeros(p.n_nodes)
    for face, q in p.flux.items():
        F += face_load(p.nx, p.ny, p.nz, p.extent, int(face), float(q))
    return F


def dirichlet_nodes(p):
    """(ids, values) of the Dirichlet nodes; the lowest face id wins on overlaps."""
    val = {}
    for face in sorted(p.dirichlet, reverse=True):
        for i in face_nodes(p.nx, p.ny, p.nz, int(face)):
            val[int(i)] = float(p.dirichlet[face])
    ids = np.array(sorted(val), dtype=np.int64)
    return ids, np.array([val[i] for i in ids], dtype=np.float64)


def apply_rows(p, x: np.ndarray, rows, sa: float, sb: float, eliminate: bool = True):
    """(sa*M + sb*K) x at the listed rows only, element by element (Eq. 1, DbD form).

    With eliminate=True the Dirichlet rows return x_i and Dirichlet columns are
    dropped, i.e. the operator of the eliminated system padded with identity.
    Used to check full-size GPU applies at sampled rows.
    """
    nx, ny, nz = p.nx, p.ny, p.nz
    Me, Ke = element_matrices(*spacing(nx, ny, nz, p.extent))
    dir_ids = set(dirichlet_nodes(p)[0].tolist()) if eliminate else set()
    out = np.zeros(len(rows))
    for t, i in enumerate(rows):
        i = int(i)
        if i in dir_ids:
            out[t] = x[i]
            continue
        iz, rem = divmod(i, (nx + 1) * (ny + 1))
        iy, ix = divmod(rem, nx + 1)
        acc = 0.0
        for c in range(8):  # this node is corner c of element (ix-cx, iy-cy, iz-cz)
            ex, ey, ez = ix - CORNERS[c, 0], iy - CORNERS[c, 1], iz - CORNERS[c, 2]
            if not (0 <= ex < nx and 0 <= ey < ny and 0 <= ez < nz):
                continue
            e = ex + nx * (ey + ny * ez)
            for b in range(8):
                j = node_id(nx, ny, ex + CORNERS[b, 0], ey + CORNERS[b, 1], ez + CORNERS[b, 2])
                if j in dir_ids:
                    continue
                acc += (sa * p.rho_c[e] * Me[c, b] + sb * p.k[e] * Ke[c, b]) * x[j]
        out[t] = acc
    return out


def _layer_connectivity(nx, ny, k0, k1):
    """(nx*ny*(k1-k0), 8) corner node ids of the elements in element layers [k0, k1)."""
    ek, ej, ei = np.meshgrid(np.arange(k0, k1), np.arange(ny), np.arange(nx), indexing="ij")
    ei, ej, ek = ei.ravel(), ej.ravel(), ek.ravel()
    conn = np.empty((ei.size, 8), dtype=np.int64)
    for c in range(8):
        cx, cy, cz = CORNERS[c]
        conn[:, c] = node_id(nx, ny, ei + cx, ej + cy, ek + cz)
    return conn


def apply_all(p, x: np.ndarray, sa: float, sb: float, eliminate: bool = True, layers: int = 16,
              absolute: bool = False):
    """(sa*M + sb*K) x at every row, element by element: y = sum_e A_e^T X_e A_e x
    with X_e = sa*rho_c_e*M_e + sb*k_e*K_e (Eq. 1 read as a product, no matrix
    assembled), taken over `layers` element layers at a time so that 200^3
    meshes fit in host memory.

    With eliminate=True Dirichlet columns are dropped and Dirichlet rows return
    x_i (the eliminated operator padded with identity, as apply_rows).
    With absolute=True every term is taken by magnitude, sum_e |X_e| |A_e x|:
    the scale ||A||x|| that rounding errors in evaluating A x are relative to.
    """
    nx, ny, nz = p.nx, p.ny, p.nz
    n = p.n_nodes
    Me, Ke = element_matrices(*spacing(nx, ny, nz, p.extent))
    xs = np.array(x, dtype=np.float64, copy=True)
    if absolute:
        Me, Ke, sa, sb, xs = np.abs(Me), np.abs(Ke), abs(sa), abs(sb), np.abs(xs)
    dir_ids = dirichlet_nodes(p)[0] if eliminate else np.zeros(0, dtype=np.int64)
    xs[dir_ids] = 0.0
    rho_c = np.asarray(p.rho_c, dtype=np.float64)
    kk = np.asarray(p.k, dtype=np.float64)
    y = np.zeros(n)
    for k0 in range(0, nz, layers):
        k1 = min(nz, k0 + layers)
        conn = _layer_connectivity(nx, ny, k0, k1)
        e0, e1 = nx * ny * k0, nx * ny * k1
        xe = xs[conn]  # (ne, 8) element vectors A_e x
        ye = (sa * rho_c[e0:e1, None]) * (xe @ Me.T) + (sb * kk[e0:e1, None]) * (xe @ Ke.T)
        y += np.bincount(conn.ravel(), weights=ye.ravel(), minlength=n)
    if eliminate:
        y[dir_ids] = np.asarray(x, dtype=np.float64)[dir_ids]
    return y


def diagonal_all(p, sa: float, sb: float):
    """diag(sa*M + sb*K) with Dirichlet rows set to 1: the Jacobi preconditioner
    P of Algorithm 1 on the eliminated system, summed element by element."""
    nx, ny, nz = p.nx, p.ny, p.nz
    Me, Ke = element_matrices(*spacing(nx, ny, nz, p.extent))
    conn = _layer_connectivity(nx, ny, 0, nz)
    w = sa * np.asarray(p.rho_c, dtype=np.float64)[:, None] * np.diag(Me)[None, :] \
        + sb * np.asarray(p.k, dtype=np.float64)[:, None] * np.diag(Ke)[None, :]
    d = np.bincount(conn.ravel(), weights=w.ravel(), minlength=p.n_nodes)
    d[dirichlet_nodes(p)[0]] = 1.0
    return d


def assemble_stencil(p, sa: float, sb: float, layers: int = 16):
    """sa*M + sb*K as a CSR matrix, built as 27 node-offset diagonals: entry
    (i, i+o) sums sa*rho_c_e*M_e[c, b] + sb*k_e*K_e[c, b] over the elements e
    in which node i is corner c and node i+o corner b (Eq. 1's assembly with
    the structured mesh's fixed offsets). The same matrix as
    sa*assemble(..., "M") + sb*assemble(..., "K"), built without a COO
    intermediate so that 200^3 meshes fit."""
    nx, ny, nz = p.nx, p.ny, p.nz
    n = p.n_nodes
    px, pxy = nx + 1, (nx + 1) * (ny + 1)
    Me, Ke = element_matrices(*spacing(nx, ny, nz, p.extent))
    rho_c = np.asarray(p.rho_c, dtype=np.float64)
    kk = np.asarray(p.k, dtype=np.float64)
    offs = {}
    for c in range(8):
        for b in range(8):
            d = CORNERS[b] - CORNERS[c]
            offs.setdefault((int(d[0]), int(d[1]), int(d[2])), []).append((c, b))
    diags = {o: np.zeros(n) for o in offs}
    for k0 in range(0, nz, layers):
        k1 = min(nz, k0 + layers)
        conn = _layer_connectivity(nx, ny, k0, k1)
        e0, e1 = nx * ny * k0, nx * ny * k1
        rc, kc = sa * rho_c[e0:e1], sb * kk[e0:e1]
        for o, pairs in offs.items():
            acc = diags[o]
            for c, b in pairs:
                acc += np.bincount(conn[:, c], weights=rc * Me[c, b] + kc * Ke[c, b], minlength=n)
    data, offsets = [], []
    for (dx, dy, dz), vals in diags.items():
        o = dx + px * dy + pxy * dz
        # dia_matrix stores diagonal o at column j = i + o: shift the row-indexed values
        col = np.zeros(n)
        if o >= 0:
            col[o:] = vals[: n - o]
        else:
            col[: n + o] = vals[-o:]
        data.append(col)
        offsets.append(o)
    return sp.dia_matrix((np.array(data), np.array(offsets)), shape=(n, n)).tocsr()
