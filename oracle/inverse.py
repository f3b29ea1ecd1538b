"""The coefficient inverse problem of §5.3 (test infrastructure only).

Corrosion of depth `depth` grows into a plate from its rear face y = y0 + Ly
with a parabolic profile in z that is constant along x; a heat source on one
face is on for the whole heating period; the observed face's temperatures at
its end are compared with noisy camera data (i.i.d. Gaussian noise, §5.3);
Metropolis-Hastings samples the depth under a uniform prior. Everything here
follows the plain definitions: coefficients by the element-centroid test, the
forward model by the oracle's transient solver with assembled matrices, the
log-likelihood as a sum of squares, and the Metropolis-Hastings rule of §5.3.
"""
from __future__ import annotations

import math

import numpy as np

from . import fem, transient


def corrosion_coefficients(nx, ny, nz, origin, extent, geom: dict, depth: float):
    """(rho_c, k) per element (element order): corroded where the centroid's
    distance from the rear face is below depth * (1 - ((z_c - z0)/w)^2) and
    |z_c - z0| < w, sound elsewhere. Operations in this order, one rounding
    each (numpy float64 scalars):
      z_c = oz + (k + 0.5) hz,  t = (z_c - z0) / w,  d = depth (1 - t t),
      y_c = oy + (j + 0.5) hy,  corroded = |t| < 1 and (y_rear - y_c) < d."""
    hy = extent[1] / ny
    hz = extent[2] / nz
    oy, oz = float(origin[1]), float(origin[2])
    y_rear = oy + extent[1]
    rho_c = np.empty(nx * ny * nz)
    k_arr = np.empty(nx * ny * nz)
    for k in range(nz):
        zc = oz + (k + 0.5) * hz
        t = (zc - geom["z0"]) / geom["half_width"]
        d = depth * (1.0 - t * t)
        for j in range(ny):
            yc = oy + (j + 0.5) * hy
            corr = abs(t) < 1.0 and (y_rear - yc) < d
            sl = slice(nx * (j + ny * k), nx * (j + ny * k) + nx)
            rho_c[sl] = geom["rho_c_corr"] if corr else geom["rho_c_sound"]
            k_arr[sl] = geom["k_corr"] if corr else geom["k_sound"]
    return rho_c, k_arr


def face_values(u, nx, ny, nz, face: int):
    """U on a face's nodes, lower tangential index fastest."""
    return np.asarray(u)[fem.face_nodes(nx, ny, nz, face)]


def loglik(u_face, data, sigma: float) -> float:
    """log p(D | U) up to a constant for i.i.d. N(0, sigma^2) noise (§5.3)."""
    r = (np.asarray(u_face) - np.asarray(data)) / sigma
    return -0.5 * float(np.sum(r * r))


def forward(plate, depth: float):
    """Temperatures at the end of the heating period for one depth: the
    oracle's transient solve (sparse LU) with the corrosion coefficients and
    the per-element face flux. `plate` is a workloads.CorrosionPlate."""
    p = plate.problem()
    p.rho_c, p.k = corrosion_coefficients(p.nx, p.ny, p.nz, p.origin, p.extent, plate.geom, depth)
    S = transient.build_system(p)
    S.F = fem.face_load_elements(p.nx, p.ny, p.nz, p.extent, plate.flux_face, plate.flux_q)
    free = S.free
    S.F[S.dir_ids] = 0.0
    res = transient.run(p, solver="direct", system=S)
    assert free.size == S.free.size
    return res.u[-1]


def mh_chain(state, state_ll, normals, uniforms, step: float, depth_max: float, loglik_fn):
    """Metropolis-Hastings (§5.3) for independent chains advancing together.

    state, state_ll: current depths and log-likelihoods (one per chain);
    normals, uniforms: (niter, nchains) draws. Proposal = depth + step*normal;
    outside [0, depth_max] (the uniform prior's support) it is rejected; else
    accepted with probability min(1, exp(ll' - ll)), i.e. when
    log(uniform) < ll' - ll. loglik_fn(depths) gives the proposals'
    log-likelihoods (all chains at once; out-of-prior chains pass their
    current depth, whose value is not used).
    Returns (depth_trace, ll_trace, accepted), each (niter, nchains)."""
    state = np.array(state, dtype=np.float64)
    ll = np.array(state_ll, dtype=np.float64)
    normals = np.asarray(normals)
    uniforms = np.asarray(uniforms)
    niter, n = normals.shape
    dtr = np.empty((niter, n))
    ltr = np.empty((niter, n))
    acc = np.zeros((niter, n), dtype=bool)
    for it in range(niter):
        prop = state + step * normals[it]
        inside = (prop >= 0.0) & (prop <= depth_max)
        pll = loglik_fn(np.where(inside, prop, state))
        for c in range(n):
            if inside[c] and math.log(uniforms[it, c]) < pll[c] - ll[c]:
                state[c] = prop[c]
                ll[c] = pll[c]
                acc[it, c] = True
        dtr[it] = state
        ltr[it] = ll
    return dtr, ltr, acc
