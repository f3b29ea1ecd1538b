"""Seeded synthetic inputs for the transient heat problems.

This module is shared by the CUDA path's tests/bench and by the CPU oracle. It
holds no finite-element arithmetic: it only draws coefficient fields, initial
temperatures and boundary-condition descriptions with numpy's PCG64 generator.

Problem statement being parameterised (§3.1): rho*C dT/dt = div(k grad T) in a
box, with prescribed inward heat flux f on some faces (Neumann), optionally a
fixed temperature on some faces (Dirichlet, a reading the paper does not use),
a theta time scheme with step dt, and material coefficients that are constant
on each element (§3.2).

Index conventions (both sides use them):
  * element (i, j, k), 0 <= i < nx, id = i + nx*(j + ny*k)  (x fastest, §4.1)
  * node    (i, j, k), 0 <= i <= nx, id = i + (nx+1)*(j + (ny+1)*k)
  * faces   0: x=x0, 1: x=x1, 2: y=y0, 3: y=y1, 4: z=z0, 5: z=z1
  * a node on several Dirichlet faces takes the value of the lowest face id.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Dict, List, Optional

import numpy as np

FACE_NAMES = ("x0", "x1", "y0", "y1", "z0", "z1")


@dataclass
class Problem:
    """One transient heat simulation, as plain arrays and scalars."""

    name: str
    nx: int
    ny: int
    nz: int
    origin: tuple = (0.0, 0.0, 0.0)
    extent: tuple = (1.0, 1.0, 1.0)
    rho_c: Optional[np.ndarray] = None  # (Ne,) float64, element order
    k: Optional[np.ndarray] = None  # (Ne,) float64, element order
    u0: Optional[np.ndarray] = None  # (N,) float64, node order
    dirichlet: Dict[int, float] = field(default_factory=dict)  # face -> value
    flux: Dict[int, float] = field(default_factory=dict)  # face -> inward q
    flux_steps: int = -1  # flux on for steps 1..flux_steps; -1 = always
    theta: float = 0.5
    dt: float = 1e-3
    nsteps: int = 1
    rtol: float = 1e-10
    element: str = "q1"  # "q1": trilinear boxes; "p1": six linear tetrahedra per box (§4.1)

    @property
    def n_nodes(self) -> int:
        return (self.nx + 1) * (self.ny + 1) * (self.nz + 1)

    @property
    def n_elems(self) -> int:
        return self.nx * self.ny * self.nz

    def dirichlet_mask(self) -> int:
        m = 0
        for f in self.dirichlet:
            m |= 1 << int(f)
        return m

    def truncated(self, nsteps: int) -> "Problem":
        """Same problem, first `nsteps` steps only."""
        p = Problem(**{**self.__dict__})
        p.nsteps = int(nsteps)
        p.name = f"{self.name}[:{nsteps}]"
        return p


def node_coords(nx, ny, nz, origin=(0.0, 0.0, 0.0), extent=(1.0, 1.0, 1.0)):
    """Node coordinate arrays X, Y, Z of shape (N,), node order."""
    xs = origin[0] + extent[0] * np.arange(nx + 1) / nx
    ys = origin[1] + extent[1] * np.arange(ny + 1) / ny
    zs = origin[2] + extent[2] * np.arange(nz + 1) / nz
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def element_centroids(nx, ny, nz, origin=(0.0, 0.0, 0.0), extent=(1.0, 1.0, 1.0)):
    """Element centroid arrays (Ne,), element order."""
    xs = origin[0] + extent[0] * (np.arange(nx) + 0.5) / nx
    ys = origin[1] + extent[1] * (np.arange(ny) + 0.5) / ny
    zs = origin[2] + extent[2] * (np.arange(nz) + 0.5) / nz
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


def apply_dirichlet_values(p: Problem, u: np.ndarray) -> np.ndarray:
    """Overwrite the Dirichlet nodes of a node-order array with their face values.

    The lowest face id wins on shared edges and corners.
    """
    u = np.array(u, dtype=np.float64, copy=True).reshape(p.nz + 1, p.ny + 1, p.nx + 1)
    sl = {0: (slice(None), slice(None), 0), 1: (slice(None), slice(None), p.nx),
          2: (slice(None), 0, slice(None)), 3: (slice(None), p.ny, slice(None)),
          4: (0, slice(None), slice(None)), 5: (p.nz, slice(None), slice(None))}
    for f in sorted(p.dirichlet, reverse=True):  # lowest id written last -> wins
        u[sl[f]] = p.dirichlet[f]
    return u.ravel()


# ---------------------------------------------------------------------------
# The five synthetic workloads (shapes and statistics of the paper's runs:
# ~1M-DoF heterogeneous transients over hundreds of steps, §5.1 and §5.3).
# ---------------------------------------------------------------------------

def two_phase_cube(n: int = 16, seed: int = 1001, p_b: float = 0.3) -> Problem:
    """16^3 two-phase cube: Bernoulli(0.3) elements get k=10, rho_c=2 (else 1, 1).

    Dirichlet u=0 on x=0, zero flux elsewhere, u0 = sin(pi x) sin(pi y) sin(pi z),
    backward Euler (theta=1), dt=1e-3, 20 steps, rtol 1e-10.
    """
    rng = np.random.default_rng(seed)
    ne = n ** 3
    phase_b = rng.random(ne) < p_b
    rho_c = np.where(phase_b, 2.0, 1.0)
    k = np.where(phase_b, 10.0, 1.0)
    X, Y, Z = node_coords(n, n, n)
    u0 = np.sin(np.pi * X) * np.sin(np.pi * Y) * np.sin(np.pi * Z)
    p = Problem("two_phase_cube_16", n, n, n, rho_c=rho_c, k=k, u0=u0,
                dirichlet={0: 0.0}, flux={}, flux_steps=-1, theta=1.0, dt=1e-3,
                nsteps=20, rtol=1e-10)
    p.u0 = apply_dirichlet_values(p, p.u0)
    return p


def _sphere_field(n, centres, radii, inside_vals, outside_vals):
    cx, cy, cz = element_centroids(n, n, n)
    inside = np.zeros(cx.shape, dtype=bool)
    for (x, y, z), r in zip(centres, radii):
        inside |= (cx - x) ** 2 + (cy - y) ** 2 + (cz - z) ** 2 <= r * r
    rho_c = np.where(inside, inside_vals[0], outside_vals[0])
    k = np.where(inside, inside_vals[1], outside_vals[1])
    return rho_c, k


def inclusions_cube(n: int = 100, seed: int = 1002, n_incl: int = 200,
                    nsteps: int = 300) -> Problem:
    """100^3 cube (1,030,301 nodes) with 200 spherical inclusions.

    Matrix k=1, rho_c=1; inclusions (centres U[0,1]^3, radius U[0.02,0.06],
    element centroid test, overlaps allowed) k=10, rho_c=3. No Dirichlet face;
    flux q=1 into z=1 for the first 50 steps (t < 0.05); dt=1e-3; 300 steps;
    theta=0.5; u0=0.
    """
    rng = np.random.default_rng(seed)
    centres = rng.random((n_incl, 3))
    radii = rng.uniform(0.02, 0.06, n_incl)
    rho_c, k = _sphere_field(n, centres, radii, (3.0, 10.0), (1.0, 1.0))
    return Problem(f"inclusions_cube_{n}", n, n, n, rho_c=rho_c, k=k,
                   u0=np.zeros((n + 1) ** 3), dirichlet={}, flux={5: 1.0},
                   flux_steps=50, theta=0.5, dt=1e-3, nsteps=nsteps, rtol=1e-10)


def lognormal_cube(sample: int, n: int = 40, nsteps: int = 150) -> Problem:
    """40^3 cube with iid log-normal k_e = exp(N(0,1)), rho_c=1 (seed 3000+sample).

    Flux q=1 into z=1 for the first 25 steps (t < 0.05 at dt=2e-3); 150 steps;
    theta=0.5; u0=0; no Dirichlet face.
    """
    rng = np.random.default_rng(3000 + sample)
    ne = n ** 3
    k = np.exp(rng.standard_normal(ne))
    return Problem(f"lognormal_cube_{n}_s{sample}", n, n, n, rho_c=np.ones(ne), k=k,
                   u0=np.zeros((n + 1) ** 3), dirichlet={}, flux={5: 1.0},
                   flux_steps=25, theta=0.5, dt=2e-3, nsteps=nsteps, rtol=1e-10)


def serving_request(r: int, n_min: int = 20, n_max: int = 120) -> Problem:
    """One request of the serving stream (seed 4000+r).

    Edge n ~ U{n_min..n_max}; volume fraction phi ~ U[0.1,0.5]; Bernoulli(phi)
    elements k=10 else 1, rho_c=1; steps ~ U{50..300}; flux q=1 into z=1 for
    50 steps (t < 0.05 at dt=1e-3); theta=0.5; u0=0; rtol 1e-8.
    """
    rng = np.random.default_rng(4000 + r)
    n = int(rng.integers(n_min, n_max + 1))
    phi = float(rng.uniform(0.1, 0.5))
    nsteps = int(rng.integers(50, 301))
    ne = n ** 3
    k = np.where(rng.random(ne) < phi, 10.0, 1.0)
    return Problem(f"request_{r}_n{n}", n, n, n, rho_c=np.ones(ne), k=k,
                   u0=np.zeros((n + 1) ** 3), dirichlet={}, flux={5: 1.0},
                   flux_steps=50, theta=0.5, dt=1e-3, nsteps=nsteps, rtol=1e-8)


def poisson_arrivals(n_req: int, rate: float = 50.0, seed: int = 4999) -> np.ndarray:
    """Arrival times (s) of a Poisson stream with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, n_req))


def layered_cube(n: int = 200, seed: int = 1005, n_layers: int = 20,
                 n_pockets: int = 30, nsteps: int = 100) -> Problem:
    """200^3 layered cube (8,120,601 nodes).

    20 horizontal layers (19 interfaces at distinct element-face heights drawn
    uniformly, each layer >= 1 element), k alternating 1 / 1000 from the bottom,
    rho_c = 1; 30 axis-aligned ellipsoidal pockets (centres U[0,1]^3, semi-axes
    U[0.02,0.10]) with k=0.01, rho_c=0.5 override the layers (centroid test).
    Dirichlet u=1 on z=0, flux-free elsewhere, u0=0 off the Dirichlet face,
    dt=5e-4, 100 steps, theta=0.5.
    """
    rng = np.random.default_rng(seed)
    cuts = np.sort(rng.choice(np.arange(1, n), size=n_layers - 1, replace=False))
    layer_of_k = np.searchsorted(cuts, np.arange(n), side="right")  # per element row k
    k_layer = np.where(layer_of_k % 2 == 0, 1.0, 1000.0)
    k = np.broadcast_to(k_layer[:, None, None], (n, n, n)).ravel().copy()
    rho_c = np.ones(n ** 3)
    centres = rng.random((n_pockets, 3))
    semi = rng.uniform(0.02, 0.10, (n_pockets, 3))
    cx, cy, cz = element_centroids(n, n, n)
    pocket = np.zeros(cx.shape, dtype=bool)
    for c, a in zip(centres, semi):
        pocket |= ((cx - c[0]) / a[0]) ** 2 + ((cy - c[1]) / a[1]) ** 2 + ((cz - c[2]) / a[2]) ** 2 <= 1.0
    k[pocket] = 0.01
    rho_c[pocket] = 0.5
    p = Problem(f"layered_cube_{n}", n, n, n, rho_c=rho_c, k=k,
                u0=np.zeros((n + 1) ** 3), dirichlet={4: 1.0}, flux={},
                flux_steps=-1, theta=0.5, dt=5e-4, nsteps=nsteps, rtol=1e-10)
    p.u0 = apply_dirichlet_values(p, p.u0)
    return p


def random_box(nx: int, ny: int, nz: int, seed: int, extent=(1.0, 1.0, 1.0),
               dirichlet=None, flux=None, theta=0.5, dt=1e-2, nsteps=3,
               flux_steps=-1, rtol=1e-12, contrast=(0.5, 2.0)) -> Problem:
    """Small box with uniform-random coefficients and random u0 (parity cases)."""
    rng = np.random.default_rng(seed)
    ne = nx * ny * nz
    lo, hi = contrast
    rho_c = rng.uniform(lo, hi, ne)
    k = rng.uniform(lo, hi, ne)
    u0 = rng.standard_normal((nx + 1) * (ny + 1) * (nz + 1))
    p = Problem(f"random_box_{nx}x{ny}x{nz}_s{seed}", nx, ny, nz,
                extent=tuple(extent), rho_c=rho_c, k=k, u0=u0,
                dirichlet=dict(dirichlet or {}), flux=dict(flux or {}),
                flux_steps=flux_steps, theta=theta, dt=dt, nsteps=nsteps, rtol=rtol)
    p.u0 = apply_dirichlet_values(p, p.u0)
    return p


@dataclass
class CorrosionPlate:
    """Synthetic stand-in for the corrosion-detection inverse problem of §5.3
    (the paper's gusset-plate geometry and camera data are not available).

    A steel plate of Lx x Ly x Lz mm (thickness Ly along y), front face y=0,
    rear face y=Ly; corrosion (oxide) grows in from the rear face with a
    parabolic profile in z of apex depth `depth`, constant along x. A Gaussian
    laser spot of power `power` W and width `beam` mm heats the front face for
    the whole period (nsteps of dt s, theta-scheme); the front face's
    temperatures at the end are the observation. Units: mm, s, W, K; steel
    k = 0.045 W/(mm K), rho*c = 3.6e-3 J/(mm^3 K); oxide k = 0.005,
    rho*c = 3.5e-3 (textbook values, not the paper's garbled ones)."""

    nx: int
    ny: int
    nz: int
    extent: tuple
    geom: dict
    flux_face: int
    flux_q: np.ndarray  # per element face of flux_face, lower tangential index fastest
    nsteps: int
    dt: float
    theta: float
    u0: float
    obs_face: int
    sigma: float
    quantum: float
    depth_true: float
    depth_max: float
    rtol: float
    seed: int
    origin: tuple = (0.0, 0.0, 0.0)

    def problem(self) -> Problem:
        """The forward problem with sound-steel coefficients (to be replaced)."""
        ne = self.nx * self.ny * self.nz
        nn = (self.nx + 1) * (self.ny + 1) * (self.nz + 1)
        return Problem(f"corrosion_plate_{self.nx}x{self.ny}x{self.nz}", self.nx, self.ny, self.nz,
                       origin=self.origin, extent=self.extent,
                       rho_c=np.full(ne, self.geom["rho_c_sound"]), k=np.full(ne, self.geom["k_sound"]),
                       u0=np.full(nn, self.u0), flux_steps=-1, theta=self.theta, dt=self.dt,
                       nsteps=self.nsteps, rtol=self.rtol)

    def camera(self, face_temps: np.ndarray) -> np.ndarray:
        """Camera model of §5.3: i.i.d. N(0, sigma^2) noise (seeded), then
        rounding to the camera's quantum."""
        rng = np.random.default_rng(self.seed + 1)
        noisy = np.asarray(face_temps) + rng.normal(0.0, self.sigma, len(face_temps))
        return np.round(noisy / self.quantum) * self.quantum

    def draws(self, niter: int, nchains: int, seed_offset: int = 0):
        """Metropolis-Hastings draws: (normals, uniforms), each (niter, nchains)."""
        rng = np.random.default_rng(self.seed + 2 + seed_offset)
        return rng.standard_normal((niter, nchains)), rng.uniform(0.0, 1.0, (niter, nchains))


def corrosion_plate(nx: int = 64, ny: int = 20, nz: int = 64, nsteps: int = 100, dt: float = 0.1,
                    seed: int = 5001, power: float = 10.0, beam: float = 2.0, sigma: float = 0.1,
                    quantum: float = 0.1, depth_true: float = 3.175, rtol: float = 1e-10) -> CorrosionPlate:
    """40 x 12.7 x 40 mm plate, corrosion apex at z = 20 mm with half-width
    15 mm, laser centred on the front face at (x, z) = (20, 20) mm; heating
    for nsteps*dt s (10 s by default, as in §5.3) from 0 K above ambient."""
    extent = (40.0, 12.7, 40.0)
    hx, hz = extent[0] / nx, extent[2] / nz
    xc = (np.arange(nx) + 0.5) * hx
    zc = (np.arange(nz) + 0.5) * hz
    X, Z = np.meshgrid(xc, zc)  # (nz, nx): x fastest, as the face's element order
    r2 = (X - 20.0) ** 2 + (Z - 20.0) ** 2
    q = power / (2.0 * np.pi * beam * beam) * np.exp(-r2 / (2.0 * beam * beam))
    geom = {"z0": 20.0, "half_width": 15.0, "rho_c_sound": 3.6e-3, "k_sound": 0.045,
            "rho_c_corr": 3.5e-3, "k_corr": 0.005}
    return CorrosionPlate(nx, ny, nz, extent, geom, 2, q.ravel(), nsteps, dt, 0.5, 0.0, 2, sigma, quantum,
                          depth_true, extent[1], rtol, seed)


WORKLOADS: List[str] = ["two_phase_cube", "inclusions_cube", "lognormal_cube",
                        "serving_request", "layered_cube", "corrosion_plate"]
