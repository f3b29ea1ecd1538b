// The step-start and refinement passes of the solver (k_open, its
// warp-segment form k_open_w) and the stored-product kernel k_product: the
// operator passes that form the right-hand side of §3.1's step system, the
// first residual of each step, Algorithm 1's periodic true residual on the
// FP64 path and the refinement's true residual on the FP32 paths. See
// tile_kernels.cuh for the iteration kernels they hand over to.
#pragma once

#include "tile_kernels.cuh"

namespace heat {

// ------------------------------------------------------------------ k_open

struct D2 {
  double a, b;
};

// Arithmetic of the operator passes of k_open: FP64 on the FP64 path. On the
// FP32 paths the passes form the refinement's right-hand side and true
// residual, and run in double-float (df.cuh): about 48 bits, several times the
// FP64 pass's speed on this GPU; the vectors and sums stay FP64.
template <int P> using OpenT = typename std::conditional<P == P_FP64, double, DF>::type;

// The operator passes of a step's start and of the refinement, for one work
// item: op(sa, sb, mask, fetch, value, out) runs one operator pass
// sum_e (sa rho_c M_e + sb k K_e) over the caller's tile (a block tile in
// k_open, a warp segment in k_open_w) with the fetch/value/out contract of
// tile_op. part receives r.P^-1 r (FP64), b.P^-1 b and r32.P^-1 r32.
template <int P, class Op>
__device__ __forceinline__ void open_passes(const SimDev& s, const Ctl& c, const Geo& g, int phase,
                                            double (&part)[3], Op&& op) {
  using TO = OpenT<P>;
  const double* __restrict__ pinv = s.pinv;
  double* __restrict__ b = s.b;
  const TO inv_dt = TO(s.inv_dt), theta = TO(s.theta), theta_m1 = TO(s.theta - 1.0);
  // the FP32 residual goes to the current slot of the fused iteration (slot 0 otherwise)
  float* __restrict__ r32out = s.fused ? s.rc32[c.cgs] : s.r32;
  // value of a Dirichlet node from its index (faces only, so rarely called)
  auto dval = [&](int m) -> double {
    const int kk = m / g.pxy, rem = m - kk * g.pxy, jj = rem / g.px;
    return dirichlet_value(s, rem - jj * g.px, jj, kk);
  };
  auto ident = [](double v) { return v; };
  if (phase == PH_OPEN) {
    const double* __restrict__ u1 = s.vec64[c.iu1];
    const double* __restrict__ u2 = s.vec64[c.iu2];
    double* __restrict__ x = s.vec64[c.ix];
    const bool hp = c.have_prev != 0;
    const bool flux_on = s.flux_steps < 0 || c.step + 1 <= s.flux_steps;
    const double* __restrict__ F = s.F;
    const double* __restrict__ lift = s.zlift;
    // On the FP32 paths the previous steps closed with an FP64 residual pass
    // that also stored A' U^{n-1} (and A' U^{n-2}); then A' x0 = 2 A' U^{n-1}
    // - A' U^{n-2} needs no operator pass and r is formed in pass 1.
    const bool use_y =
        P != P_FP64 && ((c.y_valid >> c.iu1) & 1) && (!hp || ((c.y_valid >> c.iu2) & 1));
    const double* __restrict__ y1 = s.yv[c.iu1];
    const double* __restrict__ y2 = s.yv[c.iu2];
    // pass 1: b = L u^{n-1} + F^n - A_{.D} g (free rows), g (Dirichlet rows)
    op(inv_dt, theta_m1, false,
        [&](int m, bool live) -> double { return live ? u1[m] : 0.0; }, ident,
        [&](int m, bool dir, TO yo, TO) {
          const double y = to_d(yo);
          if (dir) {
            b[m] = dval(m);
            if (use_y) {
              x[m] = dval(m);
              r32out[m] = 0.f;
            }
          } else {
            const double bn = y + (flux_on ? F[m] : 0.0) - lift[m];
            b[m] = bn;
            part[1] += bn * bn * pinv[m];
            if (use_y) {
              const double v = u1[m];  // the staged input, read back in FP64
              x[m] = hp ? 2.0 * v - u2[m] : v;
              const double rn = bn - (hp ? 2.0 * y1[m] - y2[m] : y1[m]);
              const float r32 = (float)rn;
              r32out[m] = r32;
              part[2] += (double)r32 * (double)r32 * (double)s.pinv32[m];
              part[0] += rn * rn * pinv[m];
            }
          }
        });
    // pass 2: x0 = 2u^{n-1} - u^{n-2} (u^{n-1} on the first step), r = b - A' x0
    if (!use_y) op(inv_dt, theta, true,
        [&](int m, bool live) -> D2 {
          if (!live) return {0.0, 0.0};
          return {u1[m], hp ? u2[m] : u1[m]};
        },
        [](const D2& r) { return 2.0 * r.a - r.b; },
        [&](int m, bool dir, TO yo, TO) {
          const double y = to_d(yo);
          double rn = 0.0;
          if (dir) {
            x[m] = dval(m);
          } else {
            x[m] = hp ? 2.0 * u1[m] - u2[m] : u1[m];  // the staged input, formed again in FP64
            rn = b[m] - y;
          }
          if (P == P_FP64) {
            s.r[m] = rn;
          } else {
            const float r32 = (float)rn;
            r32out[m] = r32;
            part[2] += (double)r32 * (double)r32 * (double)s.pinv32[m];
          }
          part[0] += rn * rn * pinv[m];
        });
  } else if (phase == PH_OUTER) {
    // x64 <- x64 + e32 (into the spare slot), r = b - A' x64 in FP64
    const double* __restrict__ x = s.vec64[c.ix];
    double* __restrict__ xa = s.vec64[c.ixa];
    double* __restrict__ ya = s.yv[c.ixa];  // A' x64, used by the next step if this one closes
    const float* __restrict__ e32 = s.e32;
    op(inv_dt, theta, true,
        [&](int m, bool live) -> D2 {
          if (!live) return {0.0, 0.0};
          return {x[m], (double)e32[m]};
        },
        [](const D2& r) { return r.a + r.b; },
        [&](int m, bool dir, TO yo, TO) {
          const double y = to_d(yo);
          double rn = 0.0;
          if (dir) {
            xa[m] = dval(m);
          } else {
            xa[m] = x[m] + (double)e32[m];  // the staged input, formed again in FP64
            ya[m] = y;
            rn = b[m] - y;
          }
          const float r32 = (float)rn;
          r32out[m] = r32;
          part[2] += (double)r32 * (double)r32 * (double)s.pinv32[m];
          part[0] += rn * rn * pinv[m];
        });
  } else {  // PH_RESID (FP64): r = b - A' x, x already advanced by k_update
    const double* __restrict__ x = s.vec64[c.ix];
    double* __restrict__ r = s.r;
    op(inv_dt, theta, true,
        [&](int m, bool live) -> double { return live ? x[m] : 0.0; }, ident,
        [&](int m, bool dir, TO yo, TO) {
          const double y = to_d(yo);
          const double rn = dir ? 0.0 : b[m] - y;
          r[m] = rn;
          part[0] += rn * rn * pinv[m];
        });
  }
}

// The last block's update of a simulation's scalars after its open passes
// (tot as open_passes' part, summed over the simulation's items).
template <int P>
__device__ __forceinline__ void open_finish(const SimDev& s, int phase, const double (&tot)[3]) {
  SimScalars* sc = s.sc;
  sc->count = 0;
  if (phase == PH_RESID) {
    // Either the periodic true residual (an iteration of Algorithm 1 whose
    // r comes from b - A x) or the confirmation of a converged recurrence
    // residual, which keeps the iteration's beta and is not counted.
    const double dn = tot[0];
    const bool confirm = sc->confirm != 0;
    sc->confirm = 0;
    if (s.cheb_m < 2) {  // a Chebyshev pass forms delta = r^T z and beta instead
      if (!confirm) sc->beta = dn / sc->delta;
      sc->delta = dn;
    }
    if (!confirm) {
      sc->iter += 1;
      sc->iter_step += 1;
    }
    if (!isfinite(dn)) fail(sc, ST_NONFINITE);
    else if (dn <= sc->thresh) close_step(s, sc, dn);
    else if (sc->iter_step >= s.max_iter) fail(sc, ST_NOT_CONVERGED);
    else enter_iter(s, sc);
  } else {
    if (phase == PH_OPEN) {
      sc->delta_b = tot[1];
      sc->thresh = s.rtol * s.rtol * tot[1];
      sc->iter_step = 0;
      sc->outer = 0;
    } else {
      const int t2 = sc->ix;  // the refined iterate now lives in the spare slot
      sc->ix = sc->ixa;
      sc->ixa = t2;
      sc->outer += 1;
      sc->iter_step += 1;  // the FP64 true residual counts as an iteration
    }
    sc->iter = 0;
    sc->restart = 1;
    sc->confirm = 0;
    if (!s.fused) sc->cgs = 0;
    if (!isfinite(tot[0]) || !isfinite(tot[1]) || !isfinite(tot[2])) {
      fail(sc, ST_NONFINITE);
    } else if (P == P_FP64) {
      sc->delta = tot[0];
      if (tot[0] <= sc->thresh) close_step(s, sc, tot[0]);
      else enter_iter(s, sc);
    } else {
      sc->delta_out = tot[0];
      sc->delta = tot[2];
      const bool plain_done = (P == P_FP32_PLAIN && phase == PH_OUTER);
      if (tot[0] <= sc->thresh || plain_done || tot[2] <= 0.0) {
        close_step(s, sc, tot[0], phase == PH_OUTER);
      } else if (sc->outer >= s.max_outer || sc->iter_step >= s.max_iter) {
        fail(sc, ST_NOT_CONVERGED);
      } else {
        // The inner solve reduces its residual by inner_rtol, or only as far
        // as the outer target needs (to half the target residual norm), so
        // the next sweep's FP64 residual can close the step.
        sc->thresh_in = (P == P_FP32_PLAIN) ? sc->thresh
                                            : fmax(s.inner_rtol * s.inner_rtol * tot[2], 0.25 * sc->thresh);
        enter_iter(s, sc);
      }
    }
  }
}

template <int P, int SX, int SY, int E = E_Q1>
__global__ void __launch_bounds__(SX* SY) k_open(const SimDev* __restrict__ sims, const int2* __restrict__ work,
                                                 const int* __restrict__ nwork_p) {
  using TO = OpenT<P>;
  __shared__ OpSmem<E, TO, SX, SY> sh;
  __shared__ double red[3 * 32];
  __shared__ ItemCache cache;
  int cur = -1;
  bool dep = false;
  allow_next_launch();
  const int nwork = *nwork_p;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 wi = work[w];
    cache_sim(sims, wi.x, cache, cur, dep);
    const SimDev& s = cache.s;
    const Ctl& c = cache.c;
    const int phase = c.phase;
    const bool act = phase == PH_OPEN || (P != P_FP64 && phase == PH_OUTER) || (P == P_FP64 && phase == PH_RESID);
    if (!act) continue;
    const Geo g(s);
    const TileCoords tc = tile_coords<SX, SY>(s, wi.y);
    double part[3] = {0.0, 0.0, 0.0};
    open_passes<P>(s, c, g, phase, part, [&](TO sa, TO sb, bool mask, auto&& fetch, auto&& value, auto&& out) {
      tile_op_e<E, TO, SX, SY>(g, s, s.coef, tc.i0, tc.j0, tc.k0, tc.nzt, sa, sb, mask, sh, fetch, value, out);
    });
    double tot[3];
    if (finish_item<double, 3>(s, wi.y, s.ntiles, part, tot, red)) open_finish<P>(s, phase, tot);
  }
}

// k_open with the operator in the warp-segment march (op_warp.cuh): a work
// item is a group of 32 * WARPS / SX segment tiles of (SX-2) x NY x o_tz
// nodes; no block barrier in the level loop, NY independent rows per lane.
// Same passes, arithmetic and results contract as k_open.
template <int P, int SX, int NY, int WARPS, int MINB>
__global__ void __launch_bounds__(32 * WARPS, MINB) k_open_w(const SimDev* __restrict__ sims,
                                                             const int2* __restrict__ work,
                                                             const int* __restrict__ nwork_p) {
  using TO = OpenT<P>;
  constexpr int SPC = WARPS * (32 / SX);  // segment tiles per work item
  __shared__ double red[3 * 32];
  __shared__ ItemCache cache;
  int cur = -1;
  bool dep = false;
  allow_next_launch();
  const int nwork = *nwork_p;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 wi = work[w];
    cache_sim(sims, wi.x, cache, cur, dep);
    const SimDev& s = cache.s;
    const Ctl& c = cache.c;
    const int phase = c.phase;
    const bool act = phase == PH_OPEN || (P != P_FP64 && phase == PH_OUTER) || (P == P_FP64 && phase == PH_RESID);
    if (!act) continue;
    const Geo g(s);
    const int tile = wi.y * SPC + (int)threadIdx.x / SX;
    const bool active = tile < s.o_ntiles;
    const int tx = tile % s.o_ntx, rem = tile / s.o_ntx, ty = rem % s.o_nty, tz = rem / s.o_nty;
    double part[3] = {0.0, 0.0, 0.0};
    open_passes<P>(s, c, g, phase, part, [&](TO sa, TO sb, bool mask, auto&& fetch, auto&& value, auto&& out) {
      warp_tile_op_e<E_Q1, TO, SX, NY>(g, s, s.coef, active, tx * (SX - 2), ty * NY, tz * s.o_tz, s.o_tz, sa, sb,
                                       mask, fetch, value, out);
    });
    double tot[3];
    if (finish_item<double, 3>(s, wi.y, s.o_items, part, tot, red)) open_finish<P>(s, phase, tot);
  }
}

// --------------------------------------------------------------- k_product

// y = A' u on the free rows (Dirichlet rows and columns masked), with the
// tile operator of k_open's residual passes, so the values are bitwise those
// such a pass computes for the same u: a node's value does not depend on
// where its tile starts. One block per tile of (SX-1) x (SY-1) node columns
// and tz levels. Restores the stored products A' U^{n-1}, A' U^{n-2} of a
// resumed simulation (see k_open, phase OPEN).
template <int SX, int SY, int E = E_Q1>
__global__ void __launch_bounds__(SX* SY) k_product(const SimDev* __restrict__ sd, const double* __restrict__ u,
                                                     double* __restrict__ y, int ntx, int nty, int tz) {
  using TO = OpenT<P_FP32_REFINED>;  // the arithmetic of k_open's passes on the FP32 paths
  __shared__ OpSmem<E, TO, SX, SY> sh;
  const SimDev& s = *sd;
  const Geo g(s);
  const int t = blockIdx.x;
  const int tx = t % ntx, rem = t / ntx, ty = rem % nty, tk = rem / nty;
  const int k0 = tk * tz;
  const int nzt = min(tz, s.nz + 1 - k0);
  tile_op_e<E, TO, SX, SY>(
      g, s, s.coef, tx * (SX - 1), ty * (SY - 1), k0, nzt, TO(s.inv_dt), TO(s.theta), true, sh,
      [&](int m, bool live) -> double { return live ? u[m] : 0.0; }, [](double v) { return v; },
      [&](int m, bool dir, TO yv, TO) {
        if (!dir) y[m] = to_d(yv);
      });
}

}  // namespace heat
