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
// tile_op. opA(mask, fetch, value, out) is the same with (sa, sb) = (1/dt,
// theta), the A operator, which may read the per-element coefficients
// precomputed for it. part receives r.P^-1 r (FP64), b.P^-1 b and
// r32.P^-1 r32 (each thread's terms summed in FP32 first).
// ---------------------------------------------- the A operator, precomputed

// The A operator's Walsh-pair coefficients of one element (SimDev::acoef):
// four float4 words, A_0..A_3 then B_0..B_3, as FP64 pairs (T = double) or
// as (hi, lo) float pairs (T = DF).
template <class T> struct PreAB;
template <> struct PreAB<double> {
  static __device__ __forceinline__ void get(const float4 (&w)[4], double (&A)[4], double (&B)[4]) {
    const double2 a01 = *reinterpret_cast<const double2*>(&w[0]), a23 = *reinterpret_cast<const double2*>(&w[1]);
    const double2 b01 = *reinterpret_cast<const double2*>(&w[2]), b23 = *reinterpret_cast<const double2*>(&w[3]);
    A[0] = a01.x; A[1] = a01.y; A[2] = a23.x; A[3] = a23.y;
    B[0] = b01.x; B[1] = b01.y; B[2] = b23.x; B[3] = b23.y;
  }
};
template <> struct PreAB<DF> {
  static __device__ __forceinline__ void get(const float4 (&w)[4], DF (&A)[4], DF (&B)[4]) {
    A[0] = DF(w[0].x, w[0].y); A[1] = DF(w[0].z, w[0].w); A[2] = DF(w[1].x, w[1].y); A[3] = DF(w[1].z, w[1].w);
    B[0] = DF(w[2].x, w[2].y); B[1] = DF(w[2].z, w[2].w); B[2] = DF(w[3].x, w[3].y); B[3] = DF(w[3].z, w[3].w);
  }
};

// RegSrc (op_warp.cuh) with each element row's coefficients read as a PreRec
// from SimDev::acoef: the warp-segment march of the A operator with its
// per-element coefficients precomputed.
template <class T, int NY, class Fetch, class Value>
struct PreRegSrc {
  static constexpr int NR = NY + 2, NF = NY + 1;
  using Raw = decltype(std::declval<Fetch&>()(0, false));
  const float4* __restrict__ pre;
  Fetch& fetch;
  Value& value;
  int k0;
  Raw raw[NR];
  PreRec cf[NF];

  __device__ __forceinline__ PreRegSrc(const float4* p, Fetch& f, Value& v, int k0_)
      : pre(p), fetch(f), value(v), k0(k0_) {}
  __device__ __forceinline__ void load_nodes(const LaneGeo<NY>& lg, int L) {
    const unsigned lv = lg.live_rows(L);
    const int off = lg.nbase + L * lg.pxy;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int m = off + r * lg.px;
      raw[r] = fetch(m, ((lv >> r) & 1u) && HEAT_INDEX_OK(lg.sc, m, lg.nn));
    }
  }
  __device__ __forceinline__ void load_coef(const LaneGeo<NY>& lg, int E) {
    const unsigned le = lg.live_elems(E);
#pragma unroll
    for (int r = 0; r < NF; ++r) {
      const int e = lg.ebase + r * lg.enx + E * lg.estride;
      if (((le >> r) & 1u) && HEAT_INDEX_OK(lg.sc, e, lg.ne)) {
        const float4* p = pre + 4 * (long long)e;
#pragma unroll
        for (int w = 0; w < 4; ++w) cf[r].w[w] = __ldg(p + w);
      } else {
#pragma unroll
        for (int w = 0; w < 4; ++w) cf[r].w[w] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  __device__ __forceinline__ void prologue(const LaneGeo<NY>& lg, int) {
    load_nodes(lg, k0 - 1);
    load_coef(lg, k0 - 1);
  }
  __device__ __forceinline__ void level(const LaneGeo<NY>& lg, int t, int tzl, T v[NR]) {
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = value(raw[r]);
    if (t <= tzl) load_nodes(lg, k0 + t);
  }
  __device__ __forceinline__ const PreRec& coef_row(int, int r) const { return cf[r]; }
  __device__ __forceinline__ void after_elements(const LaneGeo<NY>& lg, int t, int tzl) {
    if (t <= tzl) load_coef(lg, k0 - 1 + t);
  }
};

// tile_op (op.cuh) for the A operator on trilinear boxes, with each element's
// coefficients A_q, B_q read from SimDev::acoef instead of formed from
// (rho_c, k): the same factorised product and the same contract, about a
// third less arithmetic per node in double-float.
template <class T, int SX, int SY, class Fetch, class Value, class Out>
__device__ __forceinline__ void tile_op_pre(const Geo& g, const SimDev& s, int i0, int j0, int k0, int nzt, bool mask,
                                            TileSmem<T, SX, SY>& sh, Fetch&& fetch, Value&& value, Out&& out) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lx = (int)threadIdx.x % SX, ly = (int)threadIdx.x / SX;
  const int i = i0 - 1 + lx, j = j0 - 1 + ly;
  const bool outcol = lx >= 1 && ly >= 1 && i <= g.nx && j <= g.ny;
  const bool lastx = lx == SX - 1, lasty = ly == SY - 1;
  const bool elem_col = i >= 0 && j >= 0 && i < g.nx && j < g.ny;
  const Col c00(g, i, j), c10(g, i + 1, j), c01(g, i, j + 1), c11(g, i + 1, j + 1);
  const int estride = g.nx * g.ny;
  const int ebase = elem_col ? i + g.nx * j : 0;
  const long long nn_all = (long long)g.pxy * (g.nz + 1), ne_all = (long long)estride * g.nz;
  (void)nn_all;
  (void)ne_all;
  const int gnz = g.nz, pxy = g.pxy;
  const bool dz0 = (g.dir & 16u) != 0, dz1 = (g.dir & 32u) != 0;
  using Raw = decltype(fetch(0, false));
  auto fetch_level = [&](int L, Raw& r00, Raw& r10, Raw& r01, Raw& r11) {
    const bool kin = L >= 0 && L <= gnz;
    const bool dk = mask && ((dz0 && L == 0) || (dz1 && L == gnz));
    const int off = L * pxy;
    auto live = [&](const Col& c) {
      return c.in && kin && !dk && !(mask && c.dxy) && HEAT_INDEX_OK(s.sc, c.base + off, nn_all);
    };
    r00 = fetch(c00.base + off, live(c00));
    if (lastx) r10 = fetch(c10.base + off, live(c10));
    if (lasty) r01 = fetch(c01.base + off, live(c01));
    if (lastx && lasty) r11 = fetch(c11.base + off, live(c11));
  };
  struct Rec {
    float4 w[4];
  };
  auto pre_of = [&](int E) -> Rec {  // element (i, j, E); zero outside the mesh
    Rec r;
    if (elem_col && E >= 0 && E < gnz && HEAT_INDEX_OK(s.sc, ebase + estride * E, ne_all)) {
      const float4* p = s.acoef + 4 * ((long long)ebase + (long long)estride * E);
#pragma unroll
      for (int w = 0; w < 4; ++w) r.w[w] = __ldg(p + w);
    } else {
#pragma unroll
      for (int w = 0; w < 4; ++w) r.w[w] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    return r;
  };
  Raw r00 = fetch(0, false), r10 = r00, r01 = r00, r11 = r00;
  fetch_level(k0 - 1, r00, r10, r01, r11);
  Rec pnext = pre_of(k0 - 1);
  T Fp[4] = {T(0), T(0), T(0), T(0)};
  T Tp[4] = {T(0), T(0), T(0), T(0)};
  T rj[2] = {T(0), T(0)};
  T up[2] = {T(0), T(0)};
  T vh0 = T(0), vh1 = T(0), vh2 = T(0);
  const int ltop = k0 + nzt;
  for (int L = k0 - 1; L <= ltop + 1; ++L) {
    const int buf = L & 1;
    T e0 = T(0), e1 = T(0), a0 = T(0), a1 = T(0);
    vh2 = vh1;
    vh1 = vh0;
    vh0 = T(0);
    if (L <= ltop) {
      const T v = value(r00);
      T vr = __shfl_down_sync(FULL, v, 1, SX);
      if (lastx) vr = value(r10);
      e0 = v + vr;
      e1 = v - vr;
      vh0 = v;
      const T w = lasty ? value(r01) : T(0);
      T wr = __shfl_down_sync(FULL, w, 1, SX);
      if (lastx && lasty) wr = value(r11);
      a0 = w + wr;
      a1 = w - wr;
      sh.E[buf][ly][lx] = {e0, e1};
      if (L + 1 <= ltop) fetch_level(L + 1, r00, r10, r01, r11);
    }
    sh.F[buf][ly][lx] = {up[0], up[1]};
    __syncthreads();
    if (L >= k0 + 2) {
      T g0 = rj[0], g1 = rj[1];
      if (ly >= 1) {
        const auto f = sh.F[buf][ly - 1][lx];
        g0 += f.x;
        g1 += f.y;
      }
      const T nl = g0 + g1, nr = g0 - g1;
      const T from_left = __shfl_up_sync(FULL, nr, 1, SX);
      const int lv = L - 2;
      if (outcol && lv <= gnz && HEAT_INDEX_OK(s.sc, c00.base + lv * pxy, nn_all)) {
        const bool dir = c00.dxy || (dz0 && lv == 0) || (dz1 && lv == gnz);
        out(c00.base + lv * pxy, dir, nl + from_left, vh2);
      }
    }
    if (L <= ltop) {
      if (!lasty) {
        const auto eu = sh.E[buf][ly + 1][lx];
        a0 = eu.x;
        a1 = eu.y;
      }
      const T Fc[4] = {e0 + a0, e1 + a1, e0 - a0, e1 - a1};
      if (L >= k0) {
        // element (i, j, L-1): its coefficients, then the next level's in flight
        T A[4], B[4];
        PreAB<T>::get(pnext.w, A, B);
        pnext = pre_of(L);
        T G[4], Tn[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          G[q] = Tp[q] + A[q] * Fp[q] + B[q] * Fc[q];
          Tn[q] = B[q] * Fp[q] + A[q] * Fc[q];
        }
        rj[0] = G[0] + G[2];
        rj[1] = G[1] + G[3];
        up[0] = G[0] - G[2];
        up[1] = G[1] - G[3];
#pragma unroll
        for (int q = 0; q < 4; ++q) Tp[q] = Tn[q];
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) Fp[q] = Fc[q];
    }
  }
  __syncthreads();
}

template <int P, class Op, class OpA>
__device__ __forceinline__ void open_passes(const SimDev& s, const Ctl& c, const Geo& g, int phase,
                                            double (&part)[3], Op&& op, OpA&& opA) {
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
  // r32^T P^-1 r32, the restarted inner solve's delta: summed per thread in
  // FP32 like the inner iterations' norms, FP64 from the block sum on
  float acc2 = 0.f;
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
              acc2 += r32 * r32 * s.pinv32[m];
              part[0] += rn * rn * pinv[m];
            }
          }
        });
    // pass 2: x0 = 2u^{n-1} - u^{n-2} (u^{n-1} on the first step), r = b - A' x0
    if (!use_y) opA(true,
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
            acc2 += r32 * r32 * s.pinv32[m];
          }
          part[0] += rn * rn * pinv[m];
        });
  } else if (phase == PH_OUTER) {
    // x64 <- x64 + e32 (into the spare slot), r = b - A' x64 in FP64
    const double* __restrict__ x = s.vec64[c.ix];
    double* __restrict__ xa = s.vec64[c.ixa];
    double* __restrict__ ya = s.yv[c.ixa];  // A' x64, used by the next step if this one closes
    const float* __restrict__ e32 = s.e32;
    opA(true,
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
          acc2 += r32 * r32 * s.pinv32[m];
          part[0] += rn * rn * pinv[m];
        });
  } else {  // PH_RESID (FP64): r = b - A' x, x already advanced by k_update
    const double* __restrict__ x = s.vec64[c.ix];
    double* __restrict__ r = s.r;
    opA(true,
        [&](int m, bool live) -> double { return live ? x[m] : 0.0; }, ident,
        [&](int m, bool dir, TO yo, TO) {
          const double y = to_d(yo);
          const double rn = dir ? 0.0 : b[m] - y;
          r[m] = rn;
          part[0] += rn * rn * pinv[m];
        });
  }
  part[2] += (double)acc2;
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
    auto op = [&](TO sa, TO sb, bool mask, auto&& fetch, auto&& value, auto&& out) {
      tile_op_e<E, TO, SX, SY>(g, s, s.coef, tc.i0, tc.j0, tc.k0, tc.nzt, sa, sb, mask, sh, fetch, value, out);
    };
    auto opA = [&](bool mask, auto&& fetch, auto&& value, auto&& out) {
      if constexpr (E == E_Q1) {
        if (s.acoef) {
          tile_op_pre<TO, SX, SY>(g, s, tc.i0, tc.j0, tc.k0, tc.nzt, mask, sh, fetch, value, out);
          return;
        }
      }
      op(TO(s.inv_dt), TO(s.theta), mask, fetch, value, out);
    };
    open_passes<P>(s, c, g, phase, part, op, opA);
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
    auto op = [&](TO sa, TO sb, bool mask, auto&& fetch, auto&& value, auto&& out) {
      warp_tile_op_e<E_Q1, TO, SX, NY>(g, s, s.coef, active, tx * (SX - 2), ty * NY, tz * s.o_tz, s.o_tz, sa, sb,
                                       mask, fetch, value, out);
    };
    auto opA = [&](bool mask, auto&& fetch, auto&& value, auto&& out) {
      if (s.acoef) {
        const LaneGeo<NY> lg(g, active, (int)threadIdx.x % SX, SX, tx * (SX - 2), ty * NY, mask, s.sc);
        PreRegSrc<TO, NY, typename std::remove_reference<decltype(fetch)>::type,
                  typename std::remove_reference<decltype(value)>::type>
            src(s.acoef, fetch, value, tz * s.o_tz);
        warp_tile_march<TO, SX, NY>(lg, s, src, s.o_tz, TO(s.inv_dt), TO(s.theta), out);
        return;
      }
      op(TO(s.inv_dt), TO(s.theta), mask, fetch, value, out);
    };
    open_passes<P>(s, c, g, phase, part, op, opA);
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
