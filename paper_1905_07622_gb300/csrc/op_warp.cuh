// The factorised operator (see op.cuh) with the y direction held in
// registers: a warp-segment tile.
//
// A segment of SX lanes (SX divides 32) owns node columns x = i0-1+lx; each
// thread holds NY+2 consecutive y rows of its column and marches up the z
// levels. Forward x and the final x-sum use segment shuffles; forward y,
// forward z, scaling, inverse z, the face sums and inverse y all stay in the
// thread's registers, so the level loop has no shared memory and no barrier,
// and the NY rows are independent instruction streams. Outputs are lanes
// 1..SX-2 (the outer lanes only supply neighbours), rows 1..NY, levels
// [k0, k0+nzt): (SX-2) x NY x nzt nodes per segment.
#pragma once

#include "op.cuh"

namespace heat {

// Every lane of the segment must call this with the same tzl (the trip count
// of the level loop): shuffles span the segment. Segments with no tile pass
// active = false (they load and store nothing). Levels beyond the mesh are
// zero; outputs are clipped to the mesh.
template <class T, int SX, int NY, class Coef, class Fetch, class Value, class Out>
__device__ __forceinline__ void warp_tile_op(const Geo& g, const SimDev& s, const Coef* __restrict__ coef, bool active,
                                             int i0, int j0, int k0, int tzl, T sa, T sb, bool mask, Fetch&& fetch,
                                             Value&& value, Out&& out) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int NR = NY + 2;  // staged rows
  constexpr int NF = NY + 1;  // faces / element rows
  const int lx = (int)threadIdx.x % SX;
  const int c = i0 - 1 + lx;
  const bool col_in = active && c >= 0 && c <= g.nx;
  const bool out_lane = active && lx >= 1 && lx <= SX - 2 && c <= g.nx;
  const bool ecol = active && c >= 0 && c < g.nx;
  const bool dx = col_in && (((g.dir & 1u) && c == 0) || ((g.dir & 2u) && c == g.nx));
  // per-row flags (bit r): inside the mesh, on an x/y Dirichlet face, element row valid
  unsigned rin = 0u, rdxy = 0u, ein = 0u;
#pragma unroll
  for (int r = 0; r < NR; ++r) {
    const int j = j0 - 1 + r;
    const bool in = col_in && j >= 0 && j <= g.ny;
    if (in) rin |= 1u << r;
    if (in && (dx || ((g.dir & 4u) && j == 0) || ((g.dir & 8u) && j == g.ny))) rdxy |= 1u << r;
    if (r < NF && ecol && j >= 0 && j < g.ny) ein |= 1u << r;
  }
  const int nbase = c + g.px * (j0 - 1);  // node index of row 0 at level 0 (rows step by px)
  const int ebase = c + g.nx * (j0 - 1);  // element index of element row 0 at level 0
  const int estride = g.nx * g.ny, pxy = g.pxy, gnz = g.nz, px = g.px, enx = g.nx;
  const bool dz0 = (g.dir & 16u) != 0, dz1 = (g.dir & 32u) != 0;
  // With lam_q and lam'_q = lam_{q+4} (the two z-Walsh indices of an xy index
  // q), the face sum and the element's top half are
  //   G_q = Tp_q + A_q Fp_q + B_q F_q,  Tn_q = B_q Fp_q + A_q F_q,
  //   A_q = lam_q + lam'_q,  B_q = lam_q - lam'_q,
  // and A_q, B_q are linear in (rho_c, k) with these coefficients:
  T am[4], ak[4], bm[4], bk[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    am[q] = sa * (lam_m<T>(s, q) + lam_m<T>(s, q + 4));
    ak[q] = sb * (lam_k<T>(s, q) + lam_k<T>(s, q + 4));
    bm[q] = sa * (lam_m<T>(s, q) - lam_m<T>(s, q + 4));
    bk[q] = sb * (lam_k<T>(s, q) - lam_k<T>(s, q + 4));
  }
  using Raw = decltype(fetch(0, false));
  using CoefT = typename std::remove_cv<typename std::remove_reference<decltype(coef[0])>::type>::type;
  Raw raw[NR];
  CoefT cf[NF];
  const unsigned rstat = rin & ~(mask ? rdxy : 0u);  // rows that can be live at any level
  auto fetch_level = [&](int L) {
    const bool lev = L >= 0 && L <= gnz && !(mask && ((dz0 && L == 0) || (dz1 && L == gnz)));
    const unsigned lv = lev ? rstat : 0u;
    const int off = nbase + L * pxy;
#pragma unroll
    for (int r = 0; r < NR; ++r) raw[r] = fetch(off + r * px, (lv >> r) & 1u);
  };
  auto fetch_coef = [&](int E) {
    const bool ek = E >= 0 && E < gnz;
#pragma unroll
    for (int r = 0; r < NF; ++r) {
      CoefT z;
      z.x = T(0);
      z.y = T(0);
      cf[r] = (ek && ((ein >> r) & 1u)) ? coef[ebase + r * enx + E * estride] : z;
    }
  };
  fetch_level(k0 - 1);
  fetch_coef(k0 - 1);
  T Fp[NF][4], Tp[NF][4], vprev[NY];
#pragma unroll
  for (int r = 0; r < NF; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      Fp[r][q] = T(0);
      Tp[r][q] = T(0);
    }
#pragma unroll
  for (int r = 0; r < NY; ++r) vprev[r] = T(0);

  for (int t = 0; t <= tzl + 1; ++t) {
    const int L = k0 - 1 + t;
    T v[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = value(raw[r]);
    if (t <= tzl) fetch_level(L + 1);  // next level's loads in flight during this one
    // forward x (edges of each row) and forward y (faces between rows)
    T e0[NR], e1[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const T vr = __shfl_down_sync(FULL, v[r], 1, SX);
      e0[r] = v[r] + vr;
      e1[r] = v[r] - vr;
    }
    T F[NF][4];
#pragma unroll
    for (int r = 0; r < NF; ++r) {
      F[r][0] = e0[r] + e0[r + 1];
      F[r][1] = e1[r] + e1[r + 1];
      F[r][2] = e0[r] - e0[r + 1];
      F[r][3] = e1[r] - e1[r + 1];
    }
    if (t >= 1) {
      // elements (c, j0-1+r, L-1) between face levels L-1 and L
      T G[NF][4];
#pragma unroll
      for (int r = 0; r < NF; ++r) {
        const T rc = cf[r].x, kc = cf[r].y;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const T A = rc * am[q] + kc * ak[q], B = rc * bm[q] + kc * bk[q];
          G[r][q] = Tp[r][q] + A * Fp[r][q] + B * F[r][q];
          Tp[r][q] = B * Fp[r][q] + A * F[r][q];
        }
      }
      if (t <= tzl) fetch_coef(L);
      if (t >= 2) {
        // node level L-1 is complete: inverse y, inverse x, x-sum
        const int lv = L - 1;
        const bool lvin = lv <= gnz;
        const bool dzl = (dz0 && lv == 0) || (dz1 && lv == gnz);
#pragma unroll
        for (int r = 1; r <= NY; ++r) {
          const T g0 = (G[r][0] + G[r][2]) + (G[r - 1][0] - G[r - 1][2]);
          const T g1 = (G[r][1] + G[r][3]) + (G[r - 1][1] - G[r - 1][3]);
          const T nl = g0 + g1, nr = g0 - g1;
          const T from_left = __shfl_up_sync(FULL, nr, 1, SX);
          if (out_lane && lvin && ((rin >> r) & 1u)) {
            const bool dir = ((rdxy >> r) & 1u) || dzl;
            out(nbase + r * px + lv * pxy, dir, nl + from_left, vprev[r - 1]);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NY; ++r) vprev[r] = v[r + 1];
#pragma unroll
    for (int r = 0; r < NF; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) Fp[r][q] = F[r][q];
  }
}

}  // namespace heat
