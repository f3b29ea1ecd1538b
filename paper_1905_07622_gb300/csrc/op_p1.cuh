// The assembly-free operator on six-tetrahedra boxes (heat.h HEAT_ELEM_P1),
// in the tile form of op.cuh: the same contract as tile_op (fetch / value /
// out, tile shape, masking), so every phase-gated kernel can run either
// element.
//
// The box matrices M', K' of the split (six monotone corner paths 0 -> e_a ->
// e_a+e_b -> 7) have no reflection symmetry, so the Walsh factorisation of
// the trilinear operator does not apply. Instead the block stages node
// levels and element layers of its tile in shared memory and each output
// node gathers row c of the matrices of its <= 8 boxes (c its local corner
// in each), over the corners it shares a tetrahedron with: 46 mass entries
// and 32 stiffness entries per node, 15 distinct neighbours.
#pragma once

#include "op.cuh"

namespace heat {

template <class T, int SX, int SY>
struct TileSmemP1 {
  T X[4][SY + 1][SX + 1];                 // node levels, a ring of 4
  typename Pair<T>::type C[3][SY][SX];    // element layers (rho_c, k), a ring of 3
  T wm[64], wk[64];                       // sa * M', sb * K'
};

// Ring slots (levels start at -1, element layers at -2).
__device__ __forceinline__ int p1_xslot(int L) { return (L + 4) & 3; }
__device__ __forceinline__ int p1_cslot(int E) { return (E + 3) % 3; }

// Thread (lx, ly) stages node column (i0-1+lx, j0-1+ly), the tile's last x
// column and y row also the columns one further on, and element column
// (i0-1+lx, j0-1+ly). Level L's output (threads with lx, ly >= 1) needs node
// levels L-1..L+1 and element layers L-1 and L; iteration L of the march
// stores node level L and element layer L-1, then outputs level L-1. With 4
// node slots and 3 layer slots, one barrier per level keeps a writer from
// overtaking a reader.
template <class T, int SX, int SY, class Coef, class Fetch, class Value, class Out>
__device__ __forceinline__ void tile_op_p1(const Geo& g, const SimDev& s, const Coef* __restrict__ coef, int i0,
                                           int j0, int k0, int nzt, T sa, T sb, bool mask,
                                           TileSmemP1<T, SX, SY>& sh, Fetch&& fetch, Value&& value, Out&& out) {
  const int lx = (int)threadIdx.x % SX, ly = (int)threadIdx.x / SX;
  const int i = i0 - 1 + lx, j = j0 - 1 + ly;
  const bool outcol = lx >= 1 && ly >= 1 && i <= g.nx && j <= g.ny;
  const bool lastx = lx == SX - 1, lasty = ly == SY - 1;
  const bool elem_col = i >= 0 && j >= 0 && i < g.nx && j < g.ny;
  const Col c00(g, i, j), c10(g, i + 1, j), c01(g, i, j + 1), c11(g, i + 1, j + 1);
  const auto* w = p1_weights<T>(s);
  for (int t = (int)threadIdx.x; t < 64; t += (int)blockDim.x) {
    sh.wm[t] = sa * w[t];
    sh.wk[t] = sb * w[64 + t];
  }
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
  using CoefT = typename std::remove_cv<typename std::remove_reference<decltype(coef[0])>::type>::type;
  auto coef_of = [&](int E) -> CoefT {  // element (i, j, E); zero outside the mesh
    CoefT c;
    c.x = 0;
    c.y = 0;
    if (elem_col && E >= 0 && E < gnz && HEAT_INDEX_OK(s.sc, ebase + estride * E, ne_all))
      c = coef[ebase + estride * E];
    return c;
  };
  Raw r00 = fetch(0, false), r10 = r00, r01 = r00, r11 = r00;
  fetch_level(k0 - 1, r00, r10, r01, r11);
  CoefT cn = coef_of(k0 - 2);
  T vprev = T(0);  // own input at the level being output
  const int ltop = k0 + nzt;  // outputs at levels [k0, ltop)
  for (int L = k0 - 1; L <= ltop; ++L) {
    const int xs = p1_xslot(L);
    const T v = value(r00);
    sh.X[xs][ly][lx] = v;
    if (lastx) sh.X[xs][ly][SX] = value(r10);
    if (lasty) sh.X[xs][SY][lx] = value(r01);
    if (lastx && lasty) sh.X[xs][SY][SX] = value(r11);
    sh.C[p1_cslot(L - 1)][ly][lx] = {cn.x, cn.y};
    cn = coef_of(L);  // the next layer, in flight during this level
    if (L + 1 <= ltop) fetch_level(L + 1, r00, r10, r01, r11);
    __syncthreads();
    const int lv = L - 1;
    if (lv >= k0 && outcol && lv <= gnz && HEAT_INDEX_OK(s.sc, c00.base + lv * pxy, nn_all)) {
      T y = T(0);
#pragma unroll
      for (int dz = 0; dz < 2; ++dz)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            // box (i-1+dx, j-1+dy, lv-1+dz), in which this node is corner c
            const auto cf = sh.C[p1_cslot(lv - 1 + dz)][ly - 1 + dy][lx - 1 + dx];
            const int c = (1 - dx) | ((1 - dy) << 1) | ((1 - dz) << 2);
#pragma unroll
            for (int d = 0; d < 8; ++d) {
              if (!p1_mass_nz(c, d)) continue;
              const T x = sh.X[p1_xslot(lv - 1 + dz + ((d >> 2) & 1))][ly - 1 + dy + ((d >> 1) & 1)]
                              [lx - 1 + dx + (d & 1)];
              T wgt = cf.x * sh.wm[8 * c + d];
              if (p1_stiff_nz(c, d)) wgt += cf.y * sh.wk[8 * c + d];
              y += wgt * x;
            }
          }
      const bool dir = c00.dxy || (dz0 && lv == 0) || (dz1 && lv == gnz);
      out(c00.base + lv * pxy, dir, y, vprev);
    }
    vprev = v;
  }
  __syncthreads();  // the shared buffers are reused by the next call
}

// The operator of element type E on one block tile (tile_op's contract).
template <int E, class T, int SX, int SY>
using OpSmem = typename std::conditional<E == E_P1, TileSmemP1<T, SX, SY>, TileSmem<T, SX, SY>>::type;

template <int E, class T, int SX, int SY, class Coef, class Fetch, class Value, class Out>
__device__ __forceinline__ void tile_op_e(const Geo& g, const SimDev& s, const Coef* __restrict__ coef, int i0, int j0,
                                          int k0, int nzt, T sa, T sb, bool mask, OpSmem<E, T, SX, SY>& sh,
                                          Fetch&& fetch, Value&& value, Out&& out) {
  if constexpr (E == E_P1)
    tile_op_p1<T, SX, SY>(g, s, coef, i0, j0, k0, nzt, sa, sb, mask, sh, fetch, value, out);
  else
    tile_op<T, SX, SY>(g, s, coef, i0, j0, k0, nzt, sa, sb, mask, sh, fetch, value, out);
}

}  // namespace heat
