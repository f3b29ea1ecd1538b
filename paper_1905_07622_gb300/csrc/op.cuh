// The assembly-free operator: the assembly operator of §3.2 Eq. 1 read degree
// of freedom by degree of freedom. Each output node gathers from its <= 8
// elements and 27 neighbours; no atomics and no assembled matrix. Mhat/Khat are
// the Q1 element matrices indexed by the XOR of the two local corner numbers.
#pragma once

#include <type_traits>

#include "df.cuh"
#include "heat_dev.cuh"

namespace heat {

// ------------------------------------------------------------ the operator

template <class T> __device__ __forceinline__ const T* p1_consts(const SimDev& s);
template <> __device__ __forceinline__ const double* p1_consts<double>(const SimDev& s) { return s.p1c; }
template <> __device__ __forceinline__ const float* p1_consts<float>(const SimDev& s) { return s.p1c_f; }
// Storage type of the P1 box matrices for arithmetic type T (double-float
// operators read the FP64 copy).
template <class T> struct P1W { using type = T; };
template <> struct P1W<DF> { using type = double; };
template <class T> __device__ __forceinline__ const typename P1W<T>::type* p1_weights(const SimDev& s);
template <> __device__ __forceinline__ const double* p1_weights<double>(const SimDev& s) { return s.p1w; }
template <> __device__ __forceinline__ const float* p1_weights<float>(const SimDev& s) { return s.p1w_f; }
template <> __device__ __forceinline__ const double* p1_weights<DF>(const SimDev& s) { return s.p1w; }

// The six-tetrahedra form of gather_apply: node (i,j,k) is local corner c of
// each of its <= 8 boxes, and row c of the box matrices M', K' couples it to
// the corners d of the tetrahedra it shares (p1_mass_nz, p1_stiff_nz).
template <class T, class Load>
__device__ __forceinline__ T gather_apply_p1(const SimDev& s, T sa, T sb, int i, int j, int k, Load&& ld) {
  const auto* coef = coef_ptr<T>(s);
  const T* w = p1_weights<T>(s);
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int ex = i - (c & 1), ey = j - ((c >> 1) & 1), ez = k - ((c >> 2) & 1);
    if (ex < 0 || ey < 0 || ez < 0 || ex >= s.nx || ey >= s.ny || ez >= s.nz) continue;
    const auto cf = coef[ex + (long long)s.nx * (ey + (long long)s.ny * ez)];
    const T wa = sa * cf.x, wb = sb * cf.y;
#pragma unroll
    for (int d = 0; d < 8; ++d) {
      if (!p1_mass_nz(c, d)) continue;
      const T m = w[8 * c + d], kk = p1_stiff_nz(c, d) ? w[64 + 8 * c + d] : T(0);
      acc += (wa * m + wb * kk) * ld(ex + (d & 1), ey + ((d >> 1) & 1), ez + ((d >> 2) & 1));
    }
  }
  return acc;
}

// y at node (i,j,k) of sum_e (sa*rho_c_e*Mhat + sb*k_e*Khat) x_e, with x
// supplied by a loader ld(ii,jj,kk) for the 27 neighbours (0 outside the mesh).
// Six-tetrahedra boxes take gather_apply_p1.
template <class T, class Load>
__device__ __forceinline__ T gather_apply(const SimDev& s, T sa, T sb, int i, int j, int k, Load&& ld) {
  if (s.elem == E_P1) return gather_apply_p1<T>(s, sa, sb, i, j, k, ld);
  T v[27];
#pragma unroll
  for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int ii = i + dx, jj = j + dy, kk = k + dz;
        v[(dz + 1) * 9 + (dy + 1) * 3 + (dx + 1)] = inside_nodes(s, ii, jj, kk) ? ld(ii, jj, kk) : T(0);
      }
  const auto* coef = coef_ptr<T>(s);
  T acc = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) {  // node (i,j,k) is local corner c of element e
    const int cx = c & 1, cy = (c >> 1) & 1, cz = (c >> 2) & 1;
    const int ex = i - cx, ey = j - cy, ez = k - cz;
    if (ex < 0 || ey < 0 || ez < 0 || ex >= s.nx || ey >= s.ny || ez >= s.nz) continue;
    const auto cf = coef[ex + (long long)s.nx * (ey + (long long)s.ny * ez)];
    const T wa = sa * cf.x, wb = sb * cf.y;
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      const int b = c ^ p;
      const int ox = (b & 1) - cx, oy = ((b >> 1) & 1) - cy, oz = ((b >> 2) & 1) - cz;
      acc += (wa * mhat<T>(s, p) + wb * khat<T>(s, p)) * v[(oz + 1) * 9 + (oy + 1) * 3 + (ox + 1)];
    }
  }
  return acc;
}


// Hot per-simulation geometry, held in registers by the tile kernels.
// Node indices fit in int: heat_sim_create rejects meshes with N >= 2^31.
struct Geo {
  int nx, ny, nz;
  uint32_t dir;
  int px, pxy;  // node strides in y and z
  __device__ __forceinline__ explicit Geo(const SimDev& s)
      : nx(s.nx), ny(s.ny), nz(s.nz), dir(s.dir_faces), px(s.nx + 1), pxy((s.nx + 1) * (s.ny + 1)) {}
  __device__ __forceinline__ bool inside(int i, int j, int k) const {
    return i >= 0 && j >= 0 && k >= 0 && i <= nx && j <= ny && k <= nz;
  }
  __device__ __forceinline__ bool dirichlet(int i, int j, int k) const {
    return ((dir & 1u) && i == 0) || ((dir & 2u) && i == nx) || ((dir & 4u) && j == 0) ||
           ((dir & 8u) && j == ny) || ((dir & 16u) && k == 0) || ((dir & 32u) && k == nz);
  }
  // inside the mesh and not a Dirichlet node
  __device__ __forceinline__ bool free_node(int i, int j, int k) const { return inside(i, j, k) && !dirichlet(i, j, k); }
  __device__ __forceinline__ int idx(int i, int j, int k) const { return i + px * j + pxy * k; }
};

// ------------------------------------------------- the factorised tile operator
//
// The same operator computed once per tile with the element matrices
// diagonalised. On a box element both 1-D matrices are diagonal in the
// sum/difference basis, so with the unnormalised 8-point Walsh transform H of
// the corner values, A_e = H diag(lam_e) H / 8 with
//   lam_e[w] = sa*rho_c_e*lam_m[w] + sb*k_e*lam_k[w].
// The three butterfly stages are shared between neighbouring elements: an
// x-edge belongs to 4 elements, an xy-face to 2. Each thread of an SX x SY
// block owns node column (i, j) = (i0-1+lx, j0-1+ly) with its x-edge, its
// xy-face and its element column, and marches up the node levels of the
// tile: forward x (shuffle), forward y (shared memory), forward z and scaling
// and inverse z (registers), face sums (registers), inverse y (shared memory),
// inverse x and node sums (shuffle). Outputs are the node columns with
// lx >= 1 and ly >= 1, levels [k0, k0+nzt): (SX-1)(SY-1)nzt nodes per tile.
// About 60 floating-point operations per node instead of ~190 for the gather.

template <class T> struct Pair;
template <> struct Pair<double> { using type = double2; };
template <> struct Pair<float> { using type = float2; };
template <> struct Pair<DF> { using type = DF2; };

template <class T, int SX, int SY>
struct TileSmem {
  typename Pair<T>::type E[2][SY][SX];  // x-edges of the level being staged
  typename Pair<T>::type F[2][SY][SX];  // row j+1 halves of a finished face level
};

template <class T> __device__ __forceinline__ T lam_m(const SimDev& s, int w);
template <> __device__ __forceinline__ double lam_m<double>(const SimDev& s, int w) { return s.lam_m[w]; }
template <> __device__ __forceinline__ float lam_m<float>(const SimDev& s, int w) { return s.lam_m_f[w]; }
template <> __device__ __forceinline__ DF lam_m<DF>(const SimDev& s, int w) { return DF(s.lam_m[w]); }
template <class T> __device__ __forceinline__ T lam_k(const SimDev& s, int w);
template <> __device__ __forceinline__ double lam_k<double>(const SimDev& s, int w) { return s.lam_k[w]; }
template <> __device__ __forceinline__ float lam_k<float>(const SimDev& s, int w) { return s.lam_k_f[w]; }
template <> __device__ __forceinline__ DF lam_k<DF>(const SimDev& s, int w) { return DF(s.lam_k[w]); }

// A node column (i, j) of a tile: node index base (level 0), whether it lies
// inside the mesh, and whether an x or y Dirichlet face contains it.
struct Col {
  int base;
  bool in, dxy;
  __device__ __forceinline__ Col(const Geo& g, int i, int j) {
    in = i >= 0 && j >= 0 && i <= g.nx && j <= g.ny;
    base = in ? i + g.px * j : 0;
    dxy = in && (((g.dir & 1u) && i == 0) || ((g.dir & 2u) && i == g.nx) || ((g.dir & 4u) && j == 0) ||
                 ((g.dir & 8u) && j == g.ny));
  }
};

// The input is read in two phases so that the loads of level L+1 are in
// flight while level L is computed:
//   fetch(m, live) -> Raw: issue the loads for node index m; live == false
//     means the node is outside the mesh or masked (a Dirichlet node when
//     `mask`): return a Raw that value() maps to 0, without touching memory.
//   value(raw) -> T: the input value from the fetched data.
// Called once per staged node (plus the tile's far x column and y row).
// out(m, dir, y, v): called once per output node: index, Dirichlet row flag,
//   operator value y and the thread's own staged input v at that node.
// Must be called by every thread of the block (it synchronises).
template <class T, int SX, int SY, class Coef, class Fetch, class Value, class Out>
__device__ __forceinline__ void tile_op(const Geo& g, const SimDev& s, const Coef* __restrict__ coef, int i0, int j0,
                                        int k0, int nzt, T sa, T sb, bool mask, TileSmem<T, SX, SY>& sh,
                                        Fetch&& fetch, Value&& value, Out&& out) {
  constexpr unsigned FULL = 0xffffffffu;
  const int lx = (int)threadIdx.x % SX, ly = (int)threadIdx.x / SX;
  const int i = i0 - 1 + lx, j = j0 - 1 + ly;
  const bool outcol = lx >= 1 && ly >= 1 && i <= g.nx && j <= g.ny;
  const bool lastx = lx == SX - 1, lasty = ly == SY - 1;
  const bool elem_col = i >= 0 && j >= 0 && i < g.nx && j < g.ny;
  // the columns this thread stages: its own, and for the tile's last x column
  // and last y row the columns one further on
  const Col c00(g, i, j), c10(g, i + 1, j), c01(g, i, j + 1), c11(g, i + 1, j + 1);
  // G_q = Tp_q + A_q Fp_q + B_q F_q and Tn_q = B_q Fp_q + A_q F_q with
  // A_q = lam_q + lam_{q+4}, B_q = lam_q - lam_{q+4} (the two z-Walsh
  // indices of xy index q), linear in (rho_c, k) with these coefficients:
  T am[4], ak[4], bm[4], bk[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    am[q] = sa * (lam_m<T>(s, q) + lam_m<T>(s, q + 4));
    ak[q] = sb * (lam_k<T>(s, q) + lam_k<T>(s, q + 4));
    bm[q] = sa * (lam_m<T>(s, q) - lam_m<T>(s, q + 4));
    bk[q] = sb * (lam_k<T>(s, q) - lam_k<T>(s, q + 4));
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
      c = coef[ebase + estride * E];  // int: N < 2^31 per simulation
    return c;
  };
  Raw r00 = fetch(0, false), r10 = r00, r01 = r00, r11 = r00;
  fetch_level(k0 - 1, r00, r10, r01, r11);
  CoefT cnext = coef_of(k0 - 1);
  T Fp[4] = {T(0), T(0), T(0), T(0)};  // face at the level below
  T Tp[4] = {T(0), T(0), T(0), T(0)};  // top half of the element below
  T rj[2] = {T(0), T(0)};              // row-j half of the last finished face level
  T up[2] = {T(0), T(0)};              // row-(j+1) half, handed to the row above
  T vh0 = T(0), vh1 = T(0), vh2 = T(0);  // own staged input at levels L, L-1, L-2
  const int ltop = k0 + nzt;
  for (int L = k0 - 1; L <= ltop + 1; ++L) {
    const int buf = L & 1;
    T e0 = T(0), e1 = T(0), a0 = T(0), a1 = T(0);
    vh2 = vh1;
    vh1 = vh0;
    vh0 = T(0);
    if (L <= ltop) {
      // forward x: the x-edge (i..i+1, j, L) as (sum, difference)
      const T v = value(r00);
      T vr = __shfl_down_sync(FULL, v, 1, SX);
      if (lastx) vr = value(r10);
      e0 = v + vr;
      e1 = v - vr;
      vh0 = v;
      // the last row also needs the x-edge of row j+1
      const T w = lasty ? value(r01) : T(0);
      T wr = __shfl_down_sync(FULL, w, 1, SX);
      if (lastx && lasty) wr = value(r11);
      a0 = w + wr;
      a1 = w - wr;
      sh.E[buf][ly][lx] = {e0, e1};
      if (L + 1 <= ltop) fetch_level(L + 1, r00, r10, r01, r11);  // in flight during this level
    }
    sh.F[buf][ly][lx] = {up[0], up[1]};
    __syncthreads();
    if (L >= k0 + 2) {
      // finish node level L-2: x-edge (i..i+1, j) = row-j half of face (i, j)
      // + row-(j+1) half of face (i, j-1); inverse x; add the left edge's share
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
      // forward y: face (i..i+1, j..j+1, L), index q = wx | wy<<1
      const T Fc[4] = {e0 + a0, e1 + a1, e0 - a0, e1 - a1};
      if (L >= k0) {
        // element (i, j, L-1) between face levels L-1 (bottom) and L (top)
        const T rc = cnext.x, kc = cnext.y;
        cnext = coef_of(L);  // next level's element, in flight
        T G[4], Tn[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          // forward z, scaling and inverse z in one: bottom half into the face
          // sum, top half carried to the next level
          const T A = rc * am[q] + kc * ak[q], B = rc * bm[q] + kc * bk[q];
          G[q] = Tp[q] + A * Fp[q] + B * Fc[q];
          Tn[q] = B * Fp[q] + A * Fc[q];
        }
        // inverse y on the finished face level L-1
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
  __syncthreads();  // the shared buffers are reused by the next call
}

__device__ __forceinline__ void node_of(const SimDev& s, long long n, int& i, int& j, int& k) {
  const long long px = s.nx + 1, pxy = px * (s.ny + 1);
  k = (int)(n / pxy);
  const long long rem = n - (long long)k * pxy;
  j = (int)(rem / px);
  i = (int)(rem - (long long)j * px);
}

}  // namespace heat
