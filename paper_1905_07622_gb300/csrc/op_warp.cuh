// The factorised operator (see op.cuh) with the y direction held in
// registers: a warp-segment tile.
//
// A segment of SX lanes (SX divides 32) owns node columns x = i0-1+lx; each
// thread holds NY+2 consecutive y rows of its column and marches up the z
// levels. Forward x and the final x-sum use segment shuffles; forward y,
// forward z, scaling, inverse z, the face sums and inverse y all stay in the
// thread's registers, so the level loop has no block barrier, and the NY rows
// are independent instruction streams. Outputs are lanes 1..SX-2 (the outer
// lanes only supply neighbours), rows 1..NY, levels [k0, k0+nzt):
// (SX-2) x NY x nzt nodes per segment.
//
// Where the loads come from is a policy (the Src argument):
//  - RegSrc: plain loads one level ahead into registers;
//  - AsyncSrc: each thread copies its own rows S-1 levels ahead into a
//    private ring of S stages in shared memory with cp.async (no registers held
//    for data in flight, no barrier: a thread reads back only what it copied,
//    after waiting for its own copy groups).
#pragma once

#include <type_traits>
#include <utility>

#include "op.cuh"

namespace heat {

// Pairs of values with element-wise arithmetic: packed FP32x2 instructions for
// float (two results per issued instruction on sm_100 and later), two scalar
// operations for double. fma(a, b, c) = a*b + c with one rounding per lane.
template <class T> struct Pair2;
template <> struct Pair2<float> {
  using t = float2;
  static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
  static __device__ __forceinline__ float2 add(float2 a, float2 b) { return __fadd2_rn(a, b); }
  static __device__ __forceinline__ float2 mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
  static __device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
};
template <> struct Pair2<double> {
  using t = double2;
  static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
  static __device__ __forceinline__ double2 add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
  static __device__ __forceinline__ double2 mul(double2 a, double2 b) { return make_double2(a.x * b.x, a.y * b.y); }
  static __device__ __forceinline__ double2 fma(double2 a, double2 b, double2 c) {
    return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y));
  }
};

// Double-float pairs (df.cuh): the refinement passes' arithmetic, about 48
// significant bits from FP32 instructions.
template <> struct Pair2<DF> {
  using t = DF2;
  static __device__ __forceinline__ DF2 make(DF a, DF b) { return DF2{a, b}; }
  static __device__ __forceinline__ DF2 add(DF2 a, DF2 b) { return DF2{a.x + b.x, a.y + b.y}; }
  static __device__ __forceinline__ DF2 mul(DF2 a, DF2 b) { return DF2{a.x * b.x, a.y * b.y}; }
  static __device__ __forceinline__ DF2 fma(DF2 a, DF2 b, DF2 c) { return DF2{a.x * b.x + c.x, a.y * b.y + c.y}; }
};

// One element's precomputed Walsh-pair coefficients A_0..A_3, B_0..B_3 of the
// A operator (SimDev::acoef): FP64 pairs, or (hi, lo) float pairs for DF.
struct alignas(16) PreRec {
  float4 w[4];
};

// The march's per-element pair coefficients (A_q, B_q) for the pair halves
// h = 0 (q = 0, 1) and h = 1 (q = 2, 3): formed from the element's (rho_c,
// k) and the scaled eigenvalue sums AM, AK, BM, BK, or read from a PreRec.
template <class T, class C, class T2>
__device__ __forceinline__ void march_coeffs(const C& cf, const T2 (&AM)[2], const T2 (&AK)[2], const T2 (&BM)[2],
                                             const T2 (&BK)[2], T2 (&A)[2], T2 (&B)[2]) {
  using V = Pair2<T>;
  const T2 rc = V::make(cf.x, cf.x), kc = V::make(cf.y, cf.y);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    A[h] = V::fma(kc, AK[h], V::mul(rc, AM[h]));
    B[h] = V::fma(kc, BK[h], V::mul(rc, BM[h]));
  }
}
template <class T, class T2>
__device__ __forceinline__ void march_coeffs(const PreRec& cf, const T2 (&)[2], const T2 (&)[2], const T2 (&)[2],
                                             const T2 (&)[2], T2 (&A)[2], T2 (&B)[2]) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    if constexpr (sizeof(T) == 8 && !std::is_same<T, DF>::value) {
      A[h] = *reinterpret_cast<const T2*>(&cf.w[h]);
      B[h] = *reinterpret_cast<const T2*>(&cf.w[2 + h]);
    } else {
      A[h] = T2{T(cf.w[h].x, cf.w[h].y), T(cf.w[h].z, cf.w[h].w)};
      B[h] = T2{T(cf.w[2 + h].x, cf.w[2 + h].y), T(cf.w[2 + h].z, cf.w[2 + h].w)};
    }
  }
}

// Geometry of one lane of a segment tile: which of its rows exist, which are
// Dirichlet, where its column starts.
template <int NY>
struct LaneGeo {
  static constexpr int NR = NY + 2;  // staged rows
  static constexpr int NF = NY + 1;  // faces / element rows
  bool out_lane;
  unsigned rin, rdxy, ein, rstat;  // bit r: row inside / x-y Dirichlet / element row valid / loadable
  int nbase, ebase, estride, pxy, gnz, px, enx;
  bool dz0, dz1, mask;
  SimScalars* sc;      // where HEAT_CHECK builds count out-of-range indices
  long long nn, ne;    // node and element counts (the index bounds)

  __device__ __forceinline__ LaneGeo(const Geo& g, bool active, int lx, int SX, int i0, int j0, bool mask_,
                                     SimScalars* sc_ = nullptr) {
    sc = sc_;
    nn = (long long)g.px * (g.ny + 1) * (g.nz + 1);
    ne = (long long)g.nx * g.ny * g.nz;
    const int c = i0 - 1 + lx;
    const bool col_in = active && c >= 0 && c <= g.nx;
    out_lane = active && lx >= 1 && lx <= SX - 2 && c <= g.nx;
    const bool ecol = active && c >= 0 && c < g.nx;
    const bool dx = col_in && (((g.dir & 1u) && c == 0) || ((g.dir & 2u) && c == g.nx));
    rin = rdxy = ein = 0u;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int j = j0 - 1 + r;
      const bool in = col_in && j >= 0 && j <= g.ny;
      if (in) rin |= 1u << r;
      if (in && (dx || ((g.dir & 4u) && j == 0) || ((g.dir & 8u) && j == g.ny))) rdxy |= 1u << r;
      if (r < NF && ecol && j >= 0 && j < g.ny) ein |= 1u << r;
    }
    nbase = c + g.px * (j0 - 1);  // node index of row 0 at level 0 (rows step by px)
    ebase = c + g.nx * (j0 - 1);  // element index of element row 0 at level 0
    estride = g.nx * g.ny;
    pxy = g.pxy;
    gnz = g.nz;
    px = g.px;
    enx = g.nx;
    dz0 = (g.dir & 16u) != 0;
    dz1 = (g.dir & 32u) != 0;
    mask = mask_;
    rstat = rin & ~(mask ? rdxy : 0u);  // rows that can be live at any level
  }
  // rows of node level L that hold unknowns (bit r)
  __device__ __forceinline__ unsigned live_rows(int L) const {
    const bool lev = L >= 0 && L <= gnz && !(mask && ((dz0 && L == 0) || (dz1 && L == gnz)));
    return lev ? rstat : 0u;
  }
  // element rows of element layer E inside the mesh (bit r)
  __device__ __forceinline__ unsigned live_elems(int E) const { return (E >= 0 && E < gnz) ? ein : 0u; }
};

// Loads one level ahead into registers through caller-supplied functors:
// fetch(node, live) -> Raw, value(Raw) -> T.
template <class T, int NY, class Coef, class Fetch, class Value>
struct RegSrc {
  static constexpr int NR = NY + 2, NF = NY + 1;
  using Raw = decltype(std::declval<Fetch&>()(0, false));
  const Coef* __restrict__ coef;
  Fetch& fetch;
  Value& value;
  int k0;
  Raw raw[NR];
  Coef cf[NF];

  __device__ __forceinline__ RegSrc(const Coef* c, Fetch& f, Value& v, int k0_) : coef(c), fetch(f), value(v), k0(k0_) {}
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
      Coef z;
      z.x = 0;
      z.y = 0;
      const int e = lg.ebase + r * lg.enx + E * lg.estride;
      cf[r] = (((le >> r) & 1u) && HEAT_INDEX_OK(lg.sc, e, lg.ne)) ? coef[e] : z;
    }
  }
  // before the loop: node level k0-1, element layer k0-1 (used at t = 1)
  __device__ __forceinline__ void prologue(const LaneGeo<NY>& lg, int) {
    load_nodes(lg, k0 - 1);
    load_coef(lg, k0 - 1);
  }
  // values of node level L = k0-1+t, then the next level's loads
  __device__ __forceinline__ void level(const LaneGeo<NY>& lg, int t, int tzl, T v[NR]) {
#pragma unroll
    for (int r = 0; r < NR; ++r) v[r] = value(raw[r]);
    if (t <= tzl) load_nodes(lg, k0 + t);  // in flight during this level's arithmetic
  }
  // coefficients of element layer k0-2+t (valid for t >= 1)
  __device__ __forceinline__ Coef coef_row(int, int r) const { return cf[r]; }
  __device__ __forceinline__ void after_elements(const LaneGeo<NY>& lg, int t, int tzl) {
    if (t <= tzl) load_coef(lg, k0 - 1 + t);
  }
};

// cp.async of 4, 8 or 16 bytes into shared memory; live = false writes zeros
// and reads nothing (the source address must still be a valid pointer).
template <int BYTES>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem, bool live) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const int n = live ? BYTES : 0;
  if (BYTES == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
  else if (BYTES == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Shared-memory bytes one thread of AsyncSrc<T, NY, S> uses.
template <class T, int NY, int S>
__host__ __device__ constexpr int async_stage_bytes() {
  return S * ((NY + 2) * 3 * (int)sizeof(T) + (NY + 1) * 2 * (int)sizeof(T));
}

// The direction-fused apply's loads (P^-1, r, d_old per node; (rho_c, k) per
// element) staged through a per-thread ring of S stages; dold = nullptr is a
// restart. Stage t holds node level k0-1+t and element layer k0-2+t. Layout:
// planes of nt values (one per thread of the block), so a warp's accesses are
// conflict-free.
template <class T, int NY, int S, class Coef>
struct AsyncSrc {
  static constexpr int NR = NY + 2, NF = NY + 1;
  static_assert(S >= 2, "at least two stages");
  const T* __restrict__ pinv;
  const T* __restrict__ r;
  const T* __restrict__ dold;  // nullptr: restart, d_old = 0
  const Coef* __restrict__ coef;
  T beta;
  T* nodes;     // [S][NR][3][nt]
  Coef* elems;  // [S][NF][nt]
  int nt, tid, k0;

  __device__ __forceinline__ AsyncSrc(const T* p, const T* rr, const T* d, const Coef* c, T b, void* smem, int nthreads,
                                      int thread, int k0_)
      : pinv(p), r(rr), dold(d), coef(c), beta(b), nt(nthreads), tid(thread), k0(k0_) {
    nodes = reinterpret_cast<T*>(smem);
    elems = reinterpret_cast<Coef*>(nodes + S * NR * 3 * nt);
  }
  __device__ __forceinline__ T* node_slot(int st, int row, int comp) const {
    return nodes + ((st * NR + row) * 3 + comp) * nt + tid;
  }
  __device__ __forceinline__ Coef* elem_slot(int st, int row) const { return elems + (st * NF + row) * nt + tid; }

  // copies for stage t (node level k0-1+t, element layer k0-2+t) as one group
  __device__ __forceinline__ void issue(const LaneGeo<NY>& lg, int t) {
    const int st = t % S;
    const int L = k0 - 1 + t, E = L - 1;
    const unsigned lv = lg.live_rows(L);
    const int off = lg.nbase + L * lg.pxy;
#pragma unroll
    for (int row = 0; row < NR; ++row) {
      const bool live = ((lv >> row) & 1u) && HEAT_INDEX_OK(lg.sc, off + row * lg.px, lg.nn);
      const int m = live ? off + row * lg.px : 0;
      cp_async<sizeof(T)>(node_slot(st, row, 0), pinv + m, live);
      cp_async<sizeof(T)>(node_slot(st, row, 1), r + m, live);
      if (dold) cp_async<sizeof(T)>(node_slot(st, row, 2), dold + m, live);
    }
    const unsigned le = lg.live_elems(E);
#pragma unroll
    for (int row = 0; row < NF; ++row) {
      const bool live =
          ((le >> row) & 1u) && HEAT_INDEX_OK(lg.sc, lg.ebase + row * lg.enx + E * lg.estride, lg.ne);
      const int e = live ? lg.ebase + row * lg.enx + E * lg.estride : 0;
      cp_async<sizeof(Coef)>(elem_slot(st, row), coef + e, live);
    }
    cp_async_commit();
  }
  __device__ __forceinline__ void prologue(const LaneGeo<NY>& lg, int tzl) {
#pragma unroll
    for (int t = 0; t < S - 1; ++t) {
      if (t <= tzl + 1) issue(lg, t);
      else cp_async_commit();  // one group per stage keeps the wait count fixed
    }
  }
  __device__ __forceinline__ void level(const LaneGeo<NY>& lg, int t, int tzl, T v[NR]) {
    // stage t+S-1 reuses the slot of stage t-1, which the previous level consumed
    if (t + S - 1 <= tzl + 1) issue(lg, t + S - 1);
    else cp_async_commit();
    cp_async_wait<S - 1>();  // stage t has landed
    const int st = t % S;
#pragma unroll
    for (int row = 0; row < NR; ++row) {
      const T p = *node_slot(st, row, 0), rv = *node_slot(st, row, 1);
      const T d = dold ? *node_slot(st, row, 2) : T(0);
      v[row] = p * rv + beta * d;
    }
  }
  __device__ __forceinline__ Coef coef_row(int t, int row) const { return *elem_slot(t % S, row); }
  __device__ __forceinline__ void after_elements(const LaneGeo<NY>&, int, int) {}
};

// Every lane of the segment must call this with the same tzl (the trip count
// of the level loop): shuffles span the segment. Segments with no tile pass
// active = false (they load and store nothing). Levels beyond the mesh are
// zero; outputs are clipped to the mesh. out(node, dirichlet, y, v) receives
// the operator output y and the node's own input value v.
template <class T, int SX, int NY, class Src, class Out>
__device__ __forceinline__ void warp_tile_march(const LaneGeo<NY>& lg, const SimDev& s, Src& src, int tzl, T sa,
                                                T sb, Out&& out) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int NR = NY + 2;  // staged rows
  constexpr int NF = NY + 1;  // faces / element rows
  // With lam_q and lam'_q = lam_{q+4} (the two z-Walsh indices of an xy index
  // q), the face sum and the element's top half are
  //   G_q = Tp_q + A_q Fp_q + B_q F_q,  Tn_q = B_q Fp_q + A_q F_q,
  //   A_q = lam_q + lam'_q,  B_q = lam_q - lam'_q,
  // and A_q, B_q are linear in (rho_c, k) with these coefficients. The four
  // xy indices are processed as two pairs, h = 0: q = (0, 1), h = 1: q = (2, 3).
  using V = Pair2<T>;
  using T2 = typename V::t;
  T2 AM[2], AK[2], BM[2], BK[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q0 = 2 * h, q1 = 2 * h + 1;
    AM[h] = V::make(sa * (lam_m<T>(s, q0) + lam_m<T>(s, q0 + 4)), sa * (lam_m<T>(s, q1) + lam_m<T>(s, q1 + 4)));
    AK[h] = V::make(sb * (lam_k<T>(s, q0) + lam_k<T>(s, q0 + 4)), sb * (lam_k<T>(s, q1) + lam_k<T>(s, q1 + 4)));
    BM[h] = V::make(sa * (lam_m<T>(s, q0) - lam_m<T>(s, q0 + 4)), sa * (lam_m<T>(s, q1) - lam_m<T>(s, q1 + 4)));
    BK[h] = V::make(sb * (lam_k<T>(s, q0) - lam_k<T>(s, q0 + 4)), sb * (lam_k<T>(s, q1) - lam_k<T>(s, q1 + 4)));
  }
  const T2 M1 = V::make(T(-1), T(-1));  // a - b = fma(b, M1, a), exact as a subtraction
  src.prologue(lg, tzl);
  T2 Fp[NF][2], Tp[NF][2];
  T vprev[NY];
#pragma unroll
  for (int r = 0; r < NF; ++r)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      Fp[r][h] = V::make(T(0), T(0));
      Tp[r][h] = V::make(T(0), T(0));
    }
#pragma unroll
  for (int r = 0; r < NY; ++r) vprev[r] = T(0);

  const int k0 = src.k0;
  for (int t = 0; t <= tzl + 1; ++t) {
    const int L = k0 - 1 + t;
    T v[NR];
    src.level(lg, t, tzl, v);
    // forward x (edges of each row, as the pair (sum, difference)) and
    // forward y (faces between rows): F[r][0] = (F_0, F_1), F[r][1] = (F_2, F_3)
    T2 E[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const T vr = __shfl_down_sync(FULL, v[r], 1, SX);
      E[r] = V::make(v[r] + vr, v[r] - vr);
    }
    T2 F[NF][2];
#pragma unroll
    for (int r = 0; r < NF; ++r) {
      F[r][0] = V::add(E[r], E[r + 1]);
      F[r][1] = V::fma(E[r + 1], M1, E[r]);
    }
    if (t >= 1) {
      // elements (c, j0-1+r, L-1) between face levels L-1 and L
      T2 G[NF][2];
#pragma unroll
      for (int r = 0; r < NF; ++r) {
        T2 A[2], B[2];
        march_coeffs<T>(src.coef_row(t, r), AM, AK, BM, BK, A, B);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          G[r][h] = V::fma(B[h], F[r][h], V::fma(A[h], Fp[r][h], Tp[r][h]));
          Tp[r][h] = V::fma(A[h], F[r][h], V::mul(B[h], Fp[r][h]));
        }
      }
      src.after_elements(lg, t, tzl);
      if (t >= 2) {
        // node level L-1 is complete: inverse y, inverse x, x-sum
        const int lv = L - 1;
        const bool lvin = lv <= lg.gnz;
        const bool dzl = (lg.dz0 && lv == 0) || (lg.dz1 && lv == lg.gnz);
#pragma unroll
        for (int r = 1; r <= NY; ++r) {
          // (g0, g1) = (G_0 + G_2, G_1 + G_3) of row r + (G_0 - G_2, G_1 - G_3) of row r-1
          const T2 g = V::add(V::add(G[r][0], G[r][1]), V::fma(G[r - 1][1], M1, G[r - 1][0]));
          const T nl = g.x + g.y, nr = g.x - g.y;
          const T from_left = __shfl_up_sync(FULL, nr, 1, SX);
          const int m = lg.nbase + r * lg.px + lv * lg.pxy;
          if (lg.out_lane && lvin && ((lg.rin >> r) & 1u) && HEAT_INDEX_OK(lg.sc, m, lg.nn)) {
            const bool dir = ((lg.rdxy >> r) & 1u) || dzl;
            out(m, dir, nl + from_left, vprev[r - 1]);
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NY; ++r) vprev[r] = v[r + 1];
#pragma unroll
    for (int r = 0; r < NF; ++r)
#pragma unroll
      for (int h = 0; h < 2; ++h) Fp[r][h] = F[r][h];
  }
}

// The same contract on six-tetrahedra boxes (heat.h HEAT_ELEM_P1). Each lane
// computes its box column's boxes row by row from the staged levels L-1 and
// L of its own column and of its right neighbour (one shuffle per row), with
// the split's structure instead of an 8x8 matrix:
//  - mass: each tetrahedron t adds V/20 (x_c + s_t) at its corners, s_t the
//    sum of its four values; a box corner c lies in n_c tetrahedra (6 for
//    corners 0 and 7, 2 for the others);
//  - stiffness: sum over the 12 box edges of w_e V/h_a^2 (x_i - x_j)^2, w_e
//    the number of tetrahedra that step along the edge: 2, 1, 1, 2 for the
//    edges of axis a leaving corners 0, the two one-axis corners and the
//    two-axis corner (the path gradients are axis-aligned).
// About 90 operations per box with every weight in registers. A node sums its
// <= 8 boxes' contributions in a fixed order: the upper corners of the layer
// below (carried in registers), then this layer's lower corners, the left
// neighbour's through one shuffle per row.
template <class T, int SX, int NY, class Src, class Out>
__device__ __forceinline__ void warp_tile_march_p1(const LaneGeo<NY>& lg, const SimDev& s, Src& src, int tzl, T sa,
                                                   T sb, Out&& out) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int NR = NY + 2;  // staged rows
  constexpr int NF = NY + 1;  // box rows
  const T mw = sa * p1_consts<T>(s)[0];  // V / 20 and V / h_a^2, V = hx hy hz / 6
  const T kwx = sb * p1_consts<T>(s)[1], kwy = sb * p1_consts<T>(s)[2], kwz = sb * p1_consts<T>(s)[3];
  src.prologue(lg, tzl);
  T prv[NR], prvR[NR], carry[NY];
#pragma unroll
  for (int r = 0; r < NR; ++r) prv[r] = prvR[r] = T(0);
#pragma unroll
  for (int r = 0; r < NY; ++r) carry[r] = T(0);
  const int k0 = src.k0;
  for (int t = 0; t <= tzl + 1; ++t) {
    const int L = k0 - 1 + t;
    T cur[NR], curR[NR];
    src.level(lg, t, tzl, cur);
#pragma unroll
    for (int r = 0; r < NR; ++r) curR[r] = __shfl_down_sync(FULL, cur[r], 1, SX);
    if (t >= 1) {
      // boxes (lane column, row r, layer L-1): lower corners to level L-1,
      // upper corners to level L; cx = 1 corners belong to the right lane
      T lo0[NF], lo2[NF], lo1[NF], lo3[NF], up4[NF], up6[NF], up5[NF], up7[NF];
#pragma unroll
      for (int r = 0; r < NF; ++r) {
        const auto cf = src.coef_row(t, r);
        const T x0 = prv[r], x1 = prvR[r], x2 = prv[r + 1], x3 = prvR[r + 1];
        const T x4 = cur[r], x5 = curR[r], x6 = cur[r + 1], x7 = curR[r + 1];
        const T s07 = x0 + x7;
        const T t1 = s07 + x1 + x3, t2 = s07 + x1 + x5, t3 = s07 + x2 + x3;
        const T t4 = s07 + x2 + x6, t5 = s07 + x4 + x5, t6 = s07 + x4 + x6;
        const T S6 = ((t1 + t2) + (t3 + t4)) + (t5 + t6);
        const T m = mw * cf.x;
        const T ax = kwx * cf.y, ay = kwy * cf.y, az = kwz * cf.y;
        const T e01 = T(2) * ax * (x0 - x1), e23 = ax * (x2 - x3), e45 = ax * (x4 - x5), e67 = T(2) * ax * (x6 - x7);
        const T e02 = T(2) * ay * (x0 - x2), e13 = ay * (x1 - x3), e46 = ay * (x4 - x6), e57 = T(2) * ay * (x5 - x7);
        const T e04 = T(2) * az * (x0 - x4), e15 = az * (x1 - x5), e26 = az * (x2 - x6), e37 = T(2) * az * (x3 - x7);
        lo0[r] = m * (T(6) * x0 + S6) + e01 + e02 + e04;
        lo1[r] = m * (T(2) * x1 + t1 + t2) - e01 + e13 + e15;
        lo2[r] = m * (T(2) * x2 + t3 + t4) + e23 - e02 + e26;
        lo3[r] = m * (T(2) * x3 + t1 + t3) - e23 - e13 + e37;
        up4[r] = m * (T(2) * x4 + t5 + t6) + e45 + e46 - e04;
        up5[r] = m * (T(2) * x5 + t2 + t5) - e45 + e57 - e15;
        up6[r] = m * (T(2) * x6 + t4 + t6) + e67 - e46 - e26;
        up7[r] = m * (T(6) * x7 + S6) - e67 - e57 - e37;
      }
      src.after_elements(lg, t, tzl);
      const int lv = L - 1;
      const bool lvin = lv <= lg.gnz;
      const bool dzl = (lg.dz0 && lv == 0) || (lg.dz1 && lv == lg.gnz);
#pragma unroll
      for (int r = 1; r <= NY; ++r) {
        // node row r: boxes r (cy = 0) and r - 1 (cy = 1)
        const T from_left_lo = __shfl_up_sync(FULL, lo1[r] + lo3[r - 1], 1, SX);
        const T from_left_up = __shfl_up_sync(FULL, up5[r] + up7[r - 1], 1, SX);
        const T y = ((carry[r - 1] + lo0[r]) + lo2[r - 1]) + from_left_lo;
        carry[r - 1] = (up4[r] + up6[r - 1]) + from_left_up;
        const int m = lg.nbase + r * lg.px + lv * lg.pxy;
        if (t >= 2 && lg.out_lane && lvin && ((lg.rin >> r) & 1u) && HEAT_INDEX_OK(lg.sc, m, lg.nn)) {
          const bool dir = ((lg.rdxy >> r) & 1u) || dzl;
          out(m, dir, y, prv[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      prv[r] = cur[r];
      prvR[r] = curR[r];
    }
  }
}

// The march of element type E.
template <int E, class T, int SX, int NY, class Src, class Out>
__device__ __forceinline__ void warp_march_e(const LaneGeo<NY>& lg, const SimDev& s, Src& src, int tzl, T sa, T sb,
                                             Out&& out) {
  if constexpr (E == E_P1)
    warp_tile_march_p1<T, SX, NY>(lg, s, src, tzl, sa, sb, out);
  else
    warp_tile_march<T, SX, NY>(lg, s, src, tzl, sa, sb, out);
}

// The register-prefetch form with functor loads (see RegSrc), for element E.
template <int E, class T, int SX, int NY, class Coef, class Fetch, class Value, class Out>
__device__ __forceinline__ void warp_tile_op_e(const Geo& g, const SimDev& s, const Coef* __restrict__ coef,
                                               bool active, int i0, int j0, int k0, int tzl, T sa, T sb, bool mask,
                                               Fetch&& fetch, Value&& value, Out&& out) {
  const LaneGeo<NY> lg(g, active, (int)threadIdx.x % SX, SX, i0, j0, mask, s.sc);
  using CoefT = typename std::remove_cv<typename std::remove_reference<decltype(coef[0])>::type>::type;
  RegSrc<T, NY, CoefT, typename std::remove_reference<Fetch>::type, typename std::remove_reference<Value>::type> src(
      coef, fetch, value, k0);
  warp_march_e<E, T, SX, NY>(lg, s, src, tzl, sa, sb, out);
}

}  // namespace heat
