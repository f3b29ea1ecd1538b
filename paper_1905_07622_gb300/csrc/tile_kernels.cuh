// Phase-gated kernels of the solver (Algorithm 1, §3.3), driven by the tick
// engine over work lists of (simulation, work item) pairs (k_open and
// k_open_w live in open_kernels.cuh):
//   k_open      [operator tiles] step start: b = L u^{n-1} + F^n - lift,
//               x0 = 2u^{n-1} - u^{n-2}, r = b - A x0 (PH_OPEN); the FP64 true
//               residual r = b - A x every resid_period iterations (PH_RESID);
//               on the FP32 paths the refinement sweep x64 += e32,
//               r = b - A x64 in FP64, inner restart (PH_OUTER).
//   k_apply_dot [operator tiles] d = P^-1 r + beta d_old computed while staging
//               (so the direction update has no kernel of its own), q = A' d,
//               alpha = delta / d.q.
//   k_update    [pointwise chunks] x += alpha d, r -= alpha q, delta = r.P^-1 r,
//               beta, convergence, phase changes, step close.
//   k_cheb      [operator tiles] with a Chebyshev preconditioner, the m - 1
//               operator passes of z = p_m(D^-1 A) D^-1 r before each apply
//               (PH_CHEB); the apply then stages d = z + beta d_old.
// Every reduction is a per-item partial summed in item order by the last
// block of the simulation, so a simulation's result does not depend on what
// else shares the launch.
//
// Each block keeps the descriptor and control scalars of the simulation it is
// working on in shared memory, loaded once per simulation (a launch changes a
// simulation's scalars only after all of its items are done), instead of every
// warp re-reading them from L2.
#pragma once

#include "op.cuh"
#include "op_p1.cuh"
#include "op_warp.cuh"

namespace heat {

constexpr int kPwThreads = 256;
// Nodes per pointwise work item: QPT groups of 4 nodes per thread (float4 /
// two double2 each), all loaded before any is used. Fewer groups per thread
// mean more, smaller items and more resident blocks (the tuning table picks
// QPT per precision).
__host__ __device__ constexpr int pw_chunk(int qpt) { return kPwThreads * 4 * qpt; }
// Blocks per SM the register bound of k_update aims at, by QPT and value size.
__host__ __device__ constexpr int pw_min_blocks(int qpt, int bytes) {
  return bytes == 4 ? (qpt == 1 ? 4 : (qpt == 2 ? 3 : 2)) : (qpt == 1 ? 3 : (qpt == 2 ? 2 : 1));
}

// Control scalars of a simulation (written only by earlier kernels, or by
// the last block after all of the simulation's items of this kernel).
struct Ctl {
  int phase, iu1, iu2, ix, ixa, id, restart, have_prev, iter, step, cgs, y_valid, cheb_k;
  double alpha, beta;
};

__device__ __forceinline__ Ctl load_ctl(const SimScalars* sc) {
  Ctl c;
  c.phase = __ldcg(&sc->phase);
  c.iu1 = __ldcg(&sc->iu1);
  c.iu2 = __ldcg(&sc->iu2);
  c.ix = __ldcg(&sc->ix);
  c.ixa = __ldcg(&sc->ixa);
  c.id = __ldcg(&sc->id);
  c.restart = __ldcg(&sc->restart);
  c.have_prev = __ldcg(&sc->have_prev);
  c.iter = __ldcg(&sc->iter);
  c.step = __ldcg(&sc->step);
  c.cgs = __ldcg(&sc->cgs);
  c.y_valid = __ldcg(&sc->y_valid);
  c.cheb_k = __ldcg(&sc->cheb_k);
  c.alpha = __ldcg(&sc->alpha);
  c.beta = __ldcg(&sc->beta);
  return c;
}

// Shared-memory copy of the current simulation's descriptor and scalars.
struct ItemCache {
  SimDev s;
  Ctl c;
};

// Makes `cache` hold simulation `sim` (cur is the caller's register copy of
// the cached id; every thread tracks the same sequence, so the branch is
// uniform). Contains barriers when it reloads.
//
// The kernels are launched with programmatic dependent launch: a kernel may
// start while the previous one is finishing. The descriptor is static (set at
// upload), so it is copied before waiting; the scalars and vectors are the
// previous kernel's results, so everything after cudaGridDependencySynchronize
// (which returns at once when there is no programmatic predecessor).
__device__ __forceinline__ void cache_sim(const SimDev* __restrict__ sims, int sim, ItemCache& cache, int& cur,
                                          bool& dep_ready) {
  if (sim == cur) return;
  __syncthreads();  // the previous simulation's users are done
  if (threadIdx.x < 32) {
    const uint4* src = reinterpret_cast<const uint4*>(&sims[sim]);
    uint4* dst = reinterpret_cast<uint4*>(&cache.s);
    for (int t = threadIdx.x; t < (int)(sizeof(SimDev) / sizeof(uint4)); t += 32) dst[t] = src[t];
    __syncwarp();
  }
  if (!dep_ready) {
    cudaGridDependencySynchronize();
    dep_ready = true;
  }
  if (threadIdx.x == 0) cache.c = load_ctl(cache.s.sc);
  __syncthreads();
  cur = sim;
}

// Lets the next kernel of the stream be launched (it still waits for this
// one's completion before reading its results).
__device__ __forceinline__ void allow_next_launch() { cudaTriggerProgrammaticLaunchCompletion(); }

// Block sum of per-thread partials of type T: each warp sums in T, the warp
// sums are converted to FP64 and added by thread 0 in warp order. (On this
// GPU FP64 runs at 1/58 of the FP32 rate, so FP64 work per thread would cost
// more than the streaming it accompanies.) red: NV*32 doubles. Result in thread 0.
//
// VT > 1: each thread stands for VT threads of a block VT times larger
// (virtual thread tid + u * blockDim.x holds v[u]); the sum is then bitwise
// the one that larger block would form: virtual warp k = warp + u * nwarps.
template <class T, int NV, int VT = 1>
__device__ __forceinline__ void block_sum_t(const T (&v)[VT * NV], double (&out)[NV], double* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  T w[VT * NV];
#pragma unroll
  for (int a = 0; a < VT * NV; ++a) {
    w[a] = v[a];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) w[a] += __shfl_down_sync(0xffffffffu, w[a], o);
  }
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int u = 0; u < VT; ++u)
#pragma unroll
      for (int a = 0; a < NV; ++a) red[a * 32 + warp + u * nwarps] = (double)w[u * NV + a];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double t = 0.0;
      for (int k = 0; k < VT * nwarps; ++k) t += red[a * 32 + k];
      out[a] = t;
    }
  }
}

// Publishes a work item's partials (per-thread values of type T). Warp 0
// alone then takes the completion count; only the warp that finishes the
// simulation's last item of this kernel sums all items' partials (in item
// order) and returns true, with the totals in lane 0's out. The other warps
// do not wait for the count.
template <class T, int NV, int VT = 1>
__device__ __forceinline__ bool finish_item(const SimDev& s, int item, int nitems, const T (&v)[VT * NV],
                                            double (&out)[NV], double* red) {
  block_sum_t<T, NV, VT>(v, out, red);
  if (threadIdx.x >= 32) return false;
  int last = 0;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) s.partial[4 * item + a] = out[a];
    __threadfence();
    last = atomicAdd(&s.sc->count, 1u) == (unsigned int)(nitems - 1);
  }
  last = __shfl_sync(0xffffffffu, last, 0);
  if (!last) return false;
  __threadfence();
  double t[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) t[a] = 0.0;
  // Lane l adds items l, l+32, l+64, ... in that order; the loads of a batch
  // of 8 are all issued before the first add, so the tail is a few L2 round
  // trips instead of one per 32 items.
  constexpr int B = 8;
  for (int u0 = threadIdx.x; u0 < nitems; u0 += 32 * B) {
    double v[B][NV];
#pragma unroll
    for (int k = 0; k < B; ++k) {
      const int u = u0 + 32 * k;
#pragma unroll
      for (int a = 0; a < NV; ++a) v[k][a] = u < nitems ? __ldcg(&s.partial[4 * u + a]) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < B; ++k)
#pragma unroll
      for (int a = 0; a < NV; ++a) t[a] += v[k][a];
  }
#pragma unroll
  for (int a = 0; a < NV; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t[a] += __shfl_down_sync(0xffffffffu, t[a], o);
    out[a] = t[a];  // valid in lane 0
  }
  return threadIdx.x == 0;
}

// Step close, run by one thread: log, rotate the state ring
// (U^{n-2} <- U^{n-1} <- x; the old U^{n-2} slot becomes the next x).
// y_fresh: yv[ix] holds A' x (the closing FP64 residual pass computed it), so
// the next step's x0 product needs no operator pass; the stored product of
// U^{n-1} carries over to U^{n-2}.
__device__ __forceinline__ void close_step(const SimDev& s, SimScalars* sc, double delta_final, bool y_fresh = false) {
  sc->y_valid = (sc->y_valid & (1 << sc->iu1)) | (y_fresh ? (1 << sc->ix) : 0);
  const int st = sc->step;
  if (s.iters_log_len > 0) s.iters_log[st % s.iters_log_len] = sc->iter_step;
  sc->iters_total += sc->iter_step;
  sc->outer_total += sc->outer;
  sc->steps_total += 1;
  if (sc->iter_step > sc->max_iters_step) sc->max_iters_step = sc->iter_step;
  sc->rel_res = sc->delta_b > 0.0 ? sqrt(fmax(delta_final, 0.0) / sc->delta_b) : 0.0;
  const int t = sc->iu2;
  sc->iu2 = sc->iu1;
  sc->iu1 = sc->ix;
  sc->ix = t;
  sc->have_prev = 1;
  sc->step = st + 1;
  sc->status = ST_OK;
  sc->phase = (st + 1 >= sc->target) ? PH_DONE : PH_OPEN;
}

__device__ __forceinline__ void fail(SimScalars* sc, int status) {
  sc->status = status;
  sc->phase = PH_FAILED;
}

// The next CG iteration starts: with a Chebyshev preconditioner its passes
// come first (they set delta = r^T z and beta), otherwise the apply.
__device__ __forceinline__ void enter_iter(const SimDev& s, SimScalars* sc) {
  if (s.cheb_m >= 2) {
    sc->cheb_k = 1;
    sc->phase = PH_CHEB;
  } else {
    sc->phase = PH_ITER;
  }
}

struct TileCoords {
  int i0, j0, k0, nzt;
};

template <int SX, int SY>
__device__ __forceinline__ TileCoords tile_coords(const SimDev& s, int t) {
  const int tx = t % s.ntx;
  const int r = t / s.ntx;
  const int ty = r % s.nty;
  const int tz = r / s.nty;
  TileCoords c;
  c.i0 = tx * (SX - 1);
  c.j0 = ty * (SY - 1);
  c.k0 = tz * s.tz_len;
  c.nzt = min(s.tz_len, s.nz + 1 - c.k0);
  return c;
}

// ------------------------------------------------------------- k_apply_dot

template <class T> struct IterVecs;
template <> struct IterVecs<double> {
  __device__ static const double* r(const SimDev& s) { return s.r; }
  __device__ static const double* pinv(const SimDev& s) { return s.pinv; }
  __device__ static double* d(const SimDev& s, int id) { return s.d[id]; }
  __device__ static double* q(const SimDev& s) { return s.q; }
  __device__ static const double2* coef(const SimDev& s) { return s.coef; }
};
template <> struct IterVecs<float> {
  __device__ static const float* r(const SimDev& s) { return s.r32; }
  __device__ static const float* pinv(const SimDev& s) { return s.pinv32; }
  __device__ static float* d(const SimDev& s, int id) { return s.d32[id]; }
  __device__ static float* q(const SimDev& s) { return s.q32; }
  __device__ static const float2* coef(const SimDev& s) { return s.coef32; }
};

template <class T> struct ChebVecs;
template <> struct ChebVecs<double> {
  __device__ static double* z(const SimDev& s) { return s.yv[0]; }
  __device__ static double* res(const SimDev& s) { return s.yv[1]; }
  __device__ static double* dd(const SimDev& s, int k) { return s.yv[2 + k]; }
};
template <> struct ChebVecs<float> {
  __device__ static float* z(const SimDev& s) { return s.z32; }
  __device__ static float* res(const SimDev& s) { return s.rc32[1]; }
  __device__ static float* dd(const SimDev& s, int k) { return k ? s.p32 : s.wc32[1]; }
};

template <class T>
struct DirRaw {
  T p, r, d;
};

template <class T, int SX, int SY, int E = E_Q1>
__global__ void __launch_bounds__(SX* SY) k_apply_dot(const SimDev* __restrict__ sims, const int2* __restrict__ work,
                                                      const int* __restrict__ nwork_p) {
  __shared__ OpSmem<E, T, SX, SY> sh;
  __shared__ double red[32];
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
    if (c.phase != PH_ITER) continue;
    const Geo g(s);
    const TileCoords tc = tile_coords<SX, SY>(s, wi.y);
    // d = P^-1 r + beta d_old; after Chebyshev passes r is their P z, so d = z + beta d_old
    const T* __restrict__ r = s.cheb_m >= 2 ? ChebVecs<T>::z(s) : IterVecs<T>::r(s);
    const T* __restrict__ pinv = IterVecs<T>::pinv(s);
    const T* __restrict__ dold = IterVecs<T>::d(s, c.id);
    T* __restrict__ dnew = IterVecs<T>::d(s, c.id ^ 1);
    T* __restrict__ q = IterVecs<T>::q(s);
    const bool rs = c.restart != 0;
    const T beta = rs ? T(0) : (T)c.beta;
    // Per-thread partial in T (FP32 on the FP32 path), FP64 from the warp sums on.
    T acc = T(0);
    tile_op_e<E, T, SX, SY>(
        g, s, IterVecs<T>::coef(s), tc.i0, tc.j0, tc.k0, tc.nzt, (T)s.inv_dt, (T)s.theta, true, sh,
        [&](int m, bool live) -> DirRaw<T> {
          if (!live) return {T(0), T(0), T(0)};
          return {pinv[m], r[m], rs ? T(0) : dold[m]};
        },
        [&](const DirRaw<T>& v) -> T { return v.p * v.r + beta * v.d; },
        [&](int m, bool dir, T y, T v) {
          const T qv = dir ? T(0) : y;
          q[m] = qv;
          dnew[m] = v;
          acc += v * qv;
        });
    const T accv[1] = {acc};
    double tot[1];
    if (finish_item<T, 1>(s, wi.y, s.ntiles, accv, tot, red)) {
      SimScalars* sc = s.sc;
      sc->count = 0;
      const double dq = tot[0];
      sc->dq = dq;
      if (!isfinite(dq)) fail(sc, ST_NONFINITE);
      else if (!(dq > 0.0)) fail(sc, ST_BREAKDOWN);
      else {
        sc->alpha = sc->delta / dq;
        sc->id ^= 1;
        sc->restart = 0;
      }
    }
  }
}

// Loads of vectors that an earlier phase of the same launch wrote (the
// persistent iteration kernel, loop_kernels.cuh) go through L2 only (ld.cg):
// the SM's L1 is not coherent with other SMs' stores. Between kernels L1
// starts empty, so the separate kernels use plain loads.
template <bool CG, class T>
__device__ __forceinline__ T ld_vec(const T* p) {
  if constexpr (CG) return __ldcg(p);
  else return *p;
}

// One work item of the warp-segment apply (k_apply_dot_w): SPC consecutive
// segment tiles of one simulation in phase PH_ITER, its partial of d.q and,
// in the block that finishes the simulation's last item, alpha. CG: r and
// d_old are loaded through L2 only (see ld_vec).
template <class T, int SX, int NY, int WARPS, int STAGES, int E, bool CG>
__device__ __forceinline__ void apply_w_item(const SimDev& s, const Ctl& c, int item, double* red,
                                             unsigned char* stage_smem) {
  static_assert(!CG || STAGES == 0, "the L2-only loads exist for the register-prefetch form");
  constexpr int SPC = WARPS * (32 / SX);  // segments per block
  const Geo g(s);
  const int tile = item * SPC + (int)threadIdx.x / SX;
  const bool active = tile < s.w_ntiles;
  const int tx = tile % s.w_ntx, rem = tile / s.w_ntx, ty = rem % s.w_nty, tz = rem / s.w_nty;
  const T* __restrict__ r = s.cheb_m >= 2 ? ChebVecs<T>::z(s) : IterVecs<T>::r(s);  // see k_apply_dot
  const T* __restrict__ pinv = IterVecs<T>::pinv(s);
  const T* __restrict__ dold = IterVecs<T>::d(s, c.id);
  T* __restrict__ dnew = IterVecs<T>::d(s, c.id ^ 1);
  T* __restrict__ q = IterVecs<T>::q(s);
  const bool rs = c.restart != 0;
  const T beta = rs ? T(0) : (T)c.beta;
  T acc = T(0);
  auto out = [&](int m, bool dir, T y, T v) {
    const T qv = dir ? T(0) : y;
    q[m] = qv;
    dnew[m] = v;
    acc += v * qv;
  };
  if constexpr (STAGES == 0) {
    warp_tile_op_e<E, T, SX, NY>(
        g, s, IterVecs<T>::coef(s), active, tx * (SX - 2), ty * NY, tz * s.w_tz, s.w_tz, (T)s.inv_dt,
        (T)s.theta, true,
        [&](int m, bool live) -> DirRaw<T> {
          if (!live) return {T(0), T(0), T(0)};
          return {pinv[m], ld_vec<CG>(r + m), rs ? T(0) : ld_vec<CG>(dold + m)};
        },
        [&](const DirRaw<T>& v) -> T { return v.p * v.r + beta * v.d; }, out);
  } else {
    using CoefT = typename std::remove_cv<typename std::remove_reference<decltype(IterVecs<T>::coef(s)[0])>::type>::type;
    const LaneGeo<NY> lg(g, active, (int)threadIdx.x % SX, SX, tx * (SX - 2), ty * NY, true, s.sc);
    AsyncSrc<T, NY, STAGES, CoefT> src(pinv, r, rs ? nullptr : dold, IterVecs<T>::coef(s), beta, stage_smem,
                                       (int)blockDim.x, (int)threadIdx.x, tz * s.w_tz);
    warp_march_e<E, T, SX, NY>(lg, s, src, s.w_tz, (T)s.inv_dt, (T)s.theta, out);
  }
  const T accv[1] = {acc};
  double tot[1];
  if (finish_item<T, 1>(s, item, s.w_items, accv, tot, red)) {
    SimScalars* sc = s.sc;
    sc->count = 0;
    const double dq = tot[0];
    sc->dq = dq;
    if (!isfinite(dq)) fail(sc, ST_NONFINITE);
    else if (!(dq > 0.0)) fail(sc, ST_BREAKDOWN);
    else {
      sc->alpha = sc->delta / dq;
      sc->id ^= 1;
      sc->restart = 0;
    }
  }
}

// Warp-segment version of k_apply_dot (op_warp.cuh): a work item is a group
// of SPC consecutive segment tiles of one simulation; the level loop has no
// block barrier. Same results contract as k_apply_dot. STAGES = 0 loads one
// level ahead into registers; STAGES >= 2 stages each thread's loads through
// its own cp.async ring of that many levels in dynamic shared memory
// (async_stage_bytes per thread). MINB blocks per SM bound the registers.
template <class T, int SX, int NY, int WARPS, int STAGES, int MINB, int E = E_Q1>
__global__ void __launch_bounds__(32 * WARPS, MINB) k_apply_dot_w(const SimDev* __restrict__ sims,
                                                            const int2* __restrict__ work,
                                                            const int* __restrict__ nwork_p) {
  __shared__ double red[32];
  __shared__ ItemCache cache;
  extern __shared__ __align__(16) unsigned char stage_smem[];
  int cur = -1;
  bool dep = false;
  allow_next_launch();
  const int nwork = *nwork_p;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 wi = work[w];
    cache_sim(sims, wi.x, cache, cur, dep);
    if (cache.c.phase != PH_ITER) continue;
    apply_w_item<T, SX, NY, WARPS, STAGES, E, false>(cache.s, cache.c, wi.y, red, stage_smem);
  }
}

// ------------------------------------------------------------------ k_cheb

// One pass k (1 <= k <= m-1) of the Chebyshev preconditioner
// z = p_m(D^-1 A) D^-1 r for the interval [lam_lo, lam_hi] of D^-1 A, the
// three-term recurrence of the Chebyshev semi-iteration for A z = r started
// from z = 0 (theta, delta the interval's centre and half-width,
// sigma = theta / delta, rho_0 = 1 / sigma, rho_k = 1 / (2 sigma - rho_{k-1})):
//   dd_0 = D^-1 r / theta,  z_1 = dd_0,  res_0 = r,
//   res_k = res_{k-1} - A dd_{k-1},
//   dd_k = rho_k rho_{k-1} dd_{k-1} + (2 rho_k / delta) D^-1 res_k,
//   z_{k+1} = z_k + dd_k.
// Pass k stages dd_{k-1} (formed from r on pass 1) through the operator and
// updates its own nodes; dd_k lives in slot k & 1. The last pass sums
// r^T z_m, which becomes delta (and beta = delta / delta_old) of the CG
// iteration, and stores P z_m (z_m divided by P^-1), so that the apply forms
// d = P^-1 (P z) + beta d_old = z + beta d_old with its Jacobi staging
// unchanged (to rounding). Dirichlet rows and columns are masked as in the apply.
template <class T>
struct ChRaw {
  T a, b;
};

template <class T>
struct ChebPass {
  const T* __restrict__ r;
  const T* __restrict__ pinv;
  const T* __restrict__ ddin;
  T* __restrict__ ddout;
  T* __restrict__ res;
  T* __restrict__ z;
  T inv_th, c1, c2;
  bool first, last;
  T acc;

  __device__ __forceinline__ ChebPass(const SimDev& s, int k) {
    first = k == 1;
    last = k == s.cheb_m - 1;
    r = IterVecs<T>::r(s);
    pinv = IterVecs<T>::pinv(s);
    ddin = ChebVecs<T>::dd(s, (k - 1) & 1);
    ddout = ChebVecs<T>::dd(s, k & 1);
    res = ChebVecs<T>::res(s);
    z = ChebVecs<T>::z(s);
    inv_th = (T)__ldg(&s.cheb[0]);
    c1 = (T)__ldg(&s.cheb[2 * k - 1]);
    c2 = (T)__ldg(&s.cheb[2 * k]);
    acc = T(0);
  }
  __device__ __forceinline__ ChRaw<T> fetch(int m, bool live) const {
    if (!live) return {T(0), T(0)};
    if (first) return {pinv[m], r[m]};
    return {ddin[m], T(0)};
  }
  __device__ __forceinline__ T value(const ChRaw<T>& v) const { return first ? v.a * v.b * inv_th : v.a; }
  // v = dd_{k-1} at node m, y = (A dd_{k-1})_m
  __device__ __forceinline__ void out(int m, bool dir, T y, T v) {
    if (dir) {
      z[m] = T(0);
      return;
    }
    const T rr = (first || last) ? r[m] : T(0);
    const T p = pinv[m];
    const T rk = (first ? rr : res[m]) - y;
    const T dk = c1 * v + c2 * (p * rk);
    const T zn = (first ? v : z[m]) + dk;
    if (last) {
      acc += rr * zn;
      z[m] = zn / p;
    } else {
      z[m] = zn;
      res[m] = rk;
      ddout[m] = dk;
    }
  }
};

// The last block of a pass: advance to the next pass, or (last pass) set
// delta = r^T z, beta, and hand the iteration to the apply.
__device__ __forceinline__ void cheb_close(const SimDev& s, const Ctl& c, double gam) {
  SimScalars* sc = s.sc;
  sc->count = 0;
  if (c.cheb_k < s.cheb_m - 1) {
    sc->cheb_k = c.cheb_k + 1;
  } else if (!isfinite(gam)) {
    fail(sc, ST_NONFINITE);
  } else if (!(gam > 0.0)) {
    fail(sc, ST_BREAKDOWN);
  } else {
    if (!c.restart) sc->beta = gam / sc->delta;
    sc->delta = gam;
    sc->phase = PH_ITER;
  }
}

template <class T, int SX, int SY, int E = E_Q1>
__global__ void __launch_bounds__(SX* SY) k_cheb(const SimDev* __restrict__ sims, const int2* __restrict__ work,
                                                 const int* __restrict__ nwork_p) {
  __shared__ OpSmem<E, T, SX, SY> sh;
  __shared__ double red[32];
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
    if (c.phase != PH_CHEB) continue;
    const Geo g(s);
    const TileCoords tc = tile_coords<SX, SY>(s, wi.y);
    ChebPass<T> ps(s, c.cheb_k);
    tile_op_e<E, T, SX, SY>(
        g, s, IterVecs<T>::coef(s), tc.i0, tc.j0, tc.k0, tc.nzt, (T)s.inv_dt, (T)s.theta, true, sh,
        [&](int m, bool live) { return ps.fetch(m, live); }, [&](const ChRaw<T>& v) { return ps.value(v); },
        [&](int m, bool dir, T y, T v) { ps.out(m, dir, y, v); });
    const T accv[1] = {ps.acc};
    double tot[1];
    if (finish_item<T, 1>(s, wi.y, s.ntiles, accv, tot, red)) cheb_close(s, c, tot[0]);
  }
}

// Warp-segment form of k_cheb (the register-prefetch march of k_apply_dot_w).
template <class T, int SX, int NY, int WARPS, int MINB, int E = E_Q1>
__global__ void __launch_bounds__(32 * WARPS, MINB) k_cheb_w(const SimDev* __restrict__ sims,
                                                              const int2* __restrict__ work,
                                                              const int* __restrict__ nwork_p) {
  constexpr int SPC = WARPS * (32 / SX);  // segments per block
  __shared__ double red[32];
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
    if (c.phase != PH_CHEB) continue;
    const Geo g(s);
    const int tile = wi.y * SPC + (int)threadIdx.x / SX;
    const bool active = tile < s.w_ntiles;
    const int tx = tile % s.w_ntx, rem = tile / s.w_ntx, ty = rem % s.w_nty, tz = rem / s.w_nty;
    ChebPass<T> ps(s, c.cheb_k);
    warp_tile_op_e<E, T, SX, NY>(
        g, s, IterVecs<T>::coef(s), active, tx * (SX - 2), ty * NY, tz * s.w_tz, s.w_tz, (T)s.inv_dt, (T)s.theta,
        true, [&](int m, bool live) { return ps.fetch(m, live); }, [&](const ChRaw<T>& v) { return ps.value(v); },
        [&](int m, bool dir, T y, T v) { ps.out(m, dir, y, v); });
    const T accv[1] = {ps.acc};
    double tot[1];
    if (finish_item<T, 1>(s, wi.y, s.w_items, accv, tot, red)) cheb_close(s, c, tot[0]);
  }
}

// ---------------------------------------------------------------- k_cg_iter

// Loads and node-local updates of the fused FP32 iteration, one level ahead
// in registers (the RegSrc contract of op_warp.cuh). For every staged row it
// forms s = w + beta s_old, r' = r - alpha s and the operator input
// u' = P^-1 r'; for the rows this lane owns it also writes r', s,
// p = P^-1 r + beta p_old and e += alpha p, and sums r'.u'.
//   mode 0 (restart): u = P^-1 r, nothing written;
//   mode 1 (first update): beta = 0, p_old and e not read (e starts at 0);
//   mode 2: general update.
template <int NY>
struct CgSrc {
  static constexpr int NR = NY + 2, NF = NY + 1;
  struct Raw {
    float r, w, so, p;
  };
  const float* __restrict__ r;
  const float* __restrict__ w;
  const float* __restrict__ so;
  const float* __restrict__ pinv;
  float* __restrict__ pvec;  // p, read (mode 2) and written in place by its owner
  float* __restrict__ e;     // x of the inner solve, likewise
  float* __restrict__ rnew;
  float* __restrict__ snew;
  const float2* __restrict__ coef;
  float alpha, beta;
  int mode, k0, tzl;
  Raw raw[NR];
  float pp[NY], ee[NY];  // p_old, e of the owned rows of the staged level
  float2 cf[NF];
  float gam = 0.f;  // this thread's part of r'.u' over owned nodes

  __device__ __forceinline__ bool owned_level(const LaneGeo<NY>& lg, int L) const {
    return lg.out_lane && L >= k0 && L < k0 + tzl && L <= lg.gnz;
  }
  __device__ __forceinline__ void load_nodes(const LaneGeo<NY>& lg, int L) {
    const unsigned lv = lg.live_rows(L);
    const int off = lg.nbase + L * lg.pxy;
    const bool own = owned_level(lg, L);
#pragma unroll
    for (int row = 0; row < NR; ++row) {
      const int m = off + row * lg.px;
      const bool live = ((lv >> row) & 1u) && HEAT_INDEX_OK(lg.sc, m, lg.nn);
      Raw z = {0.f, 0.f, 0.f, 0.f};
      if (live) {
        z.r = r[m];
        z.p = pinv[m];
        if (mode > 0) z.w = w[m];
        if (mode > 1) z.so = so[m];
      }
      raw[row] = z;
      if (row >= 1 && row <= NY) {
        const bool o = own && live && mode > 1;
        pp[row - 1] = o ? pvec[m] : 0.f;
        ee[row - 1] = o ? e[m] : 0.f;
      }
    }
  }
  __device__ __forceinline__ void load_coef(const LaneGeo<NY>& lg, int E) {
    const unsigned le = lg.live_elems(E);
#pragma unroll
    for (int row = 0; row < NF; ++row) {
      const int e = lg.ebase + row * lg.enx + E * lg.estride;
      cf[row] = (((le >> row) & 1u) && HEAT_INDEX_OK(lg.sc, e, lg.ne)) ? coef[e] : make_float2(0.f, 0.f);
    }
  }
  __device__ __forceinline__ void prologue(const LaneGeo<NY>& lg, int) {
    load_nodes(lg, k0 - 1);
    load_coef(lg, k0 - 1);
  }
  __device__ __forceinline__ void level(const LaneGeo<NY>& lg, int t, int tz, float v[NR]) {
    const int L = k0 - 1 + t;
    const unsigned lv = lg.live_rows(L);
    const bool own = owned_level(lg, L);
    const int off = lg.nbase + L * lg.pxy;
#pragma unroll
    for (int row = 0; row < NR; ++row) {
      const Raw& a = raw[row];
      if (mode == 0) {
        v[row] = a.p * a.r;
        if (row >= 1 && row <= NY && own) gam += a.r * v[row];
      } else {
        const float sv = a.w + beta * a.so;  // so = 0 in mode 1
        const float rn = a.r - alpha * sv;
        v[row] = a.p * rn;
        if (row >= 1 && row <= NY && own && ((lv >> row) & 1u) && HEAT_INDEX_OK(lg.sc, off + row * lg.px, lg.nn)) {
          const int m = off + row * lg.px;
          const float pn = a.p * a.r + beta * pp[row - 1];
          rnew[m] = rn;
          snew[m] = sv;
          pvec[m] = pn;
          e[m] = ee[row - 1] + alpha * pn;
          gam += rn * v[row];
        }
      }
    }
    if (t <= tz) load_nodes(lg, k0 + t);  // in flight during this level's arithmetic
  }
  __device__ __forceinline__ float2 coef_row(int, int row) const { return cf[row]; }
  __device__ __forceinline__ void after_elements(const LaneGeo<NY>& lg, int t, int tz) {
    if (t <= tz) load_coef(lg, k0 - 1 + t);
  }
};

// One CG iteration of the FP32 inner solve in one kernel (the
// Chronopoulos-Gear arrangement of PCG: the apply acts on the new
// preconditioned residual, so both inner products of an iteration come from
// one reduction). With the slots cur and nxt = cur ^ 1 of r, w, s:
//   s = w + beta s_old, p = P^-1 r + beta p, e += alpha p, r' = r - alpha s,
//   u' = P^-1 r', w' = A' u', gamma = r'.u', delta = w'.u',
//   beta' = gamma / gamma_old, alpha' = gamma / (delta - beta' gamma / alpha).
// A restart (after k_open) computes w = A' u for u = P^-1 r and
// alpha = r.u / w.u without updating. Same work lists and results contract as
// k_apply_dot_w; the convergence tests of k_update (gamma is the r.P^-1 r of
// Algorithm 1).
template <int SX, int NY, int WARPS, int MINB, int E = E_Q1>
__global__ void __launch_bounds__(32 * WARPS, MINB) k_cg_iter(const SimDev* __restrict__ sims,
                                                               const int2* __restrict__ work,
                                                               const int* __restrict__ nwork_p) {
  constexpr int SPC = WARPS * (32 / SX);  // segments per block
  __shared__ double red[2 * 32];
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
    if (c.phase != PH_ITER) continue;
    const Geo g(s);
    const int tile = wi.y * SPC + (int)threadIdx.x / SX;
    const bool active = tile < s.w_ntiles;
    const int tx = tile % s.w_ntx, rem = tile / s.w_ntx, ty = rem % s.w_nty, tz = rem / s.w_nty;
    const int slot = c.cgs, nslot = slot ^ 1;
    const int mode = c.restart ? 0 : (c.iter == 0 ? 1 : 2);
    CgSrc<NY> src;
    src.r = s.rc32[slot];
    src.w = s.wc32[slot];
    src.so = s.sc32[slot];
    src.pinv = s.pinv32;
    src.pvec = s.p32;
    src.e = s.e32;
    src.rnew = s.rc32[nslot];
    src.snew = s.sc32[nslot];
    src.coef = s.coef32;
    src.alpha = mode == 0 ? 0.f : (float)c.alpha;
    src.beta = mode == 2 ? (float)c.beta : 0.f;
    src.mode = mode;
    src.k0 = tz * s.w_tz;
    src.tzl = s.w_tz;
    float* __restrict__ wout = mode == 0 ? s.wc32[slot] : s.wc32[nslot];
    float del = 0.f;
    const LaneGeo<NY> lg(g, active, (int)threadIdx.x % SX, SX, tx * (SX - 2), ty * NY, true, s.sc);
    warp_march_e<E, float, SX, NY>(lg, s, src, s.w_tz, (float)s.inv_dt, (float)s.theta,
                                   [&](int m, bool dir, float y, float v) {
                                     const float wv = dir ? 0.f : y;
                                     wout[m] = wv;
                                     del += v * wv;
                                   });
    const float accv[2] = {src.gam, del};
    double tot[2];
    if (finish_item<float, 2>(s, wi.y, s.w_items, accv, tot, red)) {
      SimScalars* sc = s.sc;
      sc->count = 0;
      const double gam = tot[0], dlt = tot[1];
      if (!isfinite(gam) || !isfinite(dlt)) {
        fail(sc, ST_NONFINITE);
      } else if (mode == 0) {
        sc->delta = gam;
        if (!(dlt > 0.0)) {
          fail(sc, ST_BREAKDOWN);
        } else {
          sc->alpha = gam / dlt;
          sc->beta = 0.0;
          sc->restart = 0;
        }
      } else {
        const double bnew = gam / sc->delta;
        sc->iter += 1;
        sc->iter_step += 1;
        sc->cgs = nslot;
        sc->delta = gam;
        const int cap = (s.prec == P_FP32_PLAIN) ? s.max_iter : s.inner_max_iter;
        if (sc->iter_step >= s.max_iter) {
          fail(sc, ST_NOT_CONVERGED);
        } else if (gam <= sc->thresh_in || sc->iter >= cap) {
          sc->phase = PH_OUTER;
        } else {
          const double den = dlt - bnew * gam / sc->alpha;
          if (!(den > 0.0)) {
            fail(sc, ST_BREAKDOWN);
          } else {
            sc->alpha = gam / den;
            sc->beta = bnew;
          }
        }
      }
    }
  }
}

// ---------------------------------------------------------------- k_update

// Four consecutive node values (a float4, or two double2).
template <class T> struct Quad;
template <> struct Quad<float> {
  float v[4];
  template <bool CG>
  __device__ __forceinline__ void load(const float* p) {
    const float4 t = ld_vec<CG>(reinterpret_cast<const float4*>(p));
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  }
  __device__ __forceinline__ void store(float* p) const {
    *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
  }
};
template <> struct Quad<double> {
  double v[4];
  template <bool CG>
  __device__ __forceinline__ void load(const double* p) {
    const double2 a = ld_vec<CG>(reinterpret_cast<const double2*>(p)),
                  b = ld_vec<CG>(reinterpret_cast<const double2*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
  __device__ __forceinline__ void store(double* p) const {
    reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
  }
};

// One work item of k_update (pw_chunk(QPT) nodes of one simulation in phase
// PH_ITER). VT > 1: a block of kPwThreads / VT threads does the item, each
// thread the work of VT threads of a kPwThreads block in the same order, so
// the item's results and partial are bitwise those of k_update. CG: vectors
// are loaded through L2 only (see ld_vec). Returns true in thread 0 of the
// block that finished the simulation's last item when the simulation stays
// in PH_ITER (another iteration follows).
template <class T, int P, int QPT, int VT, bool CG>
__device__ __forceinline__ bool update_item(const SimDev& s, const Ctl& c, int item, double* red) {
  const bool resid_it = (P == P_FP64) && s.resid_period > 0 && c.iter > 0 && (c.iter % s.resid_period) == 0;
  const int nn = (int)s.nn;
  const int base = item * pw_chunk(QPT);
  const int end = min(base + pw_chunk(QPT), nn);
  T* __restrict__ x = (P == P_FP64) ? reinterpret_cast<T*>(s.vec64[c.ix]) : reinterpret_cast<T*>(s.e32);
  T* __restrict__ r = const_cast<T*>(IterVecs<T>::r(s));
  const T* __restrict__ pinv = IterVecs<T>::pinv(s);
  const T* __restrict__ d = IterVecs<T>::d(s, c.id);
  const T* __restrict__ q = IterVecs<T>::q(s);
  const T alpha = (T)c.alpha;
  const bool zero_x = (P != P_FP64) && c.iter == 0;  // the inner solve starts from e = 0
  const int vblock = VT * (int)blockDim.x;             // threads of the block this one stands in for
  T part[VT];  // per-(virtual-)thread partials in T, FP64 from the warp sums on
#pragma unroll
  for (int vt = 0; vt < VT; ++vt) {
    const int tid = (int)threadIdx.x + vt * (int)blockDim.x;
    T pacc = T(0);
    // QPT groups of 4 nodes per thread, group u at base + 4*tid + u*4*vblock
    // (coalesced per group); every load is issued before any result is used
    Quad<T> xv[QPT], dv[QPT], rv[QPT], qv[QPT], pv[QPT];
    bool full[QPT];
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
      const int n = base + 4 * (tid + u * vblock);
      full[u] = n + 3 < end;
      if (full[u]) {
        dv[u].template load<CG>(d + n);
        if (!zero_x) xv[u].template load<CG>(x + n);
        if (!resid_it) {
          rv[u].template load<CG>(r + n);
          qv[u].template load<CG>(q + n);
          pv[u].template load<false>(pinv + n);
        }
      }
    }
#pragma unroll
    for (int u = 0; u < QPT; ++u) {
      const int n = base + 4 * (tid + u * vblock);
      if (full[u]) {
#pragma unroll
        for (int a = 0; a < 4; ++a) xv[u].v[a] = (zero_x ? T(0) : xv[u].v[a]) + alpha * dv[u].v[a];
        xv[u].store(x + n);
        if (!resid_it) {
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            rv[u].v[a] -= alpha * qv[u].v[a];
            pacc += rv[u].v[a] * rv[u].v[a] * pv[u].v[a];
          }
          rv[u].store(r + n);
        }
      } else {
        for (int m = n; m < end; ++m) {  // ragged end of the mesh
          x[m] = (zero_x ? T(0) : ld_vec<CG>(x + m)) + alpha * ld_vec<CG>(d + m);
          if (!resid_it) {
            const T rn = ld_vec<CG>(r + m) - alpha * ld_vec<CG>(q + m);
            r[m] = rn;
            pacc += rn * rn * pinv[m];
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < VT; ++k)
      if (k == vt) part[k] = pacc;
  }
  double pd[1];
  bool more = false;
  if (finish_item<T, 1, VT>(s, item, s.npw, part, pd, red)) {
    SimScalars* sc = s.sc;
    sc->count = 0;
    if (resid_it) {
      sc->phase = PH_RESID;  // k_open recomputes r = b - A x and finishes the iteration
    } else {
      const double dn = pd[0];
      // The stopping tests use r^T P^-1 r (Algorithm 1) with either
      // preconditioner; with Chebyshev passes they form delta = r^T z and beta.
      const bool ch = s.cheb_m >= 2;
      if (!ch) {
        sc->beta = dn / sc->delta;
        sc->delta = dn;
      }
      sc->iter += 1;
      sc->iter_step += 1;
      if (!isfinite(dn)) {
        fail(sc, ST_NONFINITE);
      } else if (P == P_FP64) {
        // The recurrence residual drifts from b - A x (by far more than
        // rounding on stiff systems), so a step closes only on the true
        // residual: k_open recomputes it and closes or continues.
        if (dn <= sc->thresh) {
          sc->confirm = 1;
          sc->phase = PH_RESID;
        } else if (sc->iter_step >= s.max_iter) fail(sc, ST_NOT_CONVERGED);
        else if (ch) enter_iter(s, sc);
        else more = true;
      } else {
        const int cap = (s.prec == P_FP32_PLAIN) ? s.max_iter : s.inner_max_iter;
        if (sc->iter_step >= s.max_iter) fail(sc, ST_NOT_CONVERGED);
        else if (dn <= sc->thresh_in || sc->iter >= cap) sc->phase = PH_OUTER;
        else if (ch) enter_iter(s, sc);
        else more = true;
      }
    }
  }
  return more;
}

template <class T, int P, int QPT>
__global__ void __launch_bounds__(kPwThreads, pw_min_blocks(QPT, sizeof(T))) k_update(const SimDev* __restrict__ sims, const int2* __restrict__ work,
                                                       const int* __restrict__ nwork_p) {
  __shared__ double red[32];
  __shared__ ItemCache cache;
  int cur = -1;
  bool dep = false;
  allow_next_launch();
  const int nwork = *nwork_p;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 wi = work[w];
    cache_sim(sims, wi.x, cache, cur, dep);
    if (cache.c.phase != PH_ITER) continue;
    update_item<T, P, QPT, 1, false>(cache.s, cache.c, wi.y, red);
  }
}

}  // namespace heat
