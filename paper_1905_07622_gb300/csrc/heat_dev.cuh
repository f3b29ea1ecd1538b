// Device-side data of the solver: per-simulation descriptors and scalars,
// Q1 element-matrix classes, node/boundary helpers and reductions.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace heat {

// Per-simulation phase of the device-driven step machine. Kernels of a tick
// act only on simulations whose phase matches them, so one launch sequence
// can carry many simulations at different points of their solves.
enum Phase : int {
  PH_IDLE = 0,    // nothing queued
  PH_OPEN = 1,    // start of a step: right-hand side, x0, first residual
  PH_ITER = 2,    // CG iterations (FP64, or FP32 inner solve)
  PH_OUTER = 3,   // FP32 path: x64 += e, FP64 true residual, restart inner
  PH_DONE = 4,    // target step reached
  PH_FAILED = 5,  // status holds the error
  PH_RESID = 6,   // FP64 path: true residual r = b - A x (every resid_period iterations)
  PH_CHEB = 7     // Chebyshev preconditioner z = p_m(D^-1 A) D^-1 r, one operator pass per kernel
};

enum Prec : int { P_FP64 = 0, P_FP32_REFINED = 1, P_FP32_PLAIN = 2 };

// Finite element on each box (heat.h heat_element).
enum Elem : int { E_Q1 = 0, E_P1 = 1 };

// Local corners c, d of a box (c = x | y<<1 | z<<2) share a tetrahedron of
// the six-tetrahedra split iff one is a bitwise subset of the other (the
// tetrahedra are the monotone paths 0 -> e_a -> e_a+e_b -> 7); their
// stiffness coupling vanishes unless they differ in one coordinate at most
// (the gradients of the path's linear functions are axis-aligned).
__host__ __device__ constexpr bool p1_mass_nz(int c, int d) { return (c & d) == c || (c & d) == d; }
__host__ __device__ constexpr bool p1_stiff_nz(int c, int d) {
  return c == d || (c ^ d) == 1 || (c ^ d) == 2 || (c ^ d) == 4;
}

// Status codes shared with heat.h.
enum : int { ST_OK = 0, ST_NOT_CONVERGED = 4, ST_NONFINITE = 5, ST_BREAKDOWN = 8 };

// Device-resident scalars of one simulation (also mirrored to pinned host
// memory for polling). Written only by the last block of a kernel for that
// simulation, read by every block of later kernels.
struct SimScalars {
  int phase;
  int status;
  int step;        // completed steps since the last set_state
  int target;      // phase becomes DONE when step == target
  int iter;        // CG iterations of the current (inner) solve
  int iter_step;   // CG iterations of the current step (inner + outer)
  int outer;       // refinement sweeps of the current step
  int restart;     // next apply takes d = P^-1 r (no previous direction)
  int have_prev;   // U^{n-2} holds a valid state
  int iu1, iu2, ix, ixa;  // vec64 pool slots: U^{n-1}, U^{n-2}, x, spare
  int id;          // current direction slot (0/1)
  int max_iters_step;
  unsigned int count;  // tiles finished in the running kernel
  int cgs;             // FP32 fused iteration: current slot of r, w, s (0/1)
  int y_valid;         // bit v: yv[v] holds A' vec64[v] (FP32 paths, see k_open)
  int cheb_k;          // next Chebyshev pass (1 .. cheb_m - 1) while phase is PH_CHEB
  int confirm;         // FP64 path: the running PH_RESID pass confirms convergence (not an iteration)
  unsigned int check_violations;  // out-of-range indices met (HEAT_CHECK builds)
  double delta;    // r^T P^-1 r of the current solve
  double delta_b;  // b^T P^-1 b of the step
  double thresh;   // rtol^2 * delta_b
  double thresh_in;  // inner threshold (FP32 paths)
  double alpha, beta, dq;
  double delta_out;  // FP64 true-residual r^T P^-1 r (FP32 paths)
  double rel_res;    // sqrt(delta / delta_b) at the last step close
  long long iters_total;  // CG iterations since the counters were cleared
  long long outer_total;
  long long steps_total;
};

struct alignas(16) SimDev {  // 16-byte aligned: blocks copy it with uint4 loads
  int nx, ny, nz;             // elements per dimension
  int ntx, nty, ntz, ntiles;  // operator tiles (x, y, z counts and total)
  int tz_len;                 // node levels per operator tile
  int npw;                    // pointwise work items (pw_chunk nodes each)
  // warp-segment tiles of the FP32 apply: (SX-2) x NY x w_tz nodes each
  int w_ntx, w_nty, w_ntz, w_tz, w_ntiles;
  int w_items;                // work items (groups of segment tiles per block)
  int fused;                  // the engine runs the FP32 inner solve as one fused kernel per iteration
  int w_pad_;
  // warp-segment tiles of the step-start and refinement passes (k_open_w):
  // (SX-2) x NY x o_tz nodes each, o_items work items
  int o_ntx, o_nty, o_ntz, o_tz, o_ntiles, o_items;
  long long nn;               // nodes
  uint32_t dir_faces;         // Dirichlet face bits
  int prec;                   // Prec
  int max_iter, resid_period, max_outer, flux_steps;
  int inner_max_iter;
  int cheb_m;                 // Chebyshev preconditioner degree (>= 2), 0: Jacobi (Algorithm 1)
  int elem;                   // Elem: finite element on each box
  int pad_elem_;
  double g[6];                // Dirichlet values
  double inv_dt, theta, rtol, inner_rtol;
  double mhat[8], khat[8];    // element mass/stiffness entry by corner XOR pattern
  float mhat_f[8], khat_f[8];
  // Eigenvalues of the element mass and stiffness matrices in the element's
  // Walsh basis (index w = wx | wy<<1 | wz<<2), divided by 8 (the inverse
  // transform's normalisation): lam_m[w] = prod_d (w_d ? h_d/6 : h_d/2) / 8,
  // lam_k[w] = sum_d (w_d ? 2/h_d : 0) prod_{d' != d} (...) / 8.
  double lam_m[8], lam_k[8];
  float lam_m_f[8], lam_k_f[8];
  const double2* coef;        // (rho_c, k) per element
  const float2* coef32;
  double* vec64[4];           // U^{n-1}, U^{n-2}, x and spare (slots in SimScalars)
  double* yv[4];              // A' vec64[v] where SimScalars.y_valid says so
  double* b;
  double* r;
  double* q;
  double* d[2];
  double* pinv;
  double* zlift;              // A_{.D} g on free rows (Dirichlet lift)
  double* F;                  // face flux vector
  float* r32;
  float* q32;
  float* e32;
  float* d32[2];
  float* pinv32;
  // The fused FP32 iteration (one kernel per CG iteration, see k_cg_iter):
  // r, w = A u and s = A p in two slots each (slot cgs is current), p.
  // rc32[0] = r32, wc32[0] = q32, sc32 = d32.
  float* rc32[2];
  float* wc32[2];
  float* sc32[2];
  float* p32;
  // Chebyshev preconditioner (cheb_m >= 2): z, the polynomial's residual res
  // and its two step vectors dd. FP32: z32, rc32[1], wc32[1], p32 (the fused
  // iteration's slots, idle on the non-fused kernels the preconditioner runs
  // with); FP64: yv[0..3] (the stored products are an FP32-path device).
  float* z32;
  // [0] 1/theta, [2k-1], [2k] the step-k coefficients rho_k rho_{k-1} and
  // 2 rho_k / delta (k = 1..7), [16] lam_lo, [17] lam_hi, [18] the bound's
  // running maximum as bits (see k_cheb_bound)
  double* cheb;
  // Six-tetrahedra boxes (elem == E_P1): the box's 8x8 mass and stiffness
  // matrices M' (entries 0..63, row-major by local corner) and K' (64..127),
  // FP64 and FP32 copies.
  const double* p1w;
  const float* p1w_f;
  // their structure for the box-centred form (op_warp.cuh): V / 20 and
  // V / h_a^2 (a = x, y, z) with V = hx hy hz / 6
  double p1c[4];
  float p1c_f[4];
  // Trilinear boxes: per element the A operator's (sa = 1/dt, sb = theta)
  // Walsh-pair coefficients A_q, B_q (q = 0..3) of the factorised form
  // (op.cuh), 64 bytes each: FP64 on the FP64 path, double-float pairs on
  // the FP32 paths (the arithmetic of their step-start and refinement passes).
  const float4* acoef;
  double* partial;            // 2 per tile
  int* iters_log;             // CG iterations of each step
  int iters_log_len;
  SimScalars* sc;
};

// Compiled-in index checks (the library built with -DHEAT_CHECK): a node or
// element index outside [0, n) is counted in SimScalars.check_violations and
// the access it guards is skipped. In normal builds the test is the constant
// true and costs nothing.
#ifdef HEAT_CHECK
__device__ __forceinline__ bool heat_index_ok(SimScalars* sc, long long idx, long long n) {
  if (idx >= 0 && idx < n) return true;
  atomicAdd(&sc->check_violations, 1u);
  return false;
}
#define HEAT_INDEX_OK(sc, idx, n) ::heat::heat_index_ok((sc), (long long)(idx), (long long)(n))
#else
#define HEAT_INDEX_OK(sc, idx, n) true
#endif

// ---------------------------------------------------------------- helpers

__device__ __forceinline__ long long node_index(const SimDev& s, int i, int j, int k) {
  return (long long)i + (long long)(s.nx + 1) * ((long long)j + (long long)(s.ny + 1) * k);
}

__device__ __forceinline__ bool inside_nodes(const SimDev& s, int i, int j, int k) {
  return i >= 0 && j >= 0 && k >= 0 && i <= s.nx && j <= s.ny && k <= s.nz;
}

// Dirichlet test from the node's position (face BCs need no mask array).
__device__ __forceinline__ bool is_dirichlet(const SimDev& s, int i, int j, int k) {
  const uint32_t f = s.dir_faces;
  return ((f & 1u) && i == 0) || ((f & 2u) && i == s.nx) || ((f & 4u) && j == 0) ||
         ((f & 8u) && j == s.ny) || ((f & 16u) && k == 0) || ((f & 32u) && k == s.nz);
}

// Value of a Dirichlet node: the lowest face id that contains it.
__device__ __forceinline__ double dirichlet_value(const SimDev& s, int i, int j, int k) {
  const uint32_t f = s.dir_faces;
  if ((f & 1u) && i == 0) return s.g[0];
  if ((f & 2u) && i == s.nx) return s.g[1];
  if ((f & 4u) && j == 0) return s.g[2];
  if ((f & 8u) && j == s.ny) return s.g[3];
  if ((f & 16u) && k == 0) return s.g[4];
  if ((f & 32u) && k == s.nz) return s.g[5];
  return 0.0;
}

template <class T> struct Coef2;
template <> struct Coef2<double> { using type = double2; };
template <> struct Coef2<float> { using type = float2; };

template <class T> __device__ __forceinline__ const typename Coef2<T>::type* coef_ptr(const SimDev& s);
template <> __device__ __forceinline__ const double2* coef_ptr<double>(const SimDev& s) { return s.coef; }
template <> __device__ __forceinline__ const float2* coef_ptr<float>(const SimDev& s) { return s.coef32; }

template <class T> __device__ __forceinline__ T mhat(const SimDev& s, int p);
template <> __device__ __forceinline__ double mhat<double>(const SimDev& s, int p) { return s.mhat[p]; }
template <> __device__ __forceinline__ float mhat<float>(const SimDev& s, int p) { return s.mhat_f[p]; }
template <class T> __device__ __forceinline__ T khat(const SimDev& s, int p);
template <> __device__ __forceinline__ double khat<double>(const SimDev& s, int p) { return s.khat[p]; }
template <> __device__ __forceinline__ float khat<float>(const SimDev& s, int p) { return s.khat_f[p]; }

// Block-wide sum of NV doubles; result valid in thread 0. `red` holds
// NV * 32 doubles of shared memory.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* red) {
#pragma unroll
  for (int a = 0; a < NV; ++a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[a] += __shfl_down_sync(0xffffffffu, v[a], o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) red[a * 32 + warp] = v[a];
  }
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) {
      double t = lane < nwarps ? red[a * 32 + lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      v[a] = t;
    }
  }
}

}  // namespace heat
