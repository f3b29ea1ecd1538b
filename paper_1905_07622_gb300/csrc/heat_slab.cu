// One simulation split into z-slabs: the partitioned form of the dual-GPU
// split of §4.4, with every slab on this GPU.
//
// The element layers of the mesh are cut into S contiguous ranges. Slab s
// owns the node layers [E_s, E_{s+1}) (the last slab also owns the top layer
// nz) and holds its own copy of every vector over the node layers
// [E_s - 1, E_{s+1}]: its owned layers plus one ghost layer on each side that
// has a neighbour, and the coefficients of every element touching an owned
// node. So the operator, the preconditioner and the right-hand side of an
// owned row need nothing outside the slab once its ghost layers are current.
//
// Halo exchange: whenever a kernel writes a vector that a later operator pass
// reads (the state x, the preconditioned residual u = P^-1 r, and the search
// direction d of Algorithm 1), it also stores the values of the slab's lowest
// and highest owned node layers into the neighbours' ghost layers. Slabs
// exchange one node layer per interface and vector, with no copy kernel of
// its own; between GPUs the same stores would be peer stores.
//
// Reductions: every CG scalar is a sum of per-tile partials. The last block of
// a launch forms each slab's sum in tile order and then adds the slab sums in
// slab order (the allreduce of a multi-GPU run), so results are deterministic.
// Two iteration forms:
//   * merged (Chronopoulos-Gear CG): per iteration one operator pass
//     w = A u with both inner products gamma = r.u and delta = w.u from the
//     same reduction, then one pointwise update (p = u + beta p,
//     s = w + beta s, x += alpha p, r -= alpha s, u = P^-1 r). One reduction
//     per iteration.
//   * Algorithm 1 (§3.3): d = u + beta d staged in the operator pass, q = A d
//     and d.q; then the update x += alpha d, r -= alpha q, u = P^-1 r and r.u.
//     Two reductions per iteration.
// Both recompute the true residual r = b - A x every resid_period iterations
// (Algorithm 1's periodic recomputation), and again when the recurrence
// residual meets the stopping rule: a step closes on the true residual only,
// as on the unsplit FP64 path.
//
// Everything runs in FP64 on trilinear boxes, with the factorised tile
// operator of op.cuh.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "engine.h"
#include "op.cuh"

struct heat_slab;

namespace {

using heat::Geo;
using heat::SimDev;

enum SlabPhase : int {
  SP_IDLE = 0,
  SP_RHS = 1,    // b = L u^{n-1} + F^n - lift, b^T P^-1 b
  SP_OPEN = 2,   // x0 = 2u^{n-1} - u^{n-2}, r = b - A x0, u = P^-1 r, r.u
  SP_ITER = 3,   // operator pass of a CG iteration
  SP_UPD = 4,    // pointwise update of a CG iteration
  SP_TRUE = 5,   // true residual r = b - A x, u = P^-1 r, r.u
  SP_DONE = 6,
  SP_FAILED = 7
};

constexpr int kSX = 16, kSY = 16, kTZ = 8, kThreads = kSX * kSY;
constexpr int kPwChunk = kThreads * 8;  // nodes per pointwise item
constexpr int kMaxSlabs = 4096;
constexpr int kLogCap = 1 << 16;       // per-step iteration log entries

// Vectors of a slab, each over its local node layers (ghosts included).
enum Vec : int { V_R = 0, V_U, V_W, V_P, V_S, V_B, V_PINV, V_LIFT, V_F, V_D0, V_D1, V_X0, V_X1, V_X2, NVEC };

struct SlabPart {
  SimDev g;          // the slab's local mesh (nz = local element layers)
  double* v[NVEC];
  int kg0;           // global node layer of local layer 0
  int own0, own1;    // owned local node layers [own0, own1]
  int lo, hi;        // has a neighbour below / above
  int ntx, nty, ntz; // operator tiles over the owned layers
  int item0, nitems; // its operator work items
  int pw0, npw;      // its pointwise work items
  int pxy;           // nodes per layer
  int nzg;           // element layers of the whole mesh
  int flux_steps;    // F^n = F for steps n <= flux_steps (< 0: always)
  uint32_t dir_global;  // Dirichlet faces of the whole mesh
  double h[3];       // element spacing
};

struct SlabScalars {
  int phase, status, step, target;
  int iter;       // CG iterations of the current step
  int since_true; // iterations since the last true residual
  int have_prev, iu1, iu2, ix, id, restart;
  int iters_step_max, merged, resid_period, max_iter;
  unsigned int count;  // work items finished in the running kernel
  int log_len;
  int confirm;    // the coming SP_TRUE pass confirms a converged recurrence residual
  int pad_;
  long long iters_total, steps_total;
  double delta_b, thresh, gamma, gamma_old, alpha, alpha_old, beta, rel_res, rtol2;
};

__device__ __forceinline__ void fail(SlabScalars* sc, int st) {
  sc->status = st;
  sc->phase = SP_FAILED;
}

// Writes value `val` of vector `vec` at owned local node m of slab s into the
// neighbours' ghost layers when m lies on the slab's lowest or highest owned
// layer.
__device__ __forceinline__ void halo_store(const SlabPart* __restrict__ parts, int s, const SlabPart& P, int vec,
                                           int m, double val) {
  if (P.lo && m < (P.own0 + 1) * P.pxy) {
    const SlabPart& N = parts[s - 1];
    N.v[vec][m - P.own0 * P.pxy + N.g.nz * N.pxy] = val;
  }
  if (P.hi && m >= P.own1 * P.pxy) {
    const SlabPart& N = parts[s + 1];
    N.v[vec][m - P.own1 * P.pxy] = val;
  }
}

// Sums the per-item partials of every slab in item order, then the slab sums
// in slab order. Called by the whole last block; result in thread 0.
template <int NV>
__device__ void slab_allreduce(const SlabPart* __restrict__ parts, int nslabs, const double* __restrict__ partials,
                               bool pointwise, double (&tot)[NV], double* red) {
  double acc[NV];
#pragma unroll
  for (int a = 0; a < NV; ++a) acc[a] = 0.0;
  for (int s = 0; s < nslabs; ++s) {
    const int i0 = pointwise ? parts[s].pw0 : parts[s].item0;
    const int n = pointwise ? parts[s].npw : parts[s].nitems;
    double v[NV];
#pragma unroll
    for (int a = 0; a < NV; ++a) v[a] = 0.0;
    for (int t = threadIdx.x; t < n; t += blockDim.x) {
#pragma unroll
      for (int a = 0; a < NV; ++a) v[a] += __ldcg(&partials[(long long)(i0 + t) * NV + a]);
    }
    heat::block_sum<NV>(v, red);
    if (threadIdx.x == 0) {
#pragma unroll
      for (int a = 0; a < NV; ++a) acc[a] += v[a];
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < NV; ++a) tot[a] = acc[a];
}

// Publishes this item's partials and reports whether it was the launch's last.
template <int NV>
__device__ __forceinline__ bool publish(double (&v)[NV], double* red, double* __restrict__ partials, int item,
                                        int nitems, SlabScalars* sc, int* s_last) {
  heat::block_sum<NV>(v, red);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int a = 0; a < NV; ++a) partials[(long long)item * NV + a] = v[a];
    __threadfence();
    *s_last = atomicAdd(&sc->count, 1u) == (unsigned int)(nitems - 1);
  }
  __syncthreads();
  const bool last = *s_last != 0;
  if (last) __threadfence();
  return last;
}

// Step close (thread 0 of the last block): log, rotate the state ring.
__device__ void close_step(SlabScalars* sc, int* log, double gamma) {
  sc->rel_res = sc->delta_b > 0.0 ? sqrt(fmax(gamma, 0.0) / sc->delta_b) : 0.0;
  sc->iters_total += sc->iter;
  sc->iters_step_max = max(sc->iters_step_max, sc->iter);
  if (sc->log_len < kLogCap) log[sc->log_len++] = sc->iter;
  const int t = sc->iu2;
  sc->iu2 = sc->iu1;
  sc->iu1 = sc->ix;
  sc->ix = t;
  sc->have_prev = 1;
  sc->step += 1;
  sc->steps_total += 1;
  sc->phase = sc->step >= sc->target ? SP_DONE : SP_RHS;
}

struct Ctl {
  int phase, iu1, iu2, ix, id, restart, have_prev, merged, step;
  double alpha, beta;
};

// The operator passes: RHS, OPEN, TRUE and the iteration's apply, chosen by
// the phase. Work items are (slab, tile) pairs; a tile is (SX-1) x (SY-1) node
// columns by up to kTZ owned node layers.
__global__ void __launch_bounds__(kThreads) k_slab_op(const SlabPart* __restrict__ parts, int nslabs,
                                                     const int2* __restrict__ items, int nitems,
                                                     double* __restrict__ partials, SlabScalars* sc, int* log) {
  __shared__ heat::TileSmem<double, kSX, kSY> sh;
  __shared__ double red[64];
  __shared__ int s_last;
  __shared__ Ctl c;
  if (threadIdx.x == 0) {
    c.phase = __ldcg(&sc->phase);
    c.iu1 = __ldcg(&sc->iu1);
    c.iu2 = __ldcg(&sc->iu2);
    c.ix = __ldcg(&sc->ix);
    c.id = __ldcg(&sc->id);
    c.restart = __ldcg(&sc->restart);
    c.have_prev = __ldcg(&sc->have_prev);
    c.merged = __ldcg(&sc->merged);
    c.step = __ldcg(&sc->step);
    c.alpha = __ldcg(&sc->alpha);
    c.beta = __ldcg(&sc->beta);
  }
  __syncthreads();
  const int phase = c.phase;
  if (phase != SP_RHS && phase != SP_OPEN && phase != SP_ITER && phase != SP_TRUE) return;
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int2 it = items[w];
    const int s = it.x;
    const SlabPart& P = parts[s];
    const SimDev& sd = P.g;
    const Geo g(sd);
    const int t = it.y;
    const int tx = t % P.ntx, ty = (t / P.ntx) % P.nty, tz = t / (P.ntx * P.nty);
    const int i0 = tx * (kSX - 1), j0 = ty * (kSY - 1), k0 = P.own0 + tz * kTZ;
    const int nzt = min(kTZ, P.own1 + 1 - k0);
    double part[2] = {0.0, 0.0};
    double* const* v = P.v;
    const double idt = sd.inv_dt, th = sd.theta;
    if (phase == SP_RHS) {
      const double* __restrict__ u1 = v[V_X0 + c.iu1];
      const bool fon = P.flux_steps < 0 || c.step + 1 <= P.flux_steps;  // the step being solved is step + 1
      heat::tile_op<double, kSX, kSY>(
          g, sd, sd.coef, i0, j0, k0, nzt, idt, th - 1.0, false, sh,
          [&](int m, bool live) -> double { return live ? u1[m] : 0.0; }, [](double x) { return x; },
          [&](int m, bool dir, double y, double) {
            const double bb = dir ? 0.0 : y + (fon ? v[V_F][m] : 0.0) - v[V_LIFT][m];
            v[V_B][m] = bb;
            part[0] += bb * bb * v[V_PINV][m];
          });
    } else if (phase == SP_OPEN || phase == SP_TRUE) {
      const bool open = phase == SP_OPEN;
      const double* __restrict__ u1 = v[V_X0 + c.iu1];
      const double* __restrict__ u2 = v[V_X0 + c.iu2];
      const double* __restrict__ xs = v[V_X0 + c.ix];
      const bool extrap = open && c.have_prev;
      // r = b - A_ff x_f: Dirichlet columns are masked (b carries the lift).
      // x is written on free nodes only; every state slot holds g on the
      // Dirichlet nodes from heat_slab_set_state on.
      heat::tile_op<double, kSX, kSY>(
          g, sd, sd.coef, i0, j0, k0, nzt, idt, th, true, sh,
          [&](int m, bool live) -> double2 {
            if (!live) return make_double2(0.0, 0.0);
            if (!open) return make_double2(xs[m], 0.0);
            return make_double2(u1[m], extrap ? u2[m] : 0.0);
          },
          [&](double2 a) { return extrap ? 2.0 * a.x - a.y : a.x; },
          [&](int m, bool dir, double y, double xv) {
            if (open && !dir) {
              v[V_X0 + c.ix][m] = xv;
              halo_store(parts, s, P, V_X0 + c.ix, m, xv);
            }
            const double r = dir ? 0.0 : v[V_B][m] - y;
            const double u = v[V_PINV][m] * r;
            v[V_R][m] = r;
            v[V_U][m] = u;
            halo_store(parts, s, P, V_U, m, u);
            part[0] += r * u;
          });
    } else if (c.merged) {  // SP_ITER, merged form: w = A u, r.u and w.u
      const double* __restrict__ u = v[V_U];
      heat::tile_op<double, kSX, kSY>(
          g, sd, sd.coef, i0, j0, k0, nzt, idt, th, true, sh,
          [&](int m, bool live) -> double { return live ? u[m] : 0.0; }, [](double x) { return x; },
          [&](int m, bool dir, double y, double uv) {
            const double wv = dir ? 0.0 : y;
            v[V_W][m] = wv;
            part[0] += v[V_R][m] * uv;
            part[1] += wv * uv;
          });
    } else {  // SP_ITER, Algorithm 1: d = u + beta d_old staged, q = A d, d.q
      const double* __restrict__ u = v[V_U];
      const double* __restrict__ dold = v[V_D0 + c.id];
      const int dn = V_D0 + (c.id ^ 1);
      const double beta = c.restart ? 0.0 : c.beta;
      const bool rs = c.restart != 0;
      heat::tile_op<double, kSX, kSY>(
          g, sd, sd.coef, i0, j0, k0, nzt, idt, th, true, sh,
          [&](int m, bool live) -> double2 {
            if (!live) return make_double2(0.0, 0.0);
            return make_double2(u[m], rs ? 0.0 : dold[m]);
          },
          [&](double2 a) { return a.x + beta * a.y; },
          [&](int m, bool dir, double y, double dv) {
            const double q = dir ? 0.0 : y;
            v[dn][m] = dv;
            halo_store(parts, s, P, dn, m, dv);
            v[V_W][m] = q;
            part[0] += dv * q;
          });
    }
    if (!publish<2>(part, red, partials, w, nitems, sc, &s_last)) continue;
    double tot[2];
    slab_allreduce<2>(parts, nslabs, partials, false, tot, red);
    if (threadIdx.x == 0) {
      sc->count = 0;
      const double th2 = sc->thresh;
      if (!isfinite(tot[0]) || !isfinite(tot[1])) {
        fail(sc, heat::ST_NONFINITE);
      } else if (phase == SP_RHS) {
        sc->delta_b = tot[0];
        sc->thresh = sc->rtol2 * tot[0];
        sc->phase = SP_OPEN;
      } else if (phase == SP_OPEN) {
        sc->iter = 0;
        sc->since_true = 0;
        sc->confirm = 0;
        sc->restart = 1;
        sc->gamma = tot[0];
        if (tot[0] <= th2) close_step(sc, log, tot[0]);
        else sc->phase = SP_ITER;
      } else if (phase == SP_TRUE) {
        sc->since_true = 0;
        // Algorithm 1's periodic pass: the true residual replaces the
        // recurrence's and forms beta; a confirmation keeps the iteration's beta
        if (!c.merged && !sc->confirm) sc->beta = sc->gamma > 0.0 ? tot[0] / sc->gamma : 0.0;
        sc->confirm = 0;
        sc->gamma = tot[0];
        if (tot[0] <= th2) close_step(sc, log, tot[0]);
        else sc->phase = SP_ITER;
      } else if (c.merged) {
        const double gam = tot[0], del = tot[1];
        sc->gamma = gam;
        if (gam <= th2) {
          sc->phase = SP_TRUE;  // confirm on the true residual
        } else {
          double beta = 0.0, alpha;
          if (c.restart) {
            alpha = del > 0.0 ? gam / del : -1.0;
          } else {
            beta = gam / sc->gamma_old;
            const double den = del - beta * gam / sc->alpha_old;
            alpha = den > 0.0 ? gam / den : -1.0;
          }
          if (!(alpha > 0.0)) {
            fail(sc, heat::ST_BREAKDOWN);
          } else {
            sc->alpha = alpha;
            sc->beta = beta;
            sc->gamma_old = gam;
            sc->alpha_old = alpha;
            sc->restart = 0;
            sc->phase = SP_UPD;
          }
        }
      } else {
        const double dq = tot[0];
        if (!(dq > 0.0)) {
          fail(sc, heat::ST_BREAKDOWN);
        } else {
          sc->alpha = sc->gamma / dq;
          sc->id ^= 1;
          sc->restart = 0;
          sc->phase = SP_UPD;
        }
      }
    }
  }
}

// The pointwise update of a CG iteration over the owned nodes of every slab;
// work items are (slab, chunk of kPwChunk owned nodes).
__global__ void __launch_bounds__(kThreads) k_slab_pw(const SlabPart* __restrict__ parts, int nslabs,
                                                     const int2* __restrict__ items, int nitems,
                                                     double* __restrict__ partials, SlabScalars* sc, int* log) {
  __shared__ double red[32];
  __shared__ int s_last;
  __shared__ Ctl c;
  if (threadIdx.x == 0) {
    c.phase = __ldcg(&sc->phase);
    c.id = __ldcg(&sc->id);
    c.ix = __ldcg(&sc->ix);
    c.merged = __ldcg(&sc->merged);
    c.alpha = __ldcg(&sc->alpha);
    c.beta = __ldcg(&sc->beta);
  }
  __syncthreads();
  if (c.phase != SP_UPD) return;
  const double alpha = c.alpha, beta = c.beta;
  const int xs = V_X0 + c.ix;
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int2 it = items[w];
    const int s = it.x;
    const SlabPart& P = parts[s];
    double* const* v = P.v;
    const int m0 = P.own0 * P.pxy + it.y * kPwChunk;
    const int m1 = min(m0 + kPwChunk, (P.own1 + 1) * P.pxy);
    double part[1] = {0.0};
    if (c.merged) {
      for (int m = m0 + (int)threadIdx.x; m < m1; m += kThreads) {
        const double u = v[V_U][m], wv = v[V_W][m];
        const double p = u + beta * v[V_P][m];
        const double sv = wv + beta * v[V_S][m];
        const double x = v[xs][m] + alpha * p;
        const double r = v[V_R][m] - alpha * sv;
        const double un = v[V_PINV][m] * r;
        v[V_P][m] = p;
        v[V_S][m] = sv;
        v[xs][m] = x;
        v[V_R][m] = r;
        v[V_U][m] = un;
        halo_store(parts, s, P, xs, m, x);
        halo_store(parts, s, P, V_U, m, un);
      }
    } else {
      const double* __restrict__ d = v[V_D0 + c.id];
      for (int m = m0 + (int)threadIdx.x; m < m1; m += kThreads) {
        const double x = v[xs][m] + alpha * d[m];
        const double r = v[V_R][m] - alpha * v[V_W][m];
        const double un = v[V_PINV][m] * r;
        v[xs][m] = x;
        v[V_R][m] = r;
        v[V_U][m] = un;
        halo_store(parts, s, P, xs, m, x);
        halo_store(parts, s, P, V_U, m, un);
        part[0] += r * un;
      }
    }
    if (!publish<1>(part, red, partials, w, nitems, sc, &s_last)) continue;
    double tot[1] = {0.0};
    if (!c.merged) slab_allreduce<1>(parts, nslabs, partials, true, tot, red);
    if (threadIdx.x == 0) {
      sc->count = 0;
      sc->iter += 1;
      sc->since_true += 1;
      if (!isfinite(tot[0])) {
        fail(sc, heat::ST_NONFINITE);
      } else if (sc->since_true >= sc->resid_period) {
        sc->phase = SP_TRUE;  // periodic true residual (Algorithm 1: i > 0 and i % period == 0)
      } else if (c.merged) {
        sc->phase = SP_ITER;
      } else {
        sc->beta = tot[0] / sc->gamma;
        sc->gamma = tot[0];
        if (tot[0] <= sc->thresh) {
          sc->confirm = 1;  // close only on the true residual
          sc->phase = SP_TRUE;
        } else {
          sc->phase = SP_ITER;
        }
      }
      if (sc->phase != SP_DONE && sc->phase != SP_RHS && sc->phase != SP_FAILED && sc->iter >= sc->max_iter)
        fail(sc, heat::ST_NOT_CONVERGED);
    }
  }
}

// Per owned node of each slab: the Jacobi diagonal's inverse, the Dirichlet
// lift A_{.D} g of free rows and the face-load vector F (q h_a h_b / 4 per
// adjacent face cell, §3.1's flux term on a box face).
struct FaceFluxes {
  double q[6];
};

__global__ void k_slab_setup(const SlabPart* __restrict__ parts, const int2* __restrict__ items, int nitems,
                             FaceFluxes fx) {
  for (int w = blockIdx.x; w < nitems; w += gridDim.x) {
    const int2 it = items[w];
    const SlabPart& P = parts[it.x];
    const SimDev& sd = P.g;
    const int m0 = P.own0 * P.pxy + it.y * kPwChunk;
    const int m1 = min(m0 + kPwChunk, (P.own1 + 1) * P.pxy);
    for (int m = m0 + (int)threadIdx.x; m < m1; m += blockDim.x) {
      const int k = m / P.pxy, rem = m - k * P.pxy;
      const int j = rem / (sd.nx + 1), i = rem - j * (sd.nx + 1);
      const bool dir = heat::is_dirichlet(sd, i, j, k);
      double diag = 0.0;
      for (int cc = 0; cc < 8; ++cc) {
        const int ex = i - (cc & 1), ey = j - ((cc >> 1) & 1), ez = k - ((cc >> 2) & 1);
        if (ex < 0 || ey < 0 || ez < 0 || ex >= sd.nx || ey >= sd.ny || ez >= sd.nz) continue;
        const double2 cf = sd.coef[ex + (long long)sd.nx * (ey + (long long)sd.ny * ez)];
        diag += sd.inv_dt * cf.x * sd.mhat[0] + sd.theta * cf.y * sd.khat[0];
      }
      P.v[V_PINV][m] = dir ? 1.0 : 1.0 / diag;
      double lift = 0.0;
      if (!dir) {
        lift = heat::gather_apply<double>(sd, sd.inv_dt, sd.theta, i, j, k, [&](int a, int b, int cz) -> double {
          return heat::is_dirichlet(sd, a, b, cz) ? heat::dirichlet_value(sd, a, b, cz) : 0.0;
        });
      }
      P.v[V_LIFT][m] = lift;
      // face loads by global position: (c_a h_a / 2)(c_b h_b / 2) per face
      // node, c the node's adjacent cells along each in-face direction
      const int kg = P.kg0 + k;
      auto share = [](int idx, int n, double h) { return (idx == 0 || idx == n) ? 0.5 * h : h; };
      const double sx = share(i, sd.nx, P.h[0]), sy = share(j, sd.ny, P.h[1]), sz = share(kg, P.nzg, P.h[2]);
      double F = 0.0;
      const uint32_t dg = P.dir_global;
      if (i == 0 && !(dg & 1u)) F += fx.q[0] * sy * sz;
      if (i == sd.nx && !(dg & 2u)) F += fx.q[1] * sy * sz;
      if (j == 0 && !(dg & 4u)) F += fx.q[2] * sx * sz;
      if (j == sd.ny && !(dg & 8u)) F += fx.q[3] * sx * sz;
      if (kg == 0 && !(dg & 16u)) F += fx.q[4] * sx * sy;
      if (kg == P.nzg && !(dg & 32u)) F += fx.q[5] * sx * sy;
      P.v[V_F][m] = F;
    }
  }
}

}  // namespace

struct heat_slab {
  int nx = 0, ny = 0, nz = 0;
  double h[3] = {0, 0, 0};
  heat_bc bc{};
  heat_params prm{};
  cudaStream_t stream = nullptr;
  int S = 0, merged = 1;
  std::vector<int> first;        // E_s, s = 0..S (E_S = nz + 1)
  std::vector<SlabPart> parts;   // host copy of the descriptors
  SlabPart* d_parts = nullptr;
  int2* d_items = nullptr;
  int nitems = 0;
  int2* d_pw = nullptr;
  int npw = 0;
  double* d_partials = nullptr;
  SlabScalars* d_sc = nullptr;
  SlabScalars* h_sc = nullptr;   // pinned mirror
  heat::SimScalars* d_chk = nullptr;
  int* d_log = nullptr;
  std::vector<void*> allocs;
  int grid_op = 1, grid_pw = 1;
  long long launches = 0;
  bool coeffs_set = false, state_set = false;
};

namespace {

heat_status slab_alloc(heat_slab* s, void** p, size_t bytes) {
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return heat::set_error(HEAT_ERR_NOMEM, "heat_slab: cudaMalloc of %zu bytes failed: %s", bytes,
                           cudaGetErrorString(e));
  }
  s->allocs.push_back(*p);
  return HEAT_OK;
}

heat_status read_scalars(heat_slab* s) {
  CUDA_TRY(cudaMemcpyAsync(s->h_sc, s->d_sc, sizeof(SlabScalars), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return HEAT_OK;
}

heat_status write_scalars(heat_slab* s) {
  CUDA_TRY(cudaMemcpyAsync(s->d_sc, s->h_sc, sizeof(SlabScalars), cudaMemcpyHostToDevice, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return HEAT_OK;
}

// Dirichlet value of global node (i, j, k) (lowest face id wins), or NaN.
double dirichlet_global(const heat_slab* s, int i, int j, int k) {
  const uint32_t f = s->bc.dirichlet_faces;
  const bool on[6] = {i == 0, i == s->nx, j == 0, j == s->ny, k == 0, k == s->nz};
  for (int a = 0; a < 6; ++a)
    if ((f >> a & 1u) && on[a]) return s->bc.dirichlet_value[a];
  return std::nan("");
}

}  // namespace

extern "C" heat_status heat_slab_plan(int nz, int nslabs, int* first_layer) {
  if (!first_layer || nz < 1 || nslabs < 1 || nslabs > nz + 1 || nslabs > kMaxSlabs)
    return heat::set_error(HEAT_ERR_ARG, "heat_slab_plan: need nz >= 1 and 1 <= nslabs <= min(nz + 1, %d)",
                           kMaxSlabs);
  for (int s = 0; s < nslabs; ++s) first_layer[s] = (int)((long long)s * (nz + 1) / nslabs);
  first_layer[nslabs] = nz + 1;
  return HEAT_OK;
}

extern "C" void heat_destroy_slab(heat_slab* s) {
  if (!s) return;
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (void* p : s->allocs) cudaFree(p);
  if (s->h_sc) cudaFreeHost(s->h_sc);
  cudaGetLastError();
  delete s;
}

extern "C" heat_status heat_slab_create(const heat_mesh* mesh, const heat_bc* bc, const heat_params* prm,
                                        int nslabs, int merged, void* cuda_stream, heat_slab** out) {
  if (!mesh || !bc || !prm || !out) return heat::set_error(HEAT_ERR_ARG, "heat_slab_create: null argument");
  *out = nullptr;
  if (prm->precision != HEAT_FP64)
    return heat::set_error(HEAT_ERR_ARG, "heat_slab_create: the slab-split solve runs in HEAT_FP64 only");
  if (prm->element != HEAT_ELEM_Q1 || prm->cheb_degree >= 2)
    return heat::set_error(HEAT_ERR_ARG, "heat_slab_create: trilinear boxes with the Jacobi preconditioner only");
  if (!(prm->dt > 0.0) || !std::isfinite(prm->dt) || !(prm->theta > 0.0 && prm->theta <= 1.0) ||
      !(prm->rtol > 0.0) || prm->max_iter < 1 || prm->resid_period < 1)
    return heat::set_error(HEAT_ERR_ARG, "heat_slab_create: bad parameters (dt, theta, rtol, max_iter, resid_period)");
  if (merged != 0 && merged != 1) return heat::set_error(HEAT_ERR_ARG, "heat_slab_create: merged must be 0 or 1");
  for (int f = 0; f < 6; ++f)
    if (!std::isfinite(bc->dirichlet_value[f]) || !std::isfinite(bc->flux[f]))
      return heat::set_error(HEAT_ERR_ARG, "heat_slab_create: non-finite boundary value");
  std::vector<int> first(nslabs > 0 ? nslabs + 1 : 1);
  heat_status st = heat_slab_plan(mesh->nz, nslabs, first.data());
  if (st != HEAT_OK) return st;

  heat_slab* s = new heat_slab();
  s->nx = mesh->nx;
  s->ny = mesh->ny;
  s->nz = mesh->nz;
  s->h[0] = mesh->extent[0] / mesh->nx;
  s->h[1] = mesh->extent[1] / mesh->ny;
  s->h[2] = mesh->extent[2] / mesh->nz;
  s->bc = *bc;
  s->bc.dirichlet_faces &= 63u;
  s->prm = *prm;
  s->stream = static_cast<cudaStream_t>(cuda_stream);
  s->S = nslabs;
  s->merged = merged;
  s->first = first;
  auto bail = [&](heat_status e) {
    heat_destroy_slab(s);
    return e;
  };

  const int pxy = (s->nx + 1) * (s->ny + 1);
  const int ntx = (s->nx + 1 + kSX - 2) / (kSX - 1), nty = (s->ny + 1 + kSY - 2) / (kSY - 1);
  double mhat[8], khat[8], lam_m[8], lam_k[8];
  heat::element_classes(s->h[0], s->h[1], s->h[2], mhat, khat);
  heat::walsh_eigenvalues(s->h[0], s->h[1], s->h[2], lam_m, lam_k);
  if (cudaMalloc(&s->d_chk, sizeof(heat::SimScalars)) != cudaSuccess) {
    cudaGetLastError();
    s->d_chk = nullptr;
    return bail(heat::set_error(HEAT_ERR_NOMEM, "heat_slab_create: out of device memory"));
  }
  s->allocs.push_back(s->d_chk);
  if (cudaMemset(s->d_chk, 0, sizeof(heat::SimScalars)) != cudaSuccess)
    return bail(heat::set_error(HEAT_ERR_CUDA, "heat_slab_create: memset failed"));
  std::vector<int2> items, pws;
  for (int k = 0; k < nslabs; ++k) {
    SlabPart P{};
    const bool lo = k > 0, hi = k < nslabs - 1;
    P.kg0 = first[k] - (lo ? 1 : 0);
    const int top = hi ? first[k + 1] : s->nz;
    const int nzl = top - P.kg0;
    P.own0 = lo ? 1 : 0;
    P.own1 = hi ? nzl - 1 : nzl;
    P.lo = lo;
    P.hi = hi;
    P.pxy = pxy;
    P.nzg = s->nz;
    P.flux_steps = bc->flux_steps;
    P.dir_global = s->bc.dirichlet_faces;
    for (int d = 0; d < 3; ++d) P.h[d] = s->h[d];
    const long long nn_l = (long long)pxy * (nzl + 1);
    if (nn_l >= (1LL << 31) - kPwChunk) return bail(heat::set_error(HEAT_ERR_ARG, "heat_slab_create: slab too large"));
    SimDev& g = P.g;
    g.nx = s->nx;
    g.ny = s->ny;
    g.nz = nzl;
    g.nn = nn_l;
    uint32_t dl = s->bc.dirichlet_faces & 15u;
    if (!lo) dl |= s->bc.dirichlet_faces & 16u;
    if (!hi) dl |= s->bc.dirichlet_faces & 32u;
    g.dir_faces = dl;
    g.prec = heat::P_FP64;
    g.elem = heat::E_Q1;
    g.max_iter = prm->max_iter;
    g.resid_period = prm->resid_period;
    for (int f = 0; f < 6; ++f) g.g[f] = s->bc.dirichlet_value[f];
    g.inv_dt = 1.0 / prm->dt;
    g.theta = prm->theta;
    g.rtol = prm->rtol;
    for (int a = 0; a < 8; ++a) {
      g.mhat[a] = mhat[a];
      g.khat[a] = khat[a];
      g.lam_m[a] = lam_m[a];
      g.lam_k[a] = lam_k[a];
    }
    g.sc = s->d_chk;
    void* cbuf = nullptr;
    st = slab_alloc(s, &cbuf, sizeof(double2) * (size_t)s->nx * s->ny * nzl);
    if (st != HEAT_OK) return bail(st);
    g.coef = static_cast<const double2*>(cbuf);
    for (int v = 0; v < NVEC; ++v) {
      void* b = nullptr;
      st = slab_alloc(s, &b, sizeof(double) * (size_t)nn_l);
      if (st != HEAT_OK) return bail(st);
      if (cudaMemset(b, 0, sizeof(double) * (size_t)nn_l) != cudaSuccess)
        return bail(heat::set_error(HEAT_ERR_CUDA, "heat_slab_create: memset failed"));
      P.v[v] = static_cast<double*>(b);
    }
    const int owned = P.own1 - P.own0 + 1;
    P.ntx = ntx;
    P.nty = nty;
    P.ntz = (owned + kTZ - 1) / kTZ;
    P.item0 = (int)items.size();
    P.nitems = ntx * nty * P.ntz;
    for (int t = 0; t < P.nitems; ++t) items.push_back(make_int2(k, t));
    P.pw0 = (int)pws.size();
    P.npw = (int)(((long long)owned * pxy + kPwChunk - 1) / kPwChunk);
    for (int t = 0; t < P.npw; ++t) pws.push_back(make_int2(k, t));
    s->parts.push_back(P);
  }
  s->nitems = (int)items.size();
  s->npw = (int)pws.size();
  void* b = nullptr;
  if ((st = slab_alloc(s, &b, sizeof(SlabPart) * nslabs)) != HEAT_OK) return bail(st);
  s->d_parts = static_cast<SlabPart*>(b);
  if ((st = slab_alloc(s, &b, sizeof(int2) * s->nitems)) != HEAT_OK) return bail(st);
  s->d_items = static_cast<int2*>(b);
  if ((st = slab_alloc(s, &b, sizeof(int2) * s->npw)) != HEAT_OK) return bail(st);
  s->d_pw = static_cast<int2*>(b);
  if ((st = slab_alloc(s, &b, sizeof(double) * 2 * (size_t)std::max(s->nitems, s->npw))) != HEAT_OK) return bail(st);
  s->d_partials = static_cast<double*>(b);
  if ((st = slab_alloc(s, &b, sizeof(SlabScalars))) != HEAT_OK) return bail(st);
  s->d_sc = static_cast<SlabScalars*>(b);
  if ((st = slab_alloc(s, &b, sizeof(int) * kLogCap)) != HEAT_OK) return bail(st);
  s->d_log = static_cast<int*>(b);
  if (cudaMallocHost(&s->h_sc, sizeof(SlabScalars)) != cudaSuccess) {
    cudaGetLastError();
    s->h_sc = nullptr;
    return bail(heat::set_error(HEAT_ERR_NOMEM, "heat_slab_create: pinned host memory"));
  }
  std::memset(s->h_sc, 0, sizeof(SlabScalars));
  if (cudaMemcpy(s->d_parts, s->parts.data(), sizeof(SlabPart) * nslabs, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->d_items, items.data(), sizeof(int2) * s->nitems, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->d_pw, pws.data(), sizeof(int2) * s->npw, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return bail(heat::set_error(HEAT_ERR_CUDA, "heat_slab_create: descriptor upload failed"));
  }
  int dev = 0, sms = 1, bop = 1, bpw = 1;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bop, k_slab_op, kThreads, 0) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bpw, k_slab_pw, kThreads, 0) != cudaSuccess) {
    cudaGetLastError();
    return bail(heat::set_error(HEAT_ERR_CUDA, "heat_slab_create: device query failed"));
  }
  s->grid_op = std::max(1, std::min(s->nitems, sms * std::max(bop, 1)));
  s->grid_pw = std::max(1, std::min(s->npw, sms * std::max(bpw, 1)));
  *out = s;
  return HEAT_OK;
}

extern "C" heat_status heat_slab_set_coeffs(heat_slab* s, const double* rho_c, const double* k) {
  if (!s || !rho_c || !k) return heat::set_error(HEAT_ERR_ARG, "heat_slab_set_coeffs: null argument");
  const long long plane = (long long)s->nx * s->ny, ne = plane * s->nz;
  for (long long e = 0; e < ne; ++e)
    if (!(rho_c[e] > 0.0) || !(k[e] > 0.0) || !std::isfinite(rho_c[e]) || !std::isfinite(k[e]))
      return heat::set_error(HEAT_ERR_ARG, "heat_slab_set_coeffs: element %lld: need finite rho_c > 0 and k > 0", e);
  std::vector<double> buf;
  for (int q = 0; q < s->S; ++q) {
    const SlabPart& P = s->parts[q];
    const long long n = plane * P.g.nz, e0 = plane * P.kg0;
    buf.resize(2 * n);
    for (long long e = 0; e < n; ++e) {
      buf[2 * e] = rho_c[e0 + e];
      buf[2 * e + 1] = k[e0 + e];
    }
    CUDA_TRY(cudaMemcpyAsync(const_cast<double2*>(P.g.coef), buf.data(), sizeof(double) * 2 * n,
                             cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
  }
  FaceFluxes fx;
  for (int f = 0; f < 6; ++f) fx.q[f] = s->bc.flux[f];
  k_slab_setup<<<s->grid_pw, kThreads, 0, s->stream>>>(s->d_parts, s->d_pw, s->npw, fx);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->launches += 1;
  s->coeffs_set = true;
  return HEAT_OK;
}

extern "C" heat_status heat_slab_set_state(heat_slab* s, const double* u) {
  if (!s || !u) return heat::set_error(HEAT_ERR_ARG, "heat_slab_set_state: null argument");
  const long long pxy = (long long)(s->nx + 1) * (s->ny + 1), nn = pxy * (s->nz + 1);
  std::vector<double> g(u, u + nn);
  for (long long m = 0; m < nn; ++m)
    if (!std::isfinite(g[m])) return heat::set_error(HEAT_ERR_ARG, "heat_slab_set_state: non-finite value at %lld", m);
  if (s->bc.dirichlet_faces) {
    for (int k = 0; k <= s->nz; ++k)
      for (int j = 0; j <= s->ny; ++j)
        for (int i = 0; i <= s->nx; ++i) {
          const double dv = dirichlet_global(s, i, j, k);
          if (!std::isnan(dv)) g[i + (s->nx + 1) * ((long long)j + (s->ny + 1) * (long long)k)] = dv;
        }
  }
  for (int q = 0; q < s->S; ++q) {
    const SlabPart& P = s->parts[q];
    const long long n = pxy * (P.g.nz + 1);
    for (int slot = 0; slot < 3; ++slot)  // every ring slot holds g on the Dirichlet nodes
      CUDA_TRY(cudaMemcpyAsync(P.v[V_X0 + slot], g.data() + pxy * P.kg0, sizeof(double) * n,
                               cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
  }
  std::memset(s->h_sc, 0, sizeof(SlabScalars));
  SlabScalars& c = *s->h_sc;
  c.phase = SP_IDLE;
  c.iu1 = 0;
  c.iu2 = 1;
  c.ix = 2;
  c.merged = s->merged;
  c.resid_period = s->prm.resid_period;
  c.max_iter = s->prm.max_iter;
  c.rtol2 = s->prm.rtol * s->prm.rtol;
  heat_status st = write_scalars(s);
  if (st != HEAT_OK) return st;
  s->state_set = true;
  return HEAT_OK;
}

extern "C" heat_status heat_slab_get_state(heat_slab* s, double* u) {
  if (!s || !u) return heat::set_error(HEAT_ERR_ARG, "heat_slab_get_state: null argument");
  if (!s->state_set) return heat::set_error(HEAT_ERR_ARG, "heat_slab_get_state: no state set");
  heat_status st = read_scalars(s);
  if (st != HEAT_OK) return st;
  const long long pxy = (long long)(s->nx + 1) * (s->ny + 1);
  for (int q = 0; q < s->S; ++q) {
    const SlabPart& P = s->parts[q];
    const long long n = pxy * (P.own1 - P.own0 + 1);
    CUDA_TRY(cudaMemcpyAsync(u + pxy * (P.kg0 + P.own0), P.v[V_X0 + s->h_sc->iu1] + pxy * P.own0,
                             sizeof(double) * n, cudaMemcpyDeviceToHost, s->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return HEAT_OK;
}

extern "C" heat_status heat_slab_step(heat_slab* s, int nsteps, heat_step_stats* stats) {
  if (!s || nsteps < 0) return heat::set_error(HEAT_ERR_ARG, "heat_slab_step: bad argument");
  if (!s->coeffs_set || !s->state_set)
    return heat::set_error(HEAT_ERR_ARG, "heat_slab_step: set coefficients and state first");
  heat_status st = read_scalars(s);
  if (st != HEAT_OK) return st;
  SlabScalars& c = *s->h_sc;
  const long long launches0 = s->launches;
  c.iters_total = 0;
  c.steps_total = 0;
  c.iters_step_max = 0;
  c.log_len = 0;
  c.status = 0;
  c.target = c.step + nsteps;
  c.phase = nsteps > 0 ? SP_RHS : SP_DONE;
  c.count = 0;
  if ((st = write_scalars(s)) != HEAT_OK) return st;
  // Each (operator, pointwise) pair advances the phase machine by at least one
  // operator phase; an iteration takes one pair and each step at most two
  // more plus one true residual per resid_period iterations and per failed
  // confirmation, so this budget is never reached by a running solve.
  const long long budget = (long long)nsteps * (3LL * s->prm.max_iter + 16) + 64;
  const int pairs_per_poll = std::max(1, s->prm.poll_period);
  long long pairs = 0;
  while (c.phase != SP_DONE && c.phase != SP_FAILED) {
    if (pairs >= budget) return heat::set_error(HEAT_ERR_TIMEOUT, "heat_slab_step: phase budget exhausted");
    for (int t = 0; t < pairs_per_poll; ++t) {
      k_slab_op<<<s->grid_op, kThreads, 0, s->stream>>>(s->d_parts, s->S, s->d_items, s->nitems, s->d_partials,
                                                      s->d_sc, s->d_log);
      k_slab_pw<<<s->grid_pw, kThreads, 0, s->stream>>>(s->d_parts, s->S, s->d_pw, s->npw, s->d_partials, s->d_sc,
                                                      s->d_log);
    }
    CUDA_TRY(cudaGetLastError());
    s->launches += 2LL * pairs_per_poll;
    pairs += pairs_per_poll;
    if ((st = read_scalars(s)) != HEAT_OK) return st;
  }
  if (stats) {
    std::memset(stats, 0, sizeof(*stats));
    stats->steps = (int)c.steps_total;
    stats->status = c.phase == SP_FAILED ? c.status : HEAT_OK;
    stats->iters = c.iters_total + (c.phase == SP_FAILED ? c.iter : 0);
    stats->max_iters_step = c.iters_step_max;
    stats->last_rel_residual = c.rel_res;
    stats->kernel_launches = s->launches - launches0;
  }
  if (c.phase == SP_FAILED) {
    const int code = c.status;
    const heat_status hs = code == heat::ST_NOT_CONVERGED ? HEAT_ERR_NOT_CONVERGED
                           : code == heat::ST_NONFINITE   ? HEAT_ERR_NONFINITE
                           : code == heat::ST_BREAKDOWN   ? HEAT_ERR_BREAKDOWN
                                                          : HEAT_ERR_CUDA;
    // the failed step is not committed: the state ring still holds the last good step
    c.phase = SP_IDLE;
    write_scalars(s);
    return heat::set_error(hs, "heat_slab_step: step %d failed (status %d) after %d iterations", c.step + 1, code,
                           c.iter);
  }
  return HEAT_OK;
}

extern "C" heat_status heat_slab_step_iterations(heat_slab* s, int* out, int cap, int* n) {
  if (!s || !n || (cap > 0 && !out)) return heat::set_error(HEAT_ERR_ARG, "heat_slab_step_iterations: bad argument");
  heat_status st = read_scalars(s);
  if (st != HEAT_OK) return st;
  const int len = std::min(s->h_sc->log_len, kLogCap);
  *n = len;
  if (cap > 0 && len > 0) {
    CUDA_TRY(cudaMemcpy(out, s->d_log, sizeof(int) * std::min(cap, len), cudaMemcpyDeviceToHost));
  }
  return HEAT_OK;
}

extern "C" heat_status heat_slab_info(const heat_slab* s, int* nslabs, int* first_layer, long long* device_bytes) {
  if (!s) return heat::set_error(HEAT_ERR_ARG, "heat_slab_info: null slab");
  if (nslabs) *nslabs = s->S;
  if (first_layer)
    for (int q = 0; q <= s->S; ++q) first_layer[q] = s->first[q];
  if (device_bytes) {
    long long b = 0;
    const long long pxy = (long long)(s->nx + 1) * (s->ny + 1);
    for (const SlabPart& P : s->parts)
      b += (long long)NVEC * 8 * pxy * (P.g.nz + 1) + 16LL * s->nx * s->ny * P.g.nz;
    *device_bytes = b;
  }
  return HEAT_OK;
}
