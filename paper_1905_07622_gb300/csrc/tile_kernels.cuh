// Phase-gated tile kernels of the solver.
//
// Operator: y_i = sum_{e containing i} sum_{j in e} (sa*rho_c_e*Mhat[c_i^c_j] +
// sb*k_e*Khat[c_i^c_j]) x_j -- the assembly operator of §3.2 Eq. 1 read degree
// of freedom by degree of freedom (each output node gathers from its <= 8
// elements and 27 neighbours; no atomics, no assembled matrix). Mhat/Khat are
// the Q1 element matrices indexed by the XOR of the two local corner numbers.
//
// Solver: Algorithm 1 (§3.3) split into three phase-gated tile kernels --
//   k_open      step start (right-hand side, x0, r = b - A x0) and, on the
//               FP32 paths, the FP64 refinement sweep (x += e, r = b - A x);
//   k_apply_dot d = P^-1 r + beta d (computed on the fly, so the direction
//               update needs no kernel of its own), q = A d, alpha = delta/(d.q);
//   k_update    x += alpha d, r -= alpha q (or r = b - A x every resid_period
//               iterations), delta = r.P^-1 r, beta, convergence, step close.
// Every reduction is a per-tile partial summed in tile order by the last block
// of the simulation, so results do not depend on what else shares a launch.
#pragma once

#include "op.cuh"

namespace heat {

// ------------------------------------------------------ phase-gated tile kernels

// Per-work-item control block, loaded by thread 0 into shared memory.
struct Ctl {
  int phase, iu1, iu2, ix, ixa, id, restart, have_prev, iter, step;
  double alpha, beta;
};

__device__ __forceinline__ void load_ctl(const SimScalars* sc, Ctl& c) {
  const volatile SimScalars* v = sc;
  c.phase = v->phase;
  c.iu1 = v->iu1;
  c.iu2 = v->iu2;
  c.ix = v->ix;
  c.ixa = v->ixa;
  c.id = v->id;
  c.restart = v->restart;
  c.have_prev = v->have_prev;
  c.iter = v->iter;
  c.step = v->step;
  c.alpha = v->alpha;
  c.beta = v->beta;
}

// Copy the work item's descriptor into shared memory (all threads), and the
// control scalars (thread 0). Ends with a barrier.
__device__ __forceinline__ void load_item(const SimDev* sims, int sim, SimDev& sh, Ctl& ctl) {
  const int* src = reinterpret_cast<const int*>(&sims[sim]);
  int* dst = reinterpret_cast<int*>(&sh);
  for (int t = threadIdx.x; t < (int)(sizeof(SimDev) / sizeof(int)); t += blockDim.x) dst[t] = src[t];
  __syncthreads();
  if (threadIdx.x == 0) load_ctl(sh.sc, ctl);
  __syncthreads();
}

__device__ __forceinline__ void tile_origin(const SimDev& s, int t, int TX, int TY, int TZ, int& i0,
                                            int& j0, int& k0) {
  const int tx = t % s.ntx;
  const int r = t / s.ntx;
  const int ty = r % s.nty;
  const int tz = r / s.nty;
  i0 = tx * TX;
  j0 = ty * TY;
  k0 = tz * TZ;
}

// Step close, run by thread 0 of the last block: log, rotate the state ring
// (U^{n-2} <- U^{n-1} <- x; the old U^{n-2} slot becomes the next x).
__device__ __forceinline__ void close_step(const SimDev& s, SimScalars* sc, double delta_final) {
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

// k_open: PH_OPEN (all precisions) and PH_OUTER (FP32 paths).
template <int P, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX* TY) k_open(const SimDev* __restrict__ sims, const int2* __restrict__ work,
                                                 const int* __restrict__ nwork_p) {
  __shared__ SimDev s;
  __shared__ Ctl ctl;
  __shared__ double red[3 * 32];
  __shared__ int s_last;
  const int nwork = *nwork_p;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 wi = work[w];
    load_item(sims, wi.x, s, ctl);
    const int phase = ctl.phase;
    if (phase != PH_OPEN && !(P != P_FP64 && phase == PH_OUTER)) {
      __syncthreads();
      continue;
    }
    int i0, j0, k0;
    tile_origin(s, wi.y, TX, TY, TZ, i0, j0, k0);
    const int i = i0 + (int)(threadIdx.x % TX), j = j0 + (int)(threadIdx.x / TX);
    double part[3] = {0.0, 0.0, 0.0};  // r.P^-1 r (FP64), b.P^-1 b, inner r32.P^-1 r32
    const double* u1 = s.vec64[ctl.iu1];
    const double* u2 = s.vec64[ctl.iu2];
    double* x = s.vec64[ctl.ix];
    double* xa = s.vec64[ctl.ixa];
    const bool hp = ctl.have_prev != 0;
    const bool flux_on = s.flux_steps < 0 || ctl.step + 1 <= s.flux_steps;
    if (i <= s.nx && j <= s.ny) {
      for (int kz = 0; kz < TZ; ++kz) {
        const int k = k0 + kz;
        if (k > s.nz) break;
        const long long n = node_index(s, i, j, k);
        const bool dir = is_dirichlet(s, i, j, k);
        double rn = 0.0, bn;
        if (phase == PH_OPEN) {
          auto x0 = [&](int a, int b, int c) -> double {
            if (is_dirichlet(s, a, b, c)) return 0.0;
            const long long m = node_index(s, a, b, c);
            return hp ? 2.0 * u1[m] - u2[m] : u1[m];
          };
          if (dir) {
            bn = dirichlet_value(s, i, j, k);
            x[n] = bn;
          } else {
            const double lu = gather_apply<double>(
                s, s.inv_dt, s.theta - 1.0, i, j, k,
                [&](int a, int b, int c) -> double { return u1[node_index(s, a, b, c)]; });
            bn = lu + (flux_on ? s.F[n] : 0.0) - s.zlift[n];
            rn = bn - gather_apply<double>(s, s.inv_dt, s.theta, i, j, k, x0);
            x[n] = x0(i, j, k);
          }
          s.b[n] = bn;
          if (!dir) part[1] += bn * bn * s.pinv[n];
        } else {  // PH_OUTER: x <- x + e, r = b - A x
          auto xe = [&](int a, int b, int c) -> double {
            if (is_dirichlet(s, a, b, c)) return 0.0;
            const long long m = node_index(s, a, b, c);
            return x[m] + (double)s.e32[m];
          };
          if (dir) {
            xa[n] = dirichlet_value(s, i, j, k);
          } else {
            rn = s.b[n] - gather_apply<double>(s, s.inv_dt, s.theta, i, j, k, xe);
            xa[n] = xe(i, j, k);
          }
        }
        if (P == P_FP64) {
          s.r[n] = rn;
        } else {
          const float r32 = (float)rn;
          s.r32[n] = r32;
          part[2] += (double)r32 * (double)r32 * (double)s.pinv32[n];
        }
        part[0] += rn * rn * s.pinv[n];
      }
    }
    block_sum<3>(part, red);
    bool last = false;
    if (threadIdx.x == 0) {
      s.partial[4 * wi.y + 0] = part[0];
      s.partial[4 * wi.y + 1] = part[1];
      s.partial[4 * wi.y + 2] = part[2];
      __threadfence();
      const unsigned int done = atomicAdd(&s.sc->count, 1u);
      last = (done == (unsigned int)(s.ntiles - 1));
      s_last = last;
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      double tot[3] = {0.0, 0.0, 0.0};
      for (int t = threadIdx.x; t < s.ntiles; t += blockDim.x) {
        tot[0] += __ldcg(&s.partial[4 * t + 0]);
        tot[1] += __ldcg(&s.partial[4 * t + 1]);
        tot[2] += __ldcg(&s.partial[4 * t + 2]);
      }
      block_sum<3>(tot, red);
      if (threadIdx.x == 0) {
        SimScalars* sc = s.sc;
        sc->count = 0;
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
        if (!isfinite(tot[0]) || !isfinite(tot[1])) {
          fail(sc, ST_NONFINITE);
        } else if (P == P_FP64) {
          sc->delta = tot[0];
          if (tot[0] <= sc->thresh) close_step(s, sc, tot[0]);
          else sc->phase = PH_ITER;
        } else {
          sc->delta_out = tot[0];
          sc->delta = tot[2];
          const bool plain_done = (P == P_FP32_PLAIN && phase == PH_OUTER);
          if (tot[0] <= sc->thresh || plain_done || tot[2] <= 0.0) {
            close_step(s, sc, tot[0]);
          } else if (sc->outer >= s.max_outer || sc->iter_step >= s.max_iter) {
            fail(sc, ST_NOT_CONVERGED);
          } else {
            sc->thresh_in = (P == P_FP32_PLAIN) ? sc->thresh : s.inner_rtol * s.inner_rtol * tot[2];
            sc->phase = PH_ITER;
          }
        }
      }
    }
    __syncthreads();
  }
}

// T = double: the FP64 path; T = float: the FP32 inner solve.
template <class T> struct IterVecs;
template <> struct IterVecs<double> {
  __device__ static const double* r(const SimDev& s) { return s.r; }
  __device__ static const double* pinv(const SimDev& s) { return s.pinv; }
  __device__ static double* d(const SimDev& s, int id) { return s.d[id]; }
  __device__ static double* q(const SimDev& s) { return s.q; }
};
template <> struct IterVecs<float> {
  __device__ static const float* r(const SimDev& s) { return s.r32; }
  __device__ static const float* pinv(const SimDev& s) { return s.pinv32; }
  __device__ static float* d(const SimDev& s, int id) { return s.d32[id]; }
  __device__ static float* q(const SimDev& s) { return s.q32; }
};

// k_apply_dot: d = P^-1 r + beta d_old (beta = 0 after a restart), q = A' d, d.q.
template <class T, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX* TY) k_apply_dot(const SimDev* __restrict__ sims, const int2* __restrict__ work,
                                                      const int* __restrict__ nwork_p) {
  __shared__ SimDev s;
  __shared__ Ctl ctl;
  __shared__ double red[32];
  __shared__ int s_last;
  const int nwork = *nwork_p;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 wi = work[w];
    load_item(sims, wi.x, s, ctl);
    if (ctl.phase != PH_ITER) {
      __syncthreads();
      continue;
    }
    int i0, j0, k0;
    tile_origin(s, wi.y, TX, TY, TZ, i0, j0, k0);
    const int i = i0 + (int)(threadIdx.x % TX), j = j0 + (int)(threadIdx.x / TX);
    const T* r = IterVecs<T>::r(s);
    const T* pinv = IterVecs<T>::pinv(s);
    const T* dold = IterVecs<T>::d(s, ctl.id);
    T* dnew = IterVecs<T>::d(s, ctl.id ^ 1);
    T* q = IterVecs<T>::q(s);
    const bool rs = ctl.restart != 0;
    const T beta = (T)ctl.beta;
    auto dl = [&](int a, int b, int c) -> T {
      if (is_dirichlet(s, a, b, c)) return T(0);
      const long long m = node_index(s, a, b, c);
      const T sv = pinv[m] * r[m];
      return rs ? sv : sv + beta * dold[m];
    };
    double part[1] = {0.0};
    if (i <= s.nx && j <= s.ny) {
      for (int kz = 0; kz < TZ; ++kz) {
        const int k = k0 + kz;
        if (k > s.nz) break;
        const long long n = node_index(s, i, j, k);
        if (is_dirichlet(s, i, j, k)) {
          dnew[n] = T(0);
          q[n] = T(0);
          continue;
        }
        const T qn = gather_apply<T>(s, (T)s.inv_dt, (T)s.theta, i, j, k, dl);
        const T dn = dl(i, j, k);
        dnew[n] = dn;
        q[n] = qn;
        part[0] += (double)dn * (double)qn;
      }
    }
    block_sum<1>(part, red);
    if (threadIdx.x == 0) {
      s.partial[4 * wi.y] = part[0];
      __threadfence();
      const unsigned int done = atomicAdd(&s.sc->count, 1u);
      s_last = (done == (unsigned int)(s.ntiles - 1));
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      double tot[1] = {0.0};
      for (int t = threadIdx.x; t < s.ntiles; t += blockDim.x) tot[0] += __ldcg(&s.partial[4 * t]);
      block_sum<1>(tot, red);
      if (threadIdx.x == 0) {
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
    __syncthreads();
  }
}

// k_update: x += alpha d, r -= alpha q (r = b - A x on true-residual
// iterations of the FP64 path), delta_new = r.P^-1 r, beta, convergence.
template <class T, int P, int TX, int TY, int TZ>
__global__ void __launch_bounds__(TX* TY) k_update(const SimDev* __restrict__ sims, const int2* __restrict__ work,
                                                   const int* __restrict__ nwork_p) {
  __shared__ SimDev s;
  __shared__ Ctl ctl;
  __shared__ double red[32];
  __shared__ int s_last;
  const int nwork = *nwork_p;
  for (int w = blockIdx.x; w < nwork; w += gridDim.x) {
    const int2 wi = work[w];
    load_item(sims, wi.x, s, ctl);
    if (ctl.phase != PH_ITER) {
      __syncthreads();
      continue;
    }
    const bool resid = (P == P_FP64) && s.resid_period > 0 && ctl.iter > 0 && (ctl.iter % s.resid_period) == 0;
    int i0, j0, k0;
    tile_origin(s, wi.y, TX, TY, TZ, i0, j0, k0);
    const int i = i0 + (int)(threadIdx.x % TX), j = j0 + (int)(threadIdx.x / TX);
    T* r = const_cast<T*>(IterVecs<T>::r(s));
    const T* pinv = IterVecs<T>::pinv(s);
    const T* d = IterVecs<T>::d(s, ctl.id);
    const T* q = IterVecs<T>::q(s);
    const T alpha = (T)ctl.alpha;
    const bool first = ctl.iter == 0;
    double part[1] = {0.0};
    if (i <= s.nx && j <= s.ny) {
      for (int kz = 0; kz < TZ; ++kz) {
        const int k = k0 + kz;
        if (k > s.nz) break;
        const long long n = node_index(s, i, j, k);
        T rn;
        if constexpr (P == P_FP64) {
          double* x = s.vec64[ctl.ix];
          if (!resid) {
            x[n] += alpha * d[n];
            rn = r[n] - alpha * q[n];
          } else {
            double* xa = s.vec64[ctl.ixa];
            if (is_dirichlet(s, i, j, k)) {
              xa[n] = dirichlet_value(s, i, j, k);
              rn = 0.0;
            } else {
              auto xl = [&](int a, int b, int c) -> double {
                if (is_dirichlet(s, a, b, c)) return 0.0;
                const long long m = node_index(s, a, b, c);
                return x[m] + alpha * d[m];
              };
              rn = s.b[n] - gather_apply<double>(s, s.inv_dt, s.theta, i, j, k, xl);
              xa[n] = xl(i, j, k);
            }
          }
        } else {
          s.e32[n] = (first ? 0.0f : s.e32[n]) + alpha * d[n];
          rn = r[n] - alpha * q[n];
        }
        r[n] = rn;
        part[0] += (double)rn * (double)rn * (double)pinv[n];
      }
    }
    block_sum<1>(part, red);
    if (threadIdx.x == 0) {
      s.partial[4 * wi.y] = part[0];
      __threadfence();
      const unsigned int done = atomicAdd(&s.sc->count, 1u);
      s_last = (done == (unsigned int)(s.ntiles - 1));
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      double tot[1] = {0.0};
      for (int t = threadIdx.x; t < s.ntiles; t += blockDim.x) tot[0] += __ldcg(&s.partial[4 * t]);
      block_sum<1>(tot, red);
      if (threadIdx.x == 0) {
        SimScalars* sc = s.sc;
        sc->count = 0;
        const double dn = tot[0];
        sc->beta = dn / sc->delta;
        sc->delta = dn;
        sc->iter += 1;
        sc->iter_step += 1;
        if (resid) {
          const int t2 = sc->ix;
          sc->ix = sc->ixa;
          sc->ixa = t2;
        }
        if (!isfinite(dn)) {
          fail(sc, ST_NONFINITE);
        } else if (P == P_FP64) {
          if (dn <= sc->thresh) close_step(s, sc, dn);
          else if (sc->iter_step >= s.max_iter) fail(sc, ST_NOT_CONVERGED);
        } else {
          const int cap = (P == P_FP32_PLAIN) ? s.max_iter : s.resid_period;
          if (dn <= sc->thresh_in || sc->iter >= cap) sc->phase = PH_OUTER;
          if (sc->iter_step >= s.max_iter) fail(sc, ST_NOT_CONVERGED);
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace heat
