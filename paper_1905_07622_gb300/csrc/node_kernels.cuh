// Per-node kernels: setup (diagonal, flux vector, Dirichlet lift, FP32
// coefficients) and the operator-level entry points (apply, right-hand side).
// One thread per node, grid-stride; included by the C ABI translation unit only.
#pragma once

#include "op.cuh"

namespace heat {

// --------------------------------------------------- per-node (setup) kernels

// Jacobi diagonal (§3.3): P_i = sum_{e contains i} (rho_c_e/dt * Mhat[0] + theta*k_e*Khat[0]),
// P = 1 on Dirichlet rows (six-tetrahedra boxes: the diagonal entry M'_cc,
// K'_cc of the node's local corner c in each box). Writes 1/P in FP64 and FP32.
__global__ void k_setup_diag(const SimDev* __restrict__ sp) {
  const SimDev& s = *sp;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < s.nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_of(s, n, i, j, k);
    double p = 1.0;
    if (!is_dirichlet(s, i, j, k)) {
      double sa = 0.0, sk = 0.0;
      for (int c = 0; c < 8; ++c) {
        const int ex = i - (c & 1), ey = j - ((c >> 1) & 1), ez = k - ((c >> 2) & 1);
        if (ex < 0 || ey < 0 || ez < 0 || ex >= s.nx || ey >= s.ny || ez >= s.nz) continue;
        const double2 cf = s.coef[ex + (long long)s.nx * (ey + (long long)s.ny * ez)];
        if (s.elem == E_P1) {
          sa += cf.x * s.p1w[9 * c];
          sk += cf.y * s.p1w[64 + 9 * c];
        } else {
          sa += cf.x;
          sk += cf.y;
        }
      }
      p = s.elem == E_P1 ? s.inv_dt * sa + s.theta * sk : s.inv_dt * s.mhat[0] * sa + s.theta * s.khat[0] * sk;
    }
    s.pinv[n] = 1.0 / p;
    s.pinv32[n] = (float)(1.0 / p);
  }
}

// Upper bound of the spectrum of D^-1 A for the Chebyshev preconditioner
// (Gershgorin, element by element): a node's absolute row sum is at most the
// sum over its elements of the element rows' absolute sums, and a ratio of
// sums of positive terms is at most the largest ratio of terms, so
//   lam_max <= max_e sum_p |a_e Mhat[p] + b_e Khat[p]| / (a_e Mhat[0] + b_e Khat[0]),
// a_e = rho_c_e / dt, b_e = theta k_e (every corner of a box element has the
// same row, indexed by the corner XOR pattern p). The maximum is taken on the
// bit patterns of the non-negative doubles (ordered like the values) in
// s.cheb[18], which the caller zeroes first; it does not depend on the order.
__global__ void k_cheb_bound(const SimDev* __restrict__ sp) {
  const SimDev& s = *sp;
  const long long ne = (long long)s.nx * s.ny * s.nz;
  double best = 0.0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    const double2 cf = s.coef[e];
    const double a = s.inv_dt * cf.x, b = s.theta * cf.y;
    if (s.elem == E_P1) {  // the rows differ by corner: the maximum runs over them
      for (int c = 0; c < 8; ++c) {
        double row = 0.0;
        for (int d = 0; d < 8; ++d) row += fabs(a * s.p1w[8 * c + d] + b * s.p1w[64 + 8 * c + d]);
        best = fmax(best, row / (a * s.p1w[9 * c] + b * s.p1w[64 + 9 * c]));
      }
      continue;
    }
    double row = 0.0;
    for (int p = 0; p < 8; ++p) row += fabs(a * s.mhat[p] + b * s.khat[p]);
    best = fmax(best, row / (a * s.mhat[0] + b * s.khat[0]));
  }
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_down_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0)
    atomicMax(reinterpret_cast<unsigned long long*>(&s.cheb[18]), (unsigned long long)__double_as_longlong(best));
}

// Coefficients of the Chebyshev passes (see k_cheb) for degree m and the
// interval [lam_hi / ratio, lam_hi]. One thread.
__global__ void k_cheb_coef(const SimDev* __restrict__ sp, int m, double ratio) {
  const SimDev& s = *sp;
  double* c = s.cheb;
  const double hi = __longlong_as_double((long long)*reinterpret_cast<const unsigned long long*>(&c[18]));
  const double lo = hi / ratio;
  const double th = 0.5 * (hi + lo), de = 0.5 * (hi - lo), sigma = th / de;
  double rho = 1.0 / sigma;
  c[0] = 1.0 / th;
  for (int k = 1; k < m; ++k) {
    const double rn = 1.0 / (2.0 * sigma - rho);
    c[2 * k - 1] = rn * rho;
    c[2 * k] = 2.0 * rn / de;
    rho = rn;
  }
  c[16] = lo;
  c[17] = hi;
}

// Per-element flux densities of the faces that have them (NULL: the face's
// uniform value applies).
struct FaceFlux {
  const double* q[6];
};

// Sum of q over the 1, 2 or 4 element faces of a face grid (na x nb element
// faces, index a + na*b) around node (a, b), in a fixed order.
__device__ __forceinline__ double face_sum(const double* q, int na, int nb, int a, int b) {
  double f = 0.0;
  for (int db = -1; db <= 0; ++db)
    for (int da = -1; da <= 0; ++da) {
      const int ea = a + da, eb = b + db;
      if (ea >= 0 && ea < na && eb >= 0 && eb < nb) f += q[ea + na * eb];
    }
  return f;
}

// The six-tetrahedra split cuts each boundary quad along its diagonal from
// the lower to the upper corner (in the face's own coordinates a < b), into
// two triangles of area A/2, each giving its vertices q A/6: a node receives
// q A/3 from the quads whose diagonal it ends (lower-left, upper-right) and
// q A/6 from the two others. Returns the sum of q times those shares / A.
__device__ __forceinline__ double face_sum_p1(const double* q, double qu, int na, int nb, int a, int b) {
  double f = 0.0;
  for (int db = -1; db <= 0; ++db)
    for (int da = -1; da <= 0; ++da) {
      const int ea = a + da, eb = b + db;
      if (ea >= 0 && ea < na && eb >= 0 && eb < nb) f += (q ? q[ea + na * eb] : qu) * (da == db ? 1.0 / 3.0 : 1.0 / 6.0);
    }
  return f;
}

// Face flux vector F_i = int_face q phi_i ds: on a face of h_a*h_b quads each
// node gets q*h_a*h_b/4 per adjacent quad (1, 2 or 4 of them), with q the
// face's uniform value or the quad's own (six-tetrahedra boxes: face_sum_p1).
__global__ void k_setup_flux(const SimDev* __restrict__ sp, const double* __restrict__ q6, FaceFlux ff,
                             double hx, double hy, double hz) {
  const SimDev& s = *sp;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < s.nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_of(s, n, i, j, k);
    const int ni = (i > 0 && i < s.nx) ? 2 : 1;
    const int nj = (j > 0 && j < s.ny) ? 2 : 1;
    const int nk = (k > 0 && k < s.nz) ? 2 : 1;
    if (s.elem == E_P1) {
      double f = 0.0;
      if (i == 0) f += face_sum_p1(ff.q[0], q6[0], s.ny, s.nz, j, k) * hy * hz;
      if (i == s.nx) f += face_sum_p1(ff.q[1], q6[1], s.ny, s.nz, j, k) * hy * hz;
      if (j == 0) f += face_sum_p1(ff.q[2], q6[2], s.nx, s.nz, i, k) * hx * hz;
      if (j == s.ny) f += face_sum_p1(ff.q[3], q6[3], s.nx, s.nz, i, k) * hx * hz;
      if (k == 0) f += face_sum_p1(ff.q[4], q6[4], s.nx, s.ny, i, j) * hx * hy;
      if (k == s.nz) f += face_sum_p1(ff.q[5], q6[5], s.nx, s.ny, i, j) * hx * hy;
      s.F[n] = is_dirichlet(s, i, j, k) ? 0.0 : f;
      continue;
    }
    const double ax = hy * hz * 0.25, ay = hx * hz * 0.25, az = hx * hy * 0.25;
    double f = 0.0;
    if (i == 0) f += ff.q[0] ? face_sum(ff.q[0], s.ny, s.nz, j, k) * ax : q6[0] * ax * nj * nk;
    if (i == s.nx) f += ff.q[1] ? face_sum(ff.q[1], s.ny, s.nz, j, k) * ax : q6[1] * ax * nj * nk;
    if (j == 0) f += ff.q[2] ? face_sum(ff.q[2], s.nx, s.nz, i, k) * ay : q6[2] * ay * ni * nk;
    if (j == s.ny) f += ff.q[3] ? face_sum(ff.q[3], s.nx, s.nz, i, k) * ay : q6[3] * ay * ni * nk;
    if (k == 0) f += ff.q[4] ? face_sum(ff.q[4], s.nx, s.ny, i, j) * az : q6[4] * az * ni * nj;
    if (k == s.nz) f += ff.q[5] ? face_sum(ff.q[5], s.nx, s.ny, i, j) * az : q6[5] * az * ni * nj;
    s.F[n] = is_dirichlet(s, i, j, k) ? 0.0 : f;
  }
}

// Dirichlet lift z = A_{.D} g on free rows (0 on Dirichlet rows).
__global__ void k_setup_lift(const SimDev* __restrict__ sp) {
  const SimDev& s = *sp;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < s.nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_of(s, n, i, j, k);
    double z = 0.0;
    if (s.dir_faces && !is_dirichlet(s, i, j, k)) {
      z = gather_apply<double>(s, s.inv_dt, s.theta, i, j, k, [&](int a, int b, int c) -> double {
        return is_dirichlet(s, a, b, c) ? dirichlet_value(s, a, b, c) : 0.0;
      });
    }
    s.zlift[n] = z;
  }
}

// FP32 copy of the coefficients; counts non-finite or non-positive entries.
// On trilinear boxes also the A operator's per-element Walsh-pair
// coefficients (SimDev::acoef): A_q = rc/dt (lm_q + lm_{q+4}) + theta k
// (lk_q + lk_{q+4}), B_q the same with differences, computed in FP64 and
// stored as FP64 (FP64 path) or as (hi, lo) float pairs (FP32 paths).
__global__ void k_setup_coef32(const SimDev* __restrict__ sp, long long ne, unsigned int* bad) {
  const SimDev& s = *sp;
  unsigned int nbad = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    const double2 c = s.coef[e];
    if (!(isfinite(c.x) && isfinite(c.y) && c.x > 0.0 && c.y > 0.0)) ++nbad;
    reinterpret_cast<float2*>(const_cast<float2*>(s.coef32))[e] = make_float2((float)c.x, (float)c.y);
    if (s.acoef && s.elem == E_Q1) {
      const double a = s.inv_dt * c.x, b = s.theta * c.y;
      double A[4], B[4];
      for (int q = 0; q < 4; ++q) {
        A[q] = a * (s.lam_m[q] + s.lam_m[q + 4]) + b * (s.lam_k[q] + s.lam_k[q + 4]);
        B[q] = a * (s.lam_m[q] - s.lam_m[q + 4]) + b * (s.lam_k[q] - s.lam_k[q + 4]);
      }
      float4* out = const_cast<float4*>(s.acoef) + 4 * e;
      if (s.prec == P_FP64) {
        double2* o = reinterpret_cast<double2*>(out);
        o[0] = make_double2(A[0], A[1]);
        o[1] = make_double2(A[2], A[3]);
        o[2] = make_double2(B[0], B[1]);
        o[3] = make_double2(B[2], B[3]);
      } else {
        float h[8], l[8];
        for (int q = 0; q < 4; ++q) {
          h[q] = (float)A[q];
          l[q] = (float)(A[q] - (double)h[q]);
          h[q + 4] = (float)B[q];
          l[q + 4] = (float)(B[q] - (double)h[q + 4]);
        }
        for (int w = 0; w < 4; ++w) out[w] = make_float4(h[2 * w], l[2 * w], h[2 * w + 1], l[2 * w + 1]);
      }
    }
  }
  if (nbad) atomicAdd(bad, nbad);
}

// Counts entries of (rho_c, k) that are non-finite or not > 0.
__global__ void k_check_coef_pair(const double* __restrict__ rc, const double* __restrict__ kk, long long ne,
                                  unsigned int* bad) {
  unsigned int nbad = 0;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne; e += (long long)gridDim.x * blockDim.x)
    if (!(isfinite(rc[e]) && isfinite(kk[e]) && rc[e] > 0.0 && kk[e] > 0.0)) ++nbad;
  if (nbad) atomicAdd(bad, nbad);
}

__global__ void k_reciprocal(const double* __restrict__ a, double* __restrict__ out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = 1.0 / a[i];
}

// y = (sa M + sb K) x; with MASK, Dirichlet rows give y = x and Dirichlet
// columns are dropped (the eliminated operator padded with the identity).
template <class T, bool MASK>
__global__ void k_apply_nodes(const SimDev* __restrict__ sp, T sa, T sb, const T* __restrict__ x,
                              T* __restrict__ y) {
  const SimDev& s = *sp;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < s.nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_of(s, n, i, j, k);
    if (MASK && is_dirichlet(s, i, j, k)) {
      y[n] = x[n];
      continue;
    }
    y[n] = gather_apply<T>(s, sa, sb, i, j, k, [&](int a, int b, int c) -> T {
      if (MASK && is_dirichlet(s, a, b, c)) return T(0);
      return x[node_index(s, a, b, c)];
    });
  }
}

// Right-hand side of step n from u_prev: b = L u_prev + F^n - z (free rows), g (Dirichlet).
__global__ void k_rhs_nodes(const SimDev* __restrict__ sp, int n_step, const double* __restrict__ u,
                            double* __restrict__ b) {
  const SimDev& s = *sp;
  const bool flux_on = s.flux_steps < 0 || n_step <= s.flux_steps;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < s.nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_of(s, n, i, j, k);
    if (is_dirichlet(s, i, j, k)) {
      b[n] = dirichlet_value(s, i, j, k);
      continue;
    }
    const double lu = gather_apply<double>(s, s.inv_dt, s.theta - 1.0, i, j, k,
                                           [&](int a, int bb, int c) -> double { return u[node_index(s, a, bb, c)]; });
    b[n] = lu + (flux_on ? s.F[n] : 0.0) - s.zlift[n];
  }
}

// Overwrite Dirichlet nodes of u with their values.
__global__ void k_impose_dirichlet(const SimDev* __restrict__ sp, double* __restrict__ u) {
  const SimDev& s = *sp;
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < s.nn;
       n += (long long)gridDim.x * blockDim.x) {
    int i, j, k;
    node_of(s, n, i, j, k);
    if (is_dirichlet(s, i, j, k)) u[n] = dirichlet_value(s, i, j, k);
  }
}

}  // namespace heat
