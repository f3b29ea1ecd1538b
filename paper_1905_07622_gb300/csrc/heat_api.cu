// C ABI of the solver (declared in include/heat.h): meshes, simulations,
// the tick engine that drives the phase-gated kernels, and operator entry points.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "heat.h"
#include "engine.h"
#include "node_kernels.cuh"

using namespace heat;

// ------------------------------------------------------------------ errors

static thread_local std::string g_err;

heat_status heat::set_error(heat_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

extern "C" const char* heat_last_error(void) { return g_err.c_str(); }

extern "C" const char* heat_status_string(heat_status s) {
  switch (s) {
    case HEAT_OK: return "ok";
    case HEAT_ERR_ARG: return "invalid argument";
    case HEAT_ERR_NOMEM: return "out of memory";
    case HEAT_ERR_CUDA: return "CUDA error";
    case HEAT_ERR_NOT_CONVERGED: return "not converged";
    case HEAT_ERR_NONFINITE: return "non-finite value";
    case HEAT_ERR_TIMEOUT: return "timeout";
    case HEAT_ERR_BUSY: return "busy";
    case HEAT_ERR_BREAKDOWN: return "CG breakdown";
  }
  return "unknown status";
}

// ------------------------------------------------------------------ mesh

extern "C" void heat_params_default(heat_params* p) {
  if (!p) return;
  p->theta = 0.5;
  p->dt = 1e-3;
  p->rtol = 1e-10;
  p->max_iter = 20000;
  p->resid_period = 50;
  p->poll_period = 32;
  p->precision = HEAT_FP64;
  p->inner_rtol = 1e-5;
  p->max_outer = 40;
  p->inner_max_iter = 2000;
  p->cheb_degree = 0;
  p->cheb_ratio = 10.0;
  p->element = HEAT_ELEM_Q1;
}

extern "C" heat_status heat_create_mesh(int nx, int ny, int nz, const double origin[3],
                                        const double extent[3], heat_mesh** out) {
  if (!out) return set_error(HEAT_ERR_ARG, "heat_create_mesh: out is NULL");
  *out = nullptr;
  if (nx < 1 || ny < 1 || nz < 1)
    return set_error(HEAT_ERR_ARG, "heat_create_mesh: nx, ny, nz must be >= 1 (got %d %d %d)", nx, ny, nz);
  const long long nn = ((long long)nx + 1) * ((long long)ny + 1) * ((long long)nz + 1);
  // node and element indices are 32-bit in the kernels
  if (nn >= (1LL << 31) - 1)
    return set_error(HEAT_ERR_ARG, "heat_create_mesh: %lld nodes; at most 2^31 - 2 per mesh", nn);
  heat_mesh* m = new heat_mesh();
  m->nx = nx;
  m->ny = ny;
  m->nz = nz;
  for (int d = 0; d < 3; ++d) {
    m->origin[d] = origin ? origin[d] : 0.0;
    m->extent[d] = extent ? extent[d] : 1.0;
    if (!(m->extent[d] > 0.0) || !std::isfinite(m->extent[d]) || !std::isfinite(m->origin[d])) {
      delete m;
      return set_error(HEAT_ERR_ARG, "heat_create_mesh: extent must be finite and > 0");
    }
  }
  *out = m;
  return HEAT_OK;
}

extern "C" void heat_destroy_mesh(heat_mesh* mesh) { delete mesh; }

extern "C" heat_status heat_mesh_sizes(const heat_mesh* m, long long* n_nodes, long long* n_elems) {
  if (!m) return set_error(HEAT_ERR_ARG, "heat_mesh_sizes: mesh is NULL");
  if (n_nodes) *n_nodes = (long long)(m->nx + 1) * (m->ny + 1) * (m->nz + 1);
  if (n_elems) *n_elems = (long long)m->nx * m->ny * m->nz;
  return HEAT_OK;
}

// Closed-form Q1 element matrices of an hx*hy*hz box indexed by the XOR
// pattern p of two corners (bit d set: the corners differ in dimension d):
// tensor products of the 1-D linear-element mass h/6*[2 1;1 2] and stiffness
// 1/h*[1 -1;-1 1] (§3.2: one element matrix pair serves the whole fixed grid).
void heat::element_classes(double hx, double hy, double hz, double mhat[8], double khat[8]) {
  const double h[3] = {hx, hy, hz};
  for (int p = 0; p < 8; ++p) {
    double m[3], kk[3];
    for (int d = 0; d < 3; ++d) {
      const bool diff = (p >> d) & 1;
      m[d] = diff ? h[d] / 6.0 : h[d] / 3.0;
      kk[d] = diff ? -1.0 / h[d] : 1.0 / h[d];
    }
    mhat[p] = m[0] * m[1] * m[2];
    khat[p] = kk[0] * m[1] * m[2] + m[0] * kk[1] * m[2] + m[0] * m[1] * kk[2];
  }
}

// Eigenvalues of the same element matrices in the Walsh basis of the corners
// (w = wx | wy<<1 | wz<<2; w_d = 0: sum, 1: difference): in 1-D the mass
// h/6*[2 1;1 2] has eigenvalues h/2 (sum) and h/6 (difference), the stiffness
// 1/h*[1 -1;-1 1] has 0 and 2/h. Divided by 8, the normalisation of the
// inverse 3-D transform.
void heat::walsh_eigenvalues(double hx, double hy, double hz, double lam_m[8], double lam_k[8]) {
  const double h[3] = {hx, hy, hz};
  for (int w = 0; w < 8; ++w) {
    double m[3], kk[3];
    for (int d = 0; d < 3; ++d) {
      const bool diff = (w >> d) & 1;
      m[d] = diff ? h[d] / 6.0 : h[d] / 2.0;
      kk[d] = diff ? 2.0 / h[d] : 0.0;
    }
    lam_m[w] = m[0] * m[1] * m[2] / 8.0;
    lam_k[w] = (kk[0] * m[1] * m[2] + m[0] * kk[1] * m[2] + m[0] * m[1] * kk[2]) / 8.0;
  }
}

// The six tetrahedra of a box are the monotone corner paths 0 -> e_a ->
// e_a + e_b -> 7 over the orderings (a, b, c) of the axes, each of volume
// V = hx hy hz / 6. On such a tetrahedron the linear interpolant is
//   u = u_0 + (u_1 - u_0) x_a / h_a + (u_2 - u_1) x_b / h_b + (u_3 - u_2) x_c / h_c,
// so the gradients of the four vertex functions are -e_a/h_a,
// e_a/h_a - e_b/h_b, e_b/h_b - e_c/h_c and e_c/h_c; the element matrices are
// K_ij = V g_i . g_j and the P1 mass V (1 + delta_ij) / 20.
void heat::p1_box_matrices(double hx, double hy, double hz, double M[64], double K[64]) {
  const double h[3] = {hx, hy, hz};
  const double vol = hx * hy * hz / 6.0;
  for (int t = 0; t < 64; ++t) M[t] = K[t] = 0.0;
  const int orders[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  for (const auto& o : orders) {
    const int v[4] = {0, 1 << o[0], (1 << o[0]) | (1 << o[1]), 7};
    double g[4][3] = {};
    g[0][o[0]] = -1.0 / h[o[0]];
    g[1][o[0]] = 1.0 / h[o[0]];
    g[1][o[1]] = -1.0 / h[o[1]];
    g[2][o[1]] = 1.0 / h[o[1]];
    g[2][o[2]] = -1.0 / h[o[2]];
    g[3][o[2]] = 1.0 / h[o[2]];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        M[8 * v[a] + v[b]] += vol * (a == b ? 2.0 : 1.0) / 20.0;
        K[8 * v[a] + v[b]] += vol * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
      }
  }
}

// ------------------------------------------------------------------ sim

static int grid_for(long long n, int block) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long g = (n + block - 1) / block;
  g = std::max(1LL, std::min(g, (long long)sms * 16));
  return (int)g;
}

heat_status heat::sim_alloc(heat_sim* s, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_error(HEAT_ERR_NOMEM, "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
  }
  s->allocs.push_back(*p);
  return HEAT_OK;
}

static heat_status check_params(const heat_params* p) {
  if (!p) return set_error(HEAT_ERR_ARG, "params is NULL");
  if (!(p->theta > 0.0 && p->theta <= 1.0)) return set_error(HEAT_ERR_ARG, "theta must be in (0, 1] (got %g)", p->theta);
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return set_error(HEAT_ERR_ARG, "dt must be finite and > 0");
  if (!(p->rtol >= 0.0) || !std::isfinite(p->rtol)) return set_error(HEAT_ERR_ARG, "rtol must be finite and >= 0");
  if (p->max_iter < 1) return set_error(HEAT_ERR_ARG, "max_iter must be >= 1");
  if (p->resid_period < 1) return set_error(HEAT_ERR_ARG, "resid_period must be >= 1");
  if (p->poll_period < 1) return set_error(HEAT_ERR_ARG, "poll_period must be >= 1");
  if (p->precision < HEAT_FP64 || p->precision > HEAT_FP32_PLAIN) return set_error(HEAT_ERR_ARG, "bad precision");
  if (p->precision == HEAT_FP32_REFINED) {
    if (!(p->inner_rtol > 0.0 && p->inner_rtol < 1.0)) return set_error(HEAT_ERR_ARG, "inner_rtol must be in (0, 1)");
    if (p->max_outer < 1) return set_error(HEAT_ERR_ARG, "max_outer must be >= 1");
    if (p->inner_max_iter < 1) return set_error(HEAT_ERR_ARG, "inner_max_iter must be >= 1");
  }
  if (p->cheb_degree < 0 || p->cheb_degree > HEAT_CHEB_MAX_DEGREE)
    return set_error(HEAT_ERR_ARG, "cheb_degree must be in [0, %d] (got %d)", HEAT_CHEB_MAX_DEGREE, p->cheb_degree);
  if (p->element != HEAT_ELEM_Q1 && p->element != HEAT_ELEM_P1)
    return set_error(HEAT_ERR_ARG, "element must be HEAT_ELEM_Q1 or HEAT_ELEM_P1 (got %d)", p->element);
  if (p->cheb_degree >= 2 && !(p->cheb_ratio > 1.0 && std::isfinite(p->cheb_ratio)))
    return set_error(HEAT_ERR_ARG, "cheb_ratio must be finite and > 1 (got %g)", p->cheb_ratio);
  return HEAT_OK;
}

static void fill_params(heat_sim* s) {
  SimDev& d = s->dev;
  d.inv_dt = 1.0 / s->prm.dt;
  d.theta = s->prm.theta;
  d.rtol = s->prm.rtol;
  d.inner_rtol = s->prm.inner_rtol;
  d.max_iter = s->prm.max_iter;
  d.resid_period = s->prm.resid_period;
  d.max_outer = s->prm.max_outer;
  d.inner_max_iter = s->prm.inner_max_iter;
  d.cheb_m = s->prm.cheb_degree >= 2 ? s->prm.cheb_degree : 0;  // degree 1 is Jacobi scaled by a constant
  d.prec = s->prm.precision;
  d.elem = s->prm.element;
}

heat_status heat::sim_upload_desc(heat_sim* s) {
  CUDA_TRY(cudaMemcpyAsync(s->d_dev, &s->dev, sizeof(SimDev), cudaMemcpyHostToDevice, s->stream));
  return HEAT_OK;
}

// Recompute diag, lift and FP32 coefficients after coefficients/params change.
heat_status heat::sim_setup_flux(heat_sim* s) {
  const heat_mesh* m = s->mesh;
  const double hx = m->extent[0] / m->nx, hy = m->extent[1] / m->ny, hz = m->extent[2] / m->nz;
  FaceFlux ff;
  for (int f = 0; f < 6; ++f) ff.q[f] = s->d_qface[f];
  k_setup_flux<<<grid_for(s->nn, 256), 256, 0, s->stream>>>(s->d_dev, s->d_q6, ff, hx, hy, hz);
  CUDA_TRY(cudaGetLastError());
  return HEAT_OK;
}

// Interval and coefficients of the Chebyshev preconditioner (when it is on).
static heat_status sim_setup_cheb(heat_sim* s) {
  if (s->dev.cheb_m < 2) return HEAT_OK;
  CUDA_TRY(cudaMemsetAsync(s->dev.cheb + 18, 0, sizeof(double), s->stream));
  k_cheb_bound<<<grid_for(s->ne, 256), 256, 0, s->stream>>>(s->d_dev);
  k_cheb_coef<<<1, 1, 0, s->stream>>>(s->d_dev, s->dev.cheb_m, s->prm.cheb_ratio);
  CUDA_TRY(cudaGetLastError());
  return HEAT_OK;
}

heat_status heat::sim_derive_async(heat_sim* s) {
  const int g = grid_for(s->nn, 256);
  CUDA_TRY(cudaMemsetAsync(&s->d_sc->y_valid, 0, sizeof(int), s->stream));
  CUDA_TRY(cudaMemsetAsync(s->d_bad, 0, sizeof(unsigned int), s->stream));
  k_setup_coef32<<<grid_for(s->ne, 256), 256, 0, s->stream>>>(s->d_dev, s->ne, s->d_bad);
  k_setup_diag<<<g, 256, 0, s->stream>>>(s->d_dev);
  k_setup_lift<<<g, 256, 0, s->stream>>>(s->d_dev);
  CUDA_TRY(cudaGetLastError());
  return sim_setup_cheb(s);
}

static heat_status sim_refresh(heat_sim* s) {
  heat_status st = sim_upload_desc(s);
  if (st != HEAT_OK) return st;
  const int g = grid_for(s->nn, 256);
  // the operator changes: stored products A' u of past states no longer hold
  CUDA_TRY(cudaMemsetAsync(&s->d_sc->y_valid, 0, sizeof(int), s->stream));
  CUDA_TRY(cudaMemsetAsync(s->d_bad, 0, sizeof(unsigned int), s->stream));
  k_setup_coef32<<<grid_for(s->ne, 256), 256, 0, s->stream>>>(s->d_dev, s->ne, s->d_bad);
  k_setup_diag<<<g, 256, 0, s->stream>>>(s->d_dev);
  k_setup_lift<<<g, 256, 0, s->stream>>>(s->d_dev);
  CUDA_TRY(cudaGetLastError());
  st = sim_setup_cheb(s);
  if (st != HEAT_OK) return st;
  unsigned int bad = 0;
  CUDA_TRY(cudaMemcpyAsync(&bad, s->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (bad) return set_error(HEAT_ERR_NONFINITE, "%u coefficient(s) are non-finite or not > 0", bad);
  return HEAT_OK;
}

heat_status heat::sim_read_scalars(heat_sim* s) {
  CUDA_TRY(cudaMemcpyAsync(s->h_sc, s->d_sc, sizeof(SimScalars), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return HEAT_OK;
}

heat_status heat::sim_write_scalars(heat_sim* s) {
  CUDA_TRY(cudaMemcpyAsync(s->d_sc, s->h_sc, sizeof(SimScalars), cudaMemcpyHostToDevice, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return HEAT_OK;
}

static void reset_scalars(SimScalars* sc) {
  const unsigned int checks = sc->check_violations;  // counted over the sim's life
  std::memset(sc, 0, sizeof(SimScalars));
  sc->check_violations = checks;
  sc->phase = PH_IDLE;
  sc->iu1 = 0;
  sc->iu2 = 1;
  sc->ix = 2;
  sc->ixa = 3;
}

extern "C" heat_status heat_sim_create(const heat_mesh* mesh, const heat_bc* bc, const heat_params* params,
                                       void* cuda_stream, heat_sim** out) {
  if (!out) return set_error(HEAT_ERR_ARG, "heat_sim_create: out is NULL");
  *out = nullptr;
  if (!mesh) return set_error(HEAT_ERR_ARG, "heat_sim_create: mesh is NULL");
  heat_params prm;
  if (params) prm = *params;
  else heat_params_default(&prm);
  heat_status st = check_params(&prm);
  if (st != HEAT_OK) return st;
  heat_bc b{};
  if (bc) b = *bc;
  b.dirichlet_faces &= 63u;
  for (int f = 0; f < 6; ++f)
    if (!std::isfinite(b.dirichlet_value[f]) || !std::isfinite(b.flux[f]))
      return set_error(HEAT_ERR_NONFINITE, "heat_sim_create: non-finite boundary value on face %d", f);

  heat_sim* s = new heat_sim();
  s->mesh = mesh;
  s->bc = b;
  s->prm = prm;
  s->stream = (cudaStream_t)cuda_stream;
  s->nn = (long long)(mesh->nx + 1) * (mesh->ny + 1) * (mesh->nz + 1);
  s->ne = (long long)mesh->nx * mesh->ny * mesh->nz;
  SimDev& d = s->dev;
  std::memset(&d, 0, sizeof(SimDev));
  d.nx = mesh->nx;
  d.ny = mesh->ny;
  d.nz = mesh->nz;
  d.nn = s->nn;
  d.dir_faces = b.dirichlet_faces;
  d.flux_steps = b.flux_steps;
  for (int f = 0; f < 6; ++f) d.g[f] = b.dirichlet_value[f];
  const double hx = mesh->extent[0] / mesh->nx, hy = mesh->extent[1] / mesh->ny, hz = mesh->extent[2] / mesh->nz;
  element_classes(hx, hy, hz, d.mhat, d.khat);
  {
    const double vol = hx * hy * hz / 6.0;
    d.p1c[0] = vol / 20.0;
    d.p1c[1] = vol / (hx * hx);
    d.p1c[2] = vol / (hy * hy);
    d.p1c[3] = vol / (hz * hz);
    for (int t = 0; t < 4; ++t) d.p1c_f[t] = (float)d.p1c[t];
  }
  walsh_eigenvalues(hx, hy, hz, d.lam_m, d.lam_k);
  for (int p = 0; p < 8; ++p) {
    d.mhat_f[p] = (float)d.mhat[p];
    d.khat_f[p] = (float)d.khat[p];
    d.lam_m_f[p] = (float)d.lam_m[p];
    d.lam_k_f[p] = (float)d.lam_k[p];
  }
  fill_params(s);

  const size_t N8 = (size_t)s->nn * 8, N4 = (size_t)s->nn * 4;
  void* p;
#define ALLOC(field, bytes, type)          \
  st = sim_alloc(s, &p, (bytes));          \
  if (st != HEAT_OK) goto fail;            \
  field = (type)p;
  ALLOC(d.coef, (size_t)s->ne * sizeof(double2), const double2*);
  ALLOC(d.coef32, (size_t)s->ne * sizeof(float2), const float2*);
  ALLOC(d.acoef, (size_t)s->ne * 4 * sizeof(float4), const float4*);
  for (int v = 0; v < 4; ++v) { ALLOC(d.vec64[v], N8, double*); }
  for (int v = 0; v < 4; ++v) { ALLOC(d.yv[v], N8, double*); }
  ALLOC(d.b, N8, double*);
  ALLOC(d.r, N8, double*);
  ALLOC(d.q, N8, double*);
  ALLOC(d.d[0], N8, double*);
  ALLOC(d.d[1], N8, double*);
  ALLOC(d.pinv, N8, double*);
  ALLOC(d.zlift, N8, double*);
  ALLOC(d.F, N8, double*);
  ALLOC(d.r32, N4, float*);
  ALLOC(d.q32, N4, float*);
  ALLOC(d.e32, N4, float*);
  ALLOC(d.d32[0], N4, float*);
  ALLOC(d.d32[1], N4, float*);
  ALLOC(d.pinv32, N4, float*);
  ALLOC(d.rc32[1], N4, float*);
  ALLOC(d.wc32[1], N4, float*);
  ALLOC(d.p32, N4, float*);
  ALLOC(d.z32, N4, float*);
  ALLOC(d.cheb, sizeof(double) * 20, double*);
  d.rc32[0] = d.r32;
  d.wc32[0] = d.q32;
  d.sc32[0] = d.d32[0];
  d.sc32[1] = d.d32[1];
  s->iters_log_cap = 4096;
  ALLOC(d.iters_log, sizeof(int) * s->iters_log_cap, int*);
  d.iters_log_len = s->iters_log_cap;
  ALLOC(s->d_dev, sizeof(SimDev), SimDev*);
  ALLOC(s->d_sc, sizeof(SimScalars), SimScalars*);
  ALLOC(s->d_q6, sizeof(double) * 6, double*);
  ALLOC(s->d_bad, sizeof(unsigned int), unsigned int*);
  ALLOC(d.p1w, sizeof(double) * 128, const double*);
  ALLOC(d.p1w_f, sizeof(float) * 128, const float*);
#undef ALLOC
  d.sc = s->d_sc;
  if (cudaMallocHost((void**)&s->h_sc, sizeof(SimScalars)) != cudaSuccess) {
    cudaGetLastError();
    st = set_error(HEAT_ERR_NOMEM, "cudaMallocHost failed");
    goto fail;
  }
  s->h_sc->check_violations = 0;
  reset_scalars(s->h_sc);
  {
    // default state: rho_c = k = 1, U^0 = 0 (Dirichlet nodes at their values)
    std::vector<double2> ones((size_t)s->ne, make_double2(1.0, 1.0));
    double p1w[128];
    float p1w_f[128];
    p1_box_matrices(hx, hy, hz, p1w, p1w + 64);
    for (int t = 0; t < 128; ++t) p1w_f[t] = (float)p1w[t];
    if (cudaMemcpy((void*)d.coef, ones.data(), (size_t)s->ne * sizeof(double2), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemsetAsync(d.vec64[0], 0, N8, s->stream) != cudaSuccess ||
        cudaMemsetAsync(d.vec64[1], 0, N8, s->stream) != cudaSuccess ||
        cudaMemsetAsync(d.vec64[2], 0, N8, s->stream) != cudaSuccess ||
        cudaMemsetAsync(d.d[0], 0, N8, s->stream) != cudaSuccess ||
        cudaMemsetAsync(d.d[1], 0, N8, s->stream) != cudaSuccess ||
        cudaMemsetAsync(d.d32[0], 0, N4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(d.d32[1], 0, N4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(d.e32, 0, N4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(d.p32, 0, N4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(d.rc32[1], 0, N4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(d.wc32[1], 0, N4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(d.z32, 0, N4, s->stream) != cudaSuccess ||
        cudaMemsetAsync(d.cheb, 0, sizeof(double) * 20, s->stream) != cudaSuccess ||
        cudaMemcpy((void*)d.p1w, p1w, sizeof(p1w), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy((void*)d.p1w_f, p1w_f, sizeof(p1w_f), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpyAsync(s->d_q6, b.flux, sizeof(double) * 6, cudaMemcpyHostToDevice, s->stream) != cudaSuccess) {
      st = set_error(HEAT_ERR_CUDA, "heat_sim_create: initialisation failed: %s", cudaGetErrorString(cudaGetLastError()));
      goto fail;
    }
    st = sim_upload_desc(s);
    if (st != HEAT_OK) goto fail;
    st = sim_setup_flux(s);
    if (st != HEAT_OK) goto fail;
    k_impose_dirichlet<<<grid_for(s->nn, 256), 256, 0, s->stream>>>(s->d_dev, d.vec64[0]);
    st = sim_refresh(s);
    if (st != HEAT_OK) goto fail;
    st = sim_write_scalars(s);
    if (st != HEAT_OK) goto fail;
  }
  *out = s;
  return HEAT_OK;
fail:
  heat_destroy_sim(s);
  return st;
}

extern "C" void heat_destroy_sim(heat_sim* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  engine_destroy(s->eng);
  s->eng = nullptr;
  for (void* p : s->allocs) cudaFree(p);
  if (s->h_sc) cudaFreeHost(s->h_sc);
  delete s;
}

static heat_status copy_in(heat_sim* s, void* dst, const void* src, size_t bytes, int on_device) {
  CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
  if (!on_device) CUDA_TRY(cudaStreamSynchronize(s->stream));
  return HEAT_OK;
}

extern "C" heat_status heat_set_coeffs(heat_sim* s, const double* rho_c, const double* k, int on_device) {
  if (!s || !rho_c || !k) return set_error(HEAT_ERR_ARG, "heat_set_coeffs: null argument");
  if (!on_device) {
    for (long long e = 0; e < s->ne; ++e) {
      if (!std::isfinite(rho_c[e]) || !std::isfinite(k[e]))
        return set_error(HEAT_ERR_NONFINITE, "heat_set_coeffs: non-finite coefficient at element %lld", e);
      if (!(rho_c[e] > 0.0) || !(k[e] > 0.0))
        return set_error(HEAT_ERR_ARG, "heat_set_coeffs: coefficients must be > 0 (element %lld)", e);
    }
  }
  // Stage both arrays in the b and q work vectors (Ne < N), check them on the
  // device, and only then interleave them into the live (rho_c, k) array.
  const size_t bytes = (size_t)s->ne * sizeof(double);
  heat_status st = copy_in(s, s->dev.b, rho_c, bytes, on_device);
  if (st != HEAT_OK) return st;
  st = copy_in(s, s->dev.q, k, bytes, on_device);
  if (st != HEAT_OK) return st;
  CUDA_TRY(cudaMemsetAsync(s->d_bad, 0, sizeof(unsigned int), s->stream));
  k_check_coef_pair<<<grid_for(s->ne, 256), 256, 0, s->stream>>>(s->dev.b, s->dev.q, s->ne, s->d_bad);
  CUDA_TRY(cudaGetLastError());
  unsigned int bad = 0;
  CUDA_TRY(cudaMemcpyAsync(&bad, s->d_bad, sizeof(bad), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (bad) return set_error(HEAT_ERR_NONFINITE, "heat_set_coeffs: %u coefficient(s) non-finite or not > 0", bad);
  CUDA_TRY(cudaMemcpy2DAsync((void*)s->dev.coef, sizeof(double2), s->dev.b, sizeof(double), sizeof(double),
                             (size_t)s->ne, cudaMemcpyDeviceToDevice, s->stream));
  CUDA_TRY(cudaMemcpy2DAsync((char*)s->dev.coef + sizeof(double), sizeof(double2), s->dev.q, sizeof(double),
                             sizeof(double), (size_t)s->ne, cudaMemcpyDeviceToDevice, s->stream));
  return sim_refresh(s);
}

extern "C" heat_status heat_get_coeffs(heat_sim* s, double* rho_c, double* k, int on_device) {
  if (!s || !rho_c || !k) return set_error(HEAT_ERR_ARG, "heat_get_coeffs: null argument");
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(cudaMemcpy2DAsync(rho_c, sizeof(double), s->dev.coef, sizeof(double2), sizeof(double), (size_t)s->ne,
                             kind, s->stream));
  CUDA_TRY(cudaMemcpy2DAsync(k, sizeof(double), (const char*)s->dev.coef + sizeof(double), sizeof(double2),
                             sizeof(double), (size_t)s->ne, kind, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return HEAT_OK;
}

extern "C" heat_status heat_set_params(heat_sim* s, const heat_params* params) {
  if (!s) return set_error(HEAT_ERR_ARG, "heat_set_params: sim is NULL");
  heat_status st = check_params(params);
  if (st != HEAT_OK) return st;
  const bool elem_changed = params->element != s->prm.element;
  const bool prec_changed = params->precision != s->prm.precision || elem_changed;
  s->prm = *params;
  fill_params(s);
  if (prec_changed) {
    engine_destroy(s->eng);
    s->eng = nullptr;
  }
  if (elem_changed) {  // the face loads depend on the element
    st = sim_upload_desc(s);
    if (st != HEAT_OK) return st;
    st = sim_setup_flux(s);
    if (st != HEAT_OK) return st;
  }
  st = sim_refresh(s);
  if (st != HEAT_OK) return st;
  if (s->eng) return engine_refresh(s->eng);
  return HEAT_OK;
}

extern "C" heat_status heat_cheb_interval(heat_sim* s, double* lam_lo, double* lam_hi) {
  if (!s || !lam_lo || !lam_hi) return set_error(HEAT_ERR_ARG, "heat_cheb_interval: null argument");
  if (s->dev.cheb_m < 2) return set_error(HEAT_ERR_ARG, "heat_cheb_interval: the Chebyshev preconditioner is off");
  double v[2];
  CUDA_TRY(cudaMemcpyAsync(v, s->dev.cheb + 16, sizeof(v), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  *lam_lo = v[0];
  *lam_hi = v[1];
  return HEAT_OK;
}

extern "C" heat_status heat_set_state(heat_sim* s, const double* u, int on_device) {
  if (!s || !u) return set_error(HEAT_ERR_ARG, "heat_set_state: null argument");
  if (!on_device) {
    for (long long n = 0; n < s->nn; ++n)
      if (!std::isfinite(u[n])) return set_error(HEAT_ERR_NONFINITE, "heat_set_state: non-finite value at node %lld", n);
  }
  heat_status st = sim_read_scalars(s);
  if (st != HEAT_OK) return st;
  reset_scalars(s->h_sc);
  st = copy_in(s, s->dev.vec64[0], u, (size_t)s->nn * 8, on_device);
  if (st != HEAT_OK) return st;
  k_impose_dirichlet<<<grid_for(s->nn, 256), 256, 0, s->stream>>>(s->d_dev, s->dev.vec64[0]);
  CUDA_TRY(cudaGetLastError());
  return sim_write_scalars(s);
}

extern "C" heat_status heat_get_state(heat_sim* s, double* u, int on_device) {
  if (!s || !u) return set_error(HEAT_ERR_ARG, "heat_get_state: null argument");
  heat_status st = sim_read_scalars(s);
  if (st != HEAT_OK) return st;
  const double* src = s->dev.vec64[s->h_sc->iu1];
  CUDA_TRY(cudaMemcpyAsync(u, src, (size_t)s->nn * 8, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                           s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return HEAT_OK;
}

extern "C" heat_status heat_get_history(heat_sim* s, double* u_prev, double* u_prev2, int* step, int* have_prev,
                                        int on_device) {
  if (!s || !u_prev) return set_error(HEAT_ERR_ARG, "heat_get_history: null argument");
  heat_status st = sim_read_scalars(s);
  if (st != HEAT_OK) return st;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  CUDA_TRY(cudaMemcpyAsync(u_prev, s->dev.vec64[s->h_sc->iu1], (size_t)s->nn * 8, kind, s->stream));
  if (u_prev2 && s->h_sc->have_prev)
    CUDA_TRY(cudaMemcpyAsync(u_prev2, s->dev.vec64[s->h_sc->iu2], (size_t)s->nn * 8, kind, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (step) *step = s->h_sc->step;
  if (have_prev) *have_prev = s->h_sc->have_prev;
  return HEAT_OK;
}

extern "C" heat_status heat_set_history(heat_sim* s, const double* u_prev, const double* u_prev2, int step,
                                        int on_device) {
  if (!s || !u_prev || step < 0) return set_error(HEAT_ERR_ARG, "heat_set_history: bad argument");
  if (!on_device) {
    for (long long n = 0; n < s->nn; ++n)
      if (!std::isfinite(u_prev[n]) || (u_prev2 && !std::isfinite(u_prev2[n])))
        return set_error(HEAT_ERR_NONFINITE, "heat_set_history: non-finite value at node %lld", n);
  }
  heat_status st = sim_read_scalars(s);
  if (st != HEAT_OK) return st;
  reset_scalars(s->h_sc);  // slots: U^{n-1} in vec64[0], U^{n-2} in vec64[1]
  st = copy_in(s, s->dev.vec64[0], u_prev, (size_t)s->nn * 8, on_device);
  if (st != HEAT_OK) return st;
  k_impose_dirichlet<<<grid_for(s->nn, 256), 256, 0, s->stream>>>(s->d_dev, s->dev.vec64[0]);
  if (u_prev2) {
    st = copy_in(s, s->dev.vec64[1], u_prev2, (size_t)s->nn * 8, on_device);
    if (st != HEAT_OK) return st;
    k_impose_dirichlet<<<grid_for(s->nn, 256), 256, 0, s->stream>>>(s->d_dev, s->dev.vec64[1]);
  }
  CUDA_TRY(cudaGetLastError());
  s->h_sc->have_prev = u_prev2 ? 1 : 0;
  s->h_sc->step = step;
  if (s->prm.precision != HEAT_FP64) {
    // the next step's x0 product comes from the stored A' U^{n-1}, A' U^{n-2},
    // as in an uninterrupted run (bitwise the same values)
    st = prime_products(s, u_prev2 ? 2 : 1);
    if (st != HEAT_OK) return st;
    s->h_sc->y_valid = u_prev2 ? 3 : 1;
  }
  return sim_write_scalars(s);
}

static heat_status ensure_log(heat_sim* s, int nsteps) {
  if (nsteps <= s->iters_log_cap) return HEAT_OK;
  void* p;
  heat_status st = sim_alloc(s, &p, sizeof(int) * (size_t)nsteps);
  if (st != HEAT_OK) return st;
  s->iters_log_cap = nsteps;
  s->dev.iters_log = (int*)p;
  s->dev.iters_log_len = nsteps;
  st = sim_upload_desc(s);
  if (st != HEAT_OK) return st;
  if (s->eng) return engine_refresh(s->eng);
  return HEAT_OK;
}

heat_status heat::sim_prepare_steps(heat_sim* s, int nsteps) {
  heat_status st = ensure_log(s, nsteps);
  if (st != HEAT_OK) return st;
  st = sim_read_scalars(s);
  if (st != HEAT_OK) return st;
  SimScalars* sc = s->h_sc;
  sc->target = sc->step + nsteps;
  sc->phase = PH_OPEN;
  sc->status = ST_OK;
  sc->count = 0;
  sc->iters_total = 0;
  sc->outer_total = 0;
  sc->steps_total = 0;
  sc->max_iters_step = 0;
  return sim_write_scalars(s);
}

size_t heat::sim_footprint(long long nn, long long ne) {
  // 16 FP64 and 10 FP32 node vectors, FP64 and FP32 coefficient pairs, the
  // A operator's per-element Walsh-pair coefficients (64 bytes), scalars
  return (size_t)nn * (16 * 8 + 10 * 4) + (size_t)ne * (16 + 8 + 64) + sizeof(SimDev) + sizeof(SimScalars) +
         4096 * sizeof(int) + 1024;
}

void heat::sim_stats(const heat_sim* s, heat_step_stats* o) {
  const SimScalars* sc = s->h_sc;
  o->steps = (int)sc->steps_total;
  o->status = sc->phase == PH_FAILED ? sc->status : HEAT_OK;
  o->iters = sc->iters_total;
  o->outer = sc->outer_total;
  o->max_iters_step = sc->max_iters_step;
  o->last_rel_residual = sc->rel_res;
  o->kernel_launches = 0;
}

extern "C" heat_status heat_step(heat_sim* s, int nsteps, heat_step_stats* stats) {
  if (!s) return set_error(HEAT_ERR_ARG, "heat_step: sim is NULL");
  if (nsteps < 0) return set_error(HEAT_ERR_ARG, "heat_step: nsteps must be >= 0");
  if (stats) std::memset(stats, 0, sizeof(*stats));
  if (nsteps == 0) return HEAT_OK;
  heat_status st = ensure_log(s, nsteps);
  if (st != HEAT_OK) return st;
  if (!s->eng) {
    st = engine_create(&s, 1, s->prm.precision, s->stream, &s->eng);
    if (st != HEAT_OK) return st;
  }
  return engine_step_all(s->eng, nsteps, stats ? stats : nullptr, 1);
}

// ------------------------------------------------------------------ batches

struct heat_batch {
  std::vector<heat_sim*> sims;
  heat::Engine* eng = nullptr;
  cudaStream_t stream = nullptr;
};

extern "C" heat_status heat_batch_create(heat_sim* const* sims, int nsims, void* cuda_stream, heat_batch** out) {
  if (!out) return set_error(HEAT_ERR_ARG, "heat_batch_create: out is NULL");
  *out = nullptr;
  if (!sims || nsims < 1) return set_error(HEAT_ERR_ARG, "heat_batch_create: need at least one simulation");
  for (int i = 0; i < nsims; ++i) {
    if (!sims[i]) return set_error(HEAT_ERR_ARG, "heat_batch_create: simulation %d is NULL", i);
    if (sims[i]->prm.precision != sims[0]->prm.precision)
      return set_error(HEAT_ERR_ARG, "heat_batch_create: simulation %d has a different precision", i);
    for (int j = 0; j < i; ++j)
      if (sims[j] == sims[i]) return set_error(HEAT_ERR_ARG, "heat_batch_create: simulation %d repeated", i);
  }
  heat_batch* b = new heat_batch();
  b->sims.assign(sims, sims + nsims);
  b->stream = (cudaStream_t)cuda_stream;
  heat_status st = engine_create(b->sims.data(), nsims, sims[0]->prm.precision, b->stream, &b->eng);
  if (st != HEAT_OK) {
    delete b;
    return st;
  }
  *out = b;
  return HEAT_OK;
}

extern "C" heat_status heat_batch_step(heat_batch* b, int nsteps, heat_step_stats* stats) {
  if (!b) return set_error(HEAT_ERR_ARG, "heat_batch_step: batch is NULL");
  if (nsteps < 0) return set_error(HEAT_ERR_ARG, "heat_batch_step: nsteps must be >= 0");
  if (stats) std::memset(stats, 0, sizeof(heat_step_stats) * b->sims.size());
  if (nsteps == 0) return HEAT_OK;
  for (heat_sim* s : b->sims) {
    if (s->prm.precision != b->sims[0]->prm.precision)
      return set_error(HEAT_ERR_ARG, "heat_batch_step: a member's precision changed");
    heat_status st = ensure_log(s, nsteps);
    if (st != HEAT_OK) return st;
  }
  // members' parameters or logs may have changed since the last call
  heat_status st = engine_refresh(b->eng);
  if (st != HEAT_OK) return st;
  return engine_step_all(b->eng, nsteps, stats, 1);
}

extern "C" heat_status heat_batch_profile_iteration(heat_batch* b, int reps, void* flush, size_t flush_bytes,
                                                    double* ms_apply, double* ms_update, double* bytes_apply,
                                                    double* bytes_update) {
  if (!b || reps < 1 || !ms_apply || !ms_update || !bytes_apply || !bytes_update)
    return set_error(HEAT_ERR_ARG, "heat_batch_profile_iteration: bad argument");
  return engine_profile(b->eng, reps, flush, flush_bytes, ms_apply, ms_update, bytes_apply, bytes_update);
}

extern "C" void heat_destroy_batch(heat_batch* b) {
  if (!b) return;
  engine_destroy(b->eng);
  delete b;
}

extern "C" heat_status heat_solve_transient(heat_sim* s, int nsteps, double* u_out, heat_step_stats* stats) {
  heat_status st = heat_step(s, nsteps, stats);
  if (st != HEAT_OK) return st;
  if (u_out) return heat_get_state(s, u_out, 0);
  return HEAT_OK;
}

extern "C" heat_status heat_step_iterations(heat_sim* s, int step, int* iters) {
  if (!s || step < 0) return set_error(HEAT_ERR_ARG, "heat_step_iterations: bad argument");
  heat_status st = sim_read_scalars(s);
  if (st != HEAT_OK) return st;
  const int nlog = (int)s->h_sc->steps_total;
  if (step >= nlog || step >= s->iters_log_cap)
    return set_error(HEAT_ERR_ARG, "heat_step_iterations: step %d not logged (%d steps)", step, nlog);
  if (iters) {
    const int idx = (s->h_sc->step - nlog + step) % s->iters_log_cap;
    CUDA_TRY(cudaMemcpy(iters, s->dev.iters_log + idx, sizeof(int), cudaMemcpyDeviceToHost));
  }
  return HEAT_OK;
}

// ------------------------------------------------------ operator entry points

extern "C" heat_status heat_apply(heat_sim* s, const double* x, double* y) {
  if (!s || !x || !y) return set_error(HEAT_ERR_ARG, "heat_apply: null argument");
  k_apply_nodes<double, true><<<grid_for(s->nn, 128), 128, 0, s->stream>>>(s->d_dev, s->dev.inv_dt, s->dev.theta, x, y);
  CUDA_TRY(cudaGetLastError());
  return HEAT_OK;
}

extern "C" heat_status heat_apply_f32(heat_sim* s, const float* x, float* y) {
  if (!s || !x || !y) return set_error(HEAT_ERR_ARG, "heat_apply_f32: null argument");
  k_apply_nodes<float, true><<<grid_for(s->nn, 128), 128, 0, s->stream>>>(s->d_dev, (float)s->dev.inv_dt,
                                                                          (float)s->dev.theta, x, y);
  CUDA_TRY(cudaGetLastError());
  return HEAT_OK;
}

extern "C" heat_status heat_apply_general(heat_sim* s, double sa, double sb, const double* x, double* y) {
  if (!s || !x || !y) return set_error(HEAT_ERR_ARG, "heat_apply_general: null argument");
  if (!std::isfinite(sa) || !std::isfinite(sb)) return set_error(HEAT_ERR_NONFINITE, "heat_apply_general: scale");
  k_apply_nodes<double, false><<<grid_for(s->nn, 128), 128, 0, s->stream>>>(s->d_dev, sa, sb, x, y);
  CUDA_TRY(cudaGetLastError());
  return HEAT_OK;
}

extern "C" heat_status heat_diagonal(heat_sim* s, double* p) {
  if (!s || !p) return set_error(HEAT_ERR_ARG, "heat_diagonal: null argument");
  k_reciprocal<<<grid_for(s->nn, 256), 256, 0, s->stream>>>(s->dev.pinv, p, s->nn);
  CUDA_TRY(cudaGetLastError());
  return HEAT_OK;
}

extern "C" heat_status heat_rhs(heat_sim* s, int n, const double* u_prev, double* b) {
  if (!s || !u_prev || !b || n < 1) return set_error(HEAT_ERR_ARG, "heat_rhs: bad argument");
  k_rhs_nodes<<<grid_for(s->nn, 128), 128, 0, s->stream>>>(s->d_dev, n, u_prev, b);
  CUDA_TRY(cudaGetLastError());
  return HEAT_OK;
}

extern "C" heat_status heat_flux_vector(heat_sim* s, double* f) {
  if (!s || !f) return set_error(HEAT_ERR_ARG, "heat_flux_vector: null argument");
  CUDA_TRY(cudaMemcpyAsync(f, s->dev.F, (size_t)s->nn * 8, cudaMemcpyDeviceToDevice, s->stream));
  return HEAT_OK;
}

// ------------------------------------------------------------ measurement

extern "C" heat_status heat_profile_iteration(heat_sim* s, int reps, void* flush, size_t flush_bytes,
                                              double* ms_apply, double* ms_update, double* bytes_apply,
                                              double* bytes_update) {
  if (!s || reps < 1 || !ms_apply || !ms_update || !bytes_apply || !bytes_update)
    return set_error(HEAT_ERR_ARG, "heat_profile_iteration: bad argument");
  if (!s->eng) return set_error(HEAT_ERR_ARG, "heat_profile_iteration: call heat_step first");
  return engine_profile(s->eng, reps, flush, flush_bytes, ms_apply, ms_update, bytes_apply, bytes_update);
}

// ------------------------------------------------------------ kernel tuning

extern "C" int heat_tuning_num_variants(void) { return num_variants(); }

extern "C" heat_status heat_tuning_variant(int v, int* seg_width, int* rows, int* warps, int* has_fp64,
                                           int* stages, int* fused) {
  int info[6];
  if (!variant_info(v, info)) return set_error(HEAT_ERR_ARG, "heat_tuning_variant: unknown variant %d", v);
  if (seg_width) *seg_width = info[0];
  if (rows) *rows = info[1];
  if (warps) *warps = info[2];
  if (has_fp64) *has_fp64 = info[3];
  if (stages) *stages = info[4];
  if (fused) *fused = info[5];
  return HEAT_OK;
}

extern "C" heat_status heat_tuning_get(heat_tuning* t) {
  if (!t) return set_error(HEAT_ERR_ARG, "heat_tuning_get: null argument");
  const Tuning x = tuning_get();
  for (int i = 0; i < 3; ++i) {
    t->variant[i] = x.variant[i];
    t->seg_nodes[i] = x.seg_nodes[i];
    t->pw_quads[i] = x.pw_quads[i];
    t->open_w[i] = x.open_w[i];
    t->loop[i] = x.loop[i];
  }
  return HEAT_OK;
}

extern "C" heat_status heat_tuning_set(const heat_tuning* t) {
  if (!t) return set_error(HEAT_ERR_ARG, "heat_tuning_set: null argument");
  Tuning x;
  for (int i = 0; i < 3; ++i) {
    x.variant[i] = t->variant[i];
    x.seg_nodes[i] = t->seg_nodes[i];
    x.pw_quads[i] = t->pw_quads[i];
    x.open_w[i] = t->open_w[i];
    x.loop[i] = t->loop[i];
  }
  return tuning_set(x);
}

extern "C" heat_status heat_autotune(heat_sim* s, int reps, heat_tuning* best, double* best_ms) {
  if (!s || reps < 1) return set_error(HEAT_ERR_ARG, "heat_autotune: bad argument");
  if (!s->eng) return set_error(HEAT_ERR_ARG, "heat_autotune: call heat_step first");
  int v = 0, seg = 0;
  double ms = 0.0;
  heat_status st = engine_autotune(&s, 1, reps, &v, &seg, &ms);
  if (st != HEAT_OK) return st;
  engine_destroy(s->eng);  // rebuilt under the new table by the next heat_step
  s->eng = nullptr;
  if (best) st = heat_tuning_get(best);
  if (best_ms) *best_ms = ms;
  return st;
}

extern "C" heat_status heat_batch_autotune(heat_batch* b, int reps, heat_tuning* best, double* best_ms) {
  if (!b || reps < 1) return set_error(HEAT_ERR_ARG, "heat_batch_autotune: bad argument");
  int v = 0, seg = 0;
  double ms = 0.0;
  heat_status st = engine_autotune(b->sims.data(), (int)b->sims.size(), reps, &v, &seg, &ms);
  if (st != HEAT_OK) return st;
  // rebuild the batch's engine under the new table
  engine_destroy(b->eng);
  b->eng = nullptr;
  st = engine_create(b->sims.data(), (int)b->sims.size(), b->sims[0]->prm.precision, b->stream, &b->eng);
  if (st != HEAT_OK) return st;
  if (best) st = heat_tuning_get(best);
  if (best_ms) *best_ms = ms;
  return st;
}

// ------------------------------------------------------------ index checks

extern "C" int heat_checks_compiled(void) {
#ifdef HEAT_CHECK
  return 1;
#else
  return 0;
#endif
}

extern "C" heat_status heat_check_violations(heat_sim* s, unsigned int* count) {
  if (!s || !count) return set_error(HEAT_ERR_ARG, "heat_check_violations: null argument");
  heat_status st = sim_read_scalars(s);
  if (st != HEAT_OK) return st;
  *count = s->h_sc->check_violations;
  return HEAT_OK;
}
