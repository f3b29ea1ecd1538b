// The coefficient inverse problem of §5.3 on the device: per-element face
// flux, coefficients from a corrosion profile, the camera log-likelihood, and
// a Metropolis-Hastings driver whose chains' forward solves share one batch.
#include <cmath>
#include <cstring>
#include <vector>

#include "engine.h"
#include "heat.h"
#include "heat_dev.cuh"

using namespace heat;

namespace {

// Number of element faces and of nodes of a face of the mesh.
void face_dims(const heat_mesh* m, int face, long long* nelem, long long* nnode) {
  const int a = face < 2 ? m->ny : m->nx;
  const int b = face < 4 ? m->nz : m->ny;
  *nelem = (long long)a * b;
  *nnode = (long long)(a + 1) * (b + 1);
}

// (rho_c, k) of every element from the corrosion profile; the FP64
// operations are rounded one by one (no contraction), in the documented order.
__global__ void k_corrosion_coeffs(double2* __restrict__ coef, int nx, int ny, int nz, double oy, double oz,
                                   double hy, double hz, double y_rear, double depth, heat_corrosion g) {
  const long long ne = (long long)nx * ny * nz;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < ne;
       e += (long long)gridDim.x * blockDim.x) {
    const long long jk = e / nx;
    const int j = (int)(jk % ny), k = (int)(jk / ny);
    const double zc = __dadd_rn(oz, __dmul_rn((double)k + 0.5, hz));
    const double t = __ddiv_rn(__dsub_rn(zc, g.z0), g.half_width);
    const double d = __dmul_rn(depth, __dsub_rn(1.0, __dmul_rn(t, t)));
    const double yc = __dadd_rn(oy, __dmul_rn((double)j + 0.5, hy));
    const bool corr = fabs(t) < 1.0 && __dsub_rn(y_rear, yc) < d;
    coef[e] = corr ? make_double2(g.rho_c_corr, g.k_corr) : make_double2(g.rho_c_sound, g.k_sound);
  }
}

// One block: -1/2 sum ((U_i - data_i) / sigma)^2 over the face's nodes, in a
// fixed order (thread t takes nodes t, t + blockDim, ...; then a fixed tree).
// U is the state slot U^{n-1} read from the device scalars.
__global__ void k_face_loglik(const SimDev* __restrict__ sp, int face, const double* __restrict__ data,
                              double inv_sigma, double* __restrict__ out) {
  const SimDev& s = *sp;
  const double* __restrict__ u = s.vec64[__ldcg(&s.sc->iu1)];
  const int px = s.nx + 1, pxy = (s.nx + 1) * (s.ny + 1);
  const int na = face < 2 ? s.ny + 1 : s.nx + 1;
  const int nb = face < 4 ? s.nz + 1 : s.ny + 1;
  const int fixed = (face & 1) ? (face < 2 ? s.nx : (face < 4 ? s.ny : s.nz)) : 0;
  double acc = 0.0;
  for (int t = threadIdx.x; t < na * nb; t += blockDim.x) {
    const int a = t % na, b = t / na;
    int n;
    if (face < 2) n = fixed + px * a + pxy * b;
    else if (face < 4) n = a + px * fixed + pxy * b;
    else n = a + px * b + pxy * fixed;
    const double r = (u[n] - data[t]) * inv_sigma;
    acc += r * r;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) tot += red[w];
    *out = -0.5 * tot;
  }
}

__global__ void k_fill(double* __restrict__ p, long long n, double v) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = v;
}

int grid_of(long long n) { return (int)std::min<long long>((n + 255) / 256, 4096); }

bool valid_geom(const heat_corrosion* g) {
  return g && std::isfinite(g->z0) && g->half_width > 0.0 && std::isfinite(g->half_width) && g->rho_c_sound > 0.0 &&
         g->k_sound > 0.0 && g->rho_c_corr > 0.0 && g->k_corr > 0.0 && std::isfinite(g->rho_c_sound) &&
         std::isfinite(g->k_sound) && std::isfinite(g->rho_c_corr) && std::isfinite(g->k_corr);
}

}  // namespace

extern "C" heat_status heat_set_face_flux(heat_sim* s, int face, const double* q, int on_device) {
  if (!s || face < 0 || face > 5) return set_error(HEAT_ERR_ARG, "heat_set_face_flux: bad argument");
  long long nel, nnode;
  face_dims(s->mesh, face, &nel, &nnode);
  if (!q) {  // back to the uniform value (the buffer stays with the sim for reuse)
    s->d_qface[face] = nullptr;
    return sim_setup_flux(s);
  }
  if (!on_device) {
    for (long long e = 0; e < nel; ++e)
      if (!std::isfinite(q[e])) return set_error(HEAT_ERR_NONFINITE, "heat_set_face_flux: non-finite q at %lld", e);
  }
  if (!s->qface_buf[face]) {
    void* p = nullptr;
    heat_status st = sim_alloc(s, &p, (size_t)nel * sizeof(double));
    if (st != HEAT_OK) return st;
    s->qface_buf[face] = (double*)p;
  }
  CUDA_TRY(cudaMemcpyAsync(s->qface_buf[face], q, (size_t)nel * sizeof(double),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
  if (!on_device) CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->d_qface[face] = s->qface_buf[face];
  return sim_setup_flux(s);
}

extern "C" heat_status heat_set_coeffs_corrosion(heat_sim* s, const heat_corrosion* g, double depth) {
  if (!s || !valid_geom(g) || !(depth >= 0.0) || !std::isfinite(depth))
    return set_error(HEAT_ERR_ARG, "heat_set_coeffs_corrosion: bad argument");
  const heat_mesh* m = s->mesh;
  const double hy = m->extent[1] / m->ny, hz = m->extent[2] / m->nz;
  const double y_rear = m->origin[1] + m->extent[1];
  k_corrosion_coeffs<<<grid_of(s->ne), 256, 0, s->stream>>>(const_cast<double2*>(s->dev.coef), m->nx, m->ny, m->nz,
                                                            m->origin[1], m->origin[2], hy, hz, y_rear, depth, *g);
  CUDA_TRY(cudaGetLastError());
  return sim_derive_async(s);
}

extern "C" heat_status heat_face_loglik(heat_sim* s, int face, const double* data, double sigma, double* loglik) {
  if (!s || face < 0 || face > 5 || !data || !loglik || !(sigma > 0.0))
    return set_error(HEAT_ERR_ARG, "heat_face_loglik: bad argument");
  k_face_loglik<<<1, 1024, 0, s->stream>>>(s->d_dev, face, data, 1.0 / sigma, loglik);
  CUDA_TRY(cudaGetLastError());
  return HEAT_OK;
}

// ----------------------------------------------------------- MH driver

struct heat_mh {
  heat_mh_config cfg{};
  heat_mesh* mesh = nullptr;
  std::vector<heat_sim*> sims;
  heat_batch* batch = nullptr;
  cudaStream_t stream = nullptr;
  double* d_data = nullptr;
  double* d_ll = nullptr;
  double* h_ll = nullptr;
  double* d_u0 = nullptr;
  long long nn = 0;
  long long solves = 0, cg_iters = 0;
};

extern "C" void heat_mh_destroy(heat_mh* mh) {
  if (!mh) return;
  if (mh->stream) cudaStreamSynchronize(mh->stream);
  heat_destroy_batch(mh->batch);
  for (heat_sim* s : mh->sims) heat_destroy_sim(s);
  heat_destroy_mesh(mh->mesh);
  cudaFree(mh->d_data);
  cudaFree(mh->d_ll);
  cudaFree(mh->d_u0);
  if (mh->h_ll) cudaFreeHost(mh->h_ll);
  delete mh;
}

extern "C" heat_status heat_mh_create(const heat_mh_config* c, void* cuda_stream, heat_mh** out) {
  if (!out) return set_error(HEAT_ERR_ARG, "heat_mh_create: out is NULL");
  *out = nullptr;
  if (!c || c->nchains < 1 || c->nsteps < 1 || !c->data || !(c->sigma > 0.0) || !(c->depth_max > 0.0) ||
      c->obs_face < 0 || c->obs_face > 5 || c->flux_face < -1 || c->flux_face > 5 || !valid_geom(&c->geom) ||
      !std::isfinite(c->u0))
    return set_error(HEAT_ERR_ARG, "heat_mh_create: bad configuration");
  heat_mh* mh = new heat_mh();
  mh->cfg = *c;
  mh->cfg.flux_q = nullptr;  // not kept: copied into each simulation below
  mh->cfg.data = nullptr;
  mh->stream = (cudaStream_t)cuda_stream;
  auto fail = [&](heat_status st) {
    heat_mh_destroy(mh);
    return st;
  };
  heat_status st = heat_create_mesh(c->nx, c->ny, c->nz, c->origin, c->extent, &mh->mesh);
  if (st != HEAT_OK) return fail(st);
  long long nn = 0, ne = 0;
  heat_mesh_sizes(mh->mesh, &nn, &ne);
  mh->nn = nn;
  long long nel, nnode;
  face_dims(mh->mesh, c->obs_face, &nel, &nnode);
  if (cudaMalloc(&mh->d_data, sizeof(double) * nnode) != cudaSuccess ||
      cudaMalloc(&mh->d_ll, sizeof(double) * c->nchains) != cudaSuccess ||
      cudaMalloc(&mh->d_u0, sizeof(double) * nn) != cudaSuccess ||
      cudaMallocHost(&mh->h_ll, sizeof(double) * c->nchains) != cudaSuccess) {
    cudaGetLastError();
    return fail(set_error(HEAT_ERR_NOMEM, "heat_mh_create: allocation failed"));
  }
  if (cudaMemcpyAsync(mh->d_data, c->data, sizeof(double) * nnode, cudaMemcpyHostToDevice, mh->stream) != cudaSuccess)
    return fail(set_error(HEAT_ERR_CUDA, "heat_mh_create: data copy failed"));
  k_fill<<<grid_of(nn), 256, 0, mh->stream>>>(mh->d_u0, nn, c->u0);
  for (int i = 0; i < c->nchains; ++i) {
    heat_sim* s = nullptr;
    st = heat_sim_create(mh->mesh, &c->bc, &c->params, cuda_stream, &s);
    if (st != HEAT_OK) return fail(st);
    mh->sims.push_back(s);
    if (c->flux_face >= 0 && c->flux_q) {
      st = heat_set_face_flux(s, c->flux_face, c->flux_q, 0);
      if (st != HEAT_OK) return fail(st);
    }
    st = heat_set_coeffs_corrosion(s, &c->geom, 0.0);
    if (st != HEAT_OK) return fail(st);
  }
  st = heat_batch_create(mh->sims.data(), c->nchains, cuda_stream, &mh->batch);
  if (st != HEAT_OK) return fail(st);
  if (cudaStreamSynchronize(mh->stream) != cudaSuccess)
    return fail(set_error(HEAT_ERR_CUDA, "heat_mh_create: initialisation failed"));
  *out = mh;
  return HEAT_OK;
}

extern "C" heat_status heat_mh_loglik(heat_mh* mh, const double* depths, double* loglik) {
  if (!mh || !depths || !loglik) return set_error(HEAT_ERR_ARG, "heat_mh_loglik: bad argument");
  const int n = mh->cfg.nchains;
  for (int i = 0; i < n; ++i)
    if (!(depths[i] >= 0.0) || !std::isfinite(depths[i]))
      return set_error(HEAT_ERR_ARG, "heat_mh_loglik: depth %d is not a finite value >= 0", i);
  for (int i = 0; i < n; ++i) {
    heat_sim* s = mh->sims[i];
    heat_status st = heat_set_coeffs_corrosion(s, &mh->cfg.geom, depths[i]);
    if (st != HEAT_OK) return st;
    st = heat_set_state(s, mh->d_u0, 1);
    if (st != HEAT_OK) return st;
  }
  std::vector<heat_step_stats> stats(n);
  heat_status st = heat_batch_step(mh->batch, mh->cfg.nsteps, stats.data());
  if (st != HEAT_OK) return st;
  mh->solves += n;
  for (const heat_step_stats& x : stats) mh->cg_iters += x.iters;
  for (int i = 0; i < n; ++i) {
    st = heat_face_loglik(mh->sims[i], mh->cfg.obs_face, mh->d_data, mh->cfg.sigma, mh->d_ll + i);
    if (st != HEAT_OK) return st;
  }
  CUDA_TRY(cudaMemcpyAsync(mh->h_ll, mh->d_ll, sizeof(double) * n, cudaMemcpyDeviceToHost, mh->stream));
  CUDA_TRY(cudaStreamSynchronize(mh->stream));
  std::memcpy(loglik, mh->h_ll, sizeof(double) * n);
  return HEAT_OK;
}

extern "C" heat_status heat_mh_run(heat_mh* mh, int niter, double step, const double* normals,
                                   const double* uniforms, double* state, double* state_ll, double* depth_trace,
                                   double* ll_trace, int* accepted) {
  if (!mh || niter < 0 || !(step > 0.0) || !normals || !uniforms || !state)
    return set_error(HEAT_ERR_ARG, "heat_mh_run: bad argument");
  const int n = mh->cfg.nchains;
  std::vector<double> ll(n), prop(n), pll(n);
  heat_status st = HEAT_OK;
  if (state_ll) {
    std::memcpy(ll.data(), state_ll, sizeof(double) * n);
  } else {
    st = heat_mh_loglik(mh, state, ll.data());
    if (st != HEAT_OK) return st;
  }
  for (int it = 0; it < niter; ++it) {
    std::vector<char> inside(n);
    for (int i = 0; i < n; ++i) {
      volatile double move = step * normals[(size_t)it * n + i];  // two roundings, never a fused multiply-add
      prop[i] = state[i] + move;
      inside[i] = prop[i] >= 0.0 && prop[i] <= mh->cfg.depth_max;
    }
    // every chain keeps its slot in the batch; a chain whose proposal is
    // outside the prior re-solves its current depth and rejects
    std::vector<double> solve(n);
    for (int i = 0; i < n; ++i) solve[i] = inside[i] ? prop[i] : state[i];
    st = heat_mh_loglik(mh, solve.data(), pll.data());
    if (st != HEAT_OK) return st;
    for (int i = 0; i < n; ++i) {
      const size_t k = (size_t)it * n + i;
      const bool acc = inside[i] && std::log(uniforms[k]) < pll[i] - ll[i];
      if (acc) {
        state[i] = prop[i];
        ll[i] = pll[i];
      }
      if (depth_trace) depth_trace[k] = state[i];
      if (ll_trace) ll_trace[k] = ll[i];
      if (accepted) accepted[k] = acc ? 1 : 0;
    }
  }
  if (state_ll) std::memcpy(state_ll, ll.data(), sizeof(double) * n);
  return HEAT_OK;
}

extern "C" heat_status heat_mh_stats(const heat_mh* mh, long long* solves, long long* cg_iters) {
  if (!mh) return set_error(HEAT_ERR_ARG, "heat_mh_stats: mh is NULL");
  if (solves) *solves = mh->solves;
  if (cg_iters) *cg_iters = mh->cg_iters;
  return HEAT_OK;
}
