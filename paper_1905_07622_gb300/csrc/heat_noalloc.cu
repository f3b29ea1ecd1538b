// heat_apply_dot_noalloc: the operator apply with its d.Ad dot product for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: real-time loops that forbid allocation
// after start-up, and hosts whose memory manager owns all device memory and
// hands out only the buffers it was given. Those callers already hold their
// inputs and outputs; what they cannot provide is the kernel's reduction
// scratch (one partial sum per tile plus a completion counter). This entry
// point keeps that scratch in a fixed file-scope device array, so a call
// allocates nothing: no cudaMalloc, no cudaFree, no allocating library
// routine. It covers trilinear boxes only.
//
// Consequences for the caller:
//   * every GPU that loads the library holds the array, (4096 + 32) doubles =
//     33,024 bytes, until exit;
//   * every call shares it, and it keeps the last call's contents: calls that
//     overlap on the GPU (two streams, or two host threads) race on it and
//     must be serialised by the caller;
//   * the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call
//     before any stream capture.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "engine.h"
#include "op.cuh"

// One FP64 partial sum per tile, then the completion counter (as an unsigned
// int in the first slot after the partials).
static __device__ __align__(256) double g_noalloc_scratch[HEAT_NOALLOC_MAX_TILES + 32];

namespace {

constexpr int kTX = 32, kTY = 4, kTZ = 8;  // nodes per tile (1024), one thread per (x, y) column

// y = A' x (A = M/dt + theta K with Dirichlet rows and columns replaced by the
// identity), and xdoty = x . y summed per tile in tile order by the last block.
__global__ void __launch_bounds__(kTX* kTY)
    k_apply_dot_noalloc(const heat::SimDev s, const double* __restrict__ x, double* __restrict__ y,
                        double* __restrict__ xdoty, double* __restrict__ scratch) {
  __shared__ double red[32];
  __shared__ int s_last;
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + HEAT_NOALLOC_MAX_TILES);
  const int ntx = (s.nx + kTX) / kTX, nty = (s.ny + kTY) / kTY;
  for (int t = blockIdx.x; t < s.ntiles; t += gridDim.x) {
    const int tx = t % ntx, ty = (t / ntx) % nty, tz = t / (ntx * nty);
    const int i = tx * kTX + (int)(threadIdx.x % kTX), j = ty * kTY + (int)(threadIdx.x / kTX);
    double part[1] = {0.0};
    if (i <= s.nx && j <= s.ny) {
      for (int kz = 0; kz < kTZ; ++kz) {
        const int k = tz * kTZ + kz;
        if (k > s.nz) break;
        const long long n = heat::node_index(s, i, j, k);
        double yn;
        if (heat::is_dirichlet(s, i, j, k)) {
          yn = x[n];
        } else {
          yn = heat::gather_apply<double>(s, s.inv_dt, s.theta, i, j, k, [&](int a, int b, int c) -> double {
            return heat::is_dirichlet(s, a, b, c) ? 0.0 : x[heat::node_index(s, a, b, c)];
          });
        }
        y[n] = yn;
        part[0] += x[n] * yn;
      }
    }
    heat::block_sum<1>(part, red);
    if (threadIdx.x == 0) {
      scratch[t] = part[0];
      __threadfence();
      s_last = (atomicAdd(counter, 1u) == (unsigned int)(s.ntiles - 1));
    }
    __syncthreads();
    if (s_last) {
      __threadfence();
      double tot[1] = {0.0};
      for (int u = threadIdx.x; u < s.ntiles; u += blockDim.x) tot[0] += __ldcg(&scratch[u]);
      heat::block_sum<1>(tot, red);
      if (threadIdx.x == 0) {
        *xdoty = tot[0];
        *counter = 0u;
      }
    }
    __syncthreads();
  }
}

std::mutex g_mu;
double* g_scratch_ptr[64] = {};

// Device address of g_noalloc_scratch on the current device (looked up once).
heat_status scratch_for_current_device(double** out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return heat::set_error(HEAT_ERR_ARG, "heat_apply_dot_noalloc: device id %d >= 64", dev);
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return heat::set_error(HEAT_ERR_CUDA, "heat_apply_dot_noalloc: cudaGetSymbolAddress failed: %s",
                             cudaGetErrorString(e));
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return HEAT_OK;
}

}  // namespace

extern "C" heat_status heat_apply_dot_noalloc(int nx, int ny, int nz, const double extent[3], double dt,
                                              double theta, uint32_t dirichlet_faces, const double* coef,
                                              const double* x, double* y, double* xdoty, void* cuda_stream) {
  if (nx < 1 || ny < 1 || nz < 1 || !extent || !coef || !x || !y || !xdoty)
    return heat::set_error(HEAT_ERR_ARG, "heat_apply_dot_noalloc: bad mesh size or null pointer");
  for (int d = 0; d < 3; ++d)
    if (!(extent[d] > 0.0) || !std::isfinite(extent[d]))
      return heat::set_error(HEAT_ERR_ARG, "heat_apply_dot_noalloc: extent must be finite and > 0");
  if (!(dt > 0.0) || !std::isfinite(dt) || !(theta > 0.0 && theta <= 1.0))
    return heat::set_error(HEAT_ERR_ARG, "heat_apply_dot_noalloc: need dt > 0 and 0 < theta <= 1");
  if (reinterpret_cast<uintptr_t>(coef) % 16 != 0)
    return heat::set_error(HEAT_ERR_ARG, "heat_apply_dot_noalloc: coef must be 16-byte aligned");
  const long long ntiles = (long long)((nx + kTX) / kTX) * ((ny + kTY) / kTY) * ((nz + kTZ) / kTZ);
  if (ntiles > HEAT_NOALLOC_MAX_TILES)
    return heat::set_error(HEAT_ERR_ARG,
                           "heat_apply_dot_noalloc: a %dx%dx%d mesh needs %lld tiles of 32x4x8 nodes; the static "
                           "scratch holds at most %d (use heat_sim_create + heat_apply for larger meshes)",
                           nx, ny, nz, ntiles, HEAT_NOALLOC_MAX_TILES);
  double* scratch = nullptr;
  heat_status st = scratch_for_current_device(&scratch);
  if (st != HEAT_OK) return st;

  heat::SimDev s{};
  s.nx = nx;
  s.ny = ny;
  s.nz = nz;
  s.nn = (long long)(nx + 1) * (ny + 1) * (nz + 1);
  s.ntiles = (int)ntiles;
  s.dir_faces = dirichlet_faces & 63u;
  s.inv_dt = 1.0 / dt;
  s.theta = theta;
  heat::element_classes(extent[0] / nx, extent[1] / ny, extent[2] / nz, s.mhat, s.khat);
  s.coef = reinterpret_cast<const double2*>(coef);

  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  // the completion counter must start at zero (a previous call leaves it at
  // zero, but an interrupted one might not)
  CUDA_TRY(cudaMemsetAsync(scratch + HEAT_NOALLOC_MAX_TILES, 0, sizeof(unsigned int), stream));
  int dev = 0, sms = 148;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::min<long long>(ntiles, (long long)sms * 8);
  k_apply_dot_noalloc<<<grid, kTX * kTY, 0, stream>>>(s, x, y, xdoty, scratch);
  CUDA_TRY(cudaGetLastError());
  return HEAT_OK;
}
