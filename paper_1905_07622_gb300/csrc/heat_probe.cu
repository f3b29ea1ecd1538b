// heat_probe_fma_rate: the fused multiply-add throughput of this GPU in FP64
// or FP32, the ceiling of the FP64 operator apply (whose arithmetic, not its
// memory traffic, bounds it on this GPU) and of the double-float passes.
//
// Every thread runs kChains independent FMA chains of kIters steps on
// registers (no memory traffic in the loop); the grid fills every SM several
// times over. The result is 2 flops per FMA over the CUDA-event time of the
// launch, best of `reps` launches.
#include <algorithm>
#include <cmath>

#include "engine.h"
#include "loop_kernels.cuh"

namespace {

constexpr int kChains = 8, kIters = 4096, kThreads = 256, kBlocksPerSM = 8;

template <class T>
__global__ void __launch_bounds__(kThreads) k_fma_rate(T seed, T* out) {
  T a[kChains];
  const T m = seed * T(0.999), c = T(1e-7);
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = seed + T(threadIdx.x + i);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = a[i] * m + c;
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == T(-1.2345)) out[0] = s;  // keeps the chains alive; never taken for seed in (0, 1)
}

template <class T>
heat_status probe(int reps, double* tflops) {
  int dev = 0, sms = 1;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  T* out = nullptr;
  CUDA_TRY(cudaMalloc(&out, sizeof(T)));
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  heat_status rc = HEAT_OK;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
      cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    rc = heat::set_error(HEAT_ERR_CUDA, "heat_probe_fma_rate: stream or event creation failed");
  }
  const int grid = sms * kBlocksPerSM;
  double best = 0.0;
  for (int r = -1; r < reps && rc == HEAT_OK; ++r) {  // r = -1: warm-up
    cudaEventRecord(a, st);
    k_fma_rate<T><<<grid, kThreads, 0, st>>>(T(0.5), out);
    cudaEventRecord(b, st);
    if (cudaEventSynchronize(b) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      rc = heat::set_error(HEAT_ERR_CUDA, "heat_probe_fma_rate: launch failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double flops = 2.0 * (double)grid * kThreads * kChains * kIters;
    if (r >= 0 && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e12);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  if (rc == HEAT_OK) *tflops = best;
  return rc;
}

// reps grid barriers of the persistent iteration (grid_barrier), nothing else
__global__ void __launch_bounds__(128) k_barrier_rate(heat::GridSync* gs, int reps, int* passed) {
  bool any = false;
  int ok = 1;
  for (int r = 0; r < reps && ok; ++r) ok = heat::grid_barrier(gs, gridDim.x, false, any) ? 1 : 0;
  if (threadIdx.x == 0 && ok) atomicAdd(passed, 1);
}

}  // namespace

// The cost of one grid barrier of the persistent iteration on its own: a
// cooperative launch of blocks_per_sm 128-thread blocks per SM runs reps
// barriers; best of three launches, after one warm-up.
extern "C" heat_status heat_probe_grid_barrier(int blocks_per_sm, int reps, double* us_per_barrier) {
  if (!us_per_barrier || blocks_per_sm < 1 || blocks_per_sm > 16 || reps < 1 || reps > 100000)
    return heat::set_error(HEAT_ERR_ARG, "heat_probe_grid_barrier: need 1 <= blocks_per_sm <= 16, 1 <= reps <= 1e5");
  int dev = 0, sms = 1, occ = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_barrier_rate, 128, 0));
  if (blocks_per_sm > occ) return heat::set_error(HEAT_ERR_ARG, "heat_probe_grid_barrier: at most %d blocks per SM", occ);
  heat::GridSync* gs = nullptr;
  int* passed = nullptr;
  CUDA_TRY(cudaMalloc(&gs, sizeof(heat::GridSync)));
  if (cudaMalloc(&passed, sizeof(int)) != cudaSuccess) {
    cudaFree(gs);
    return heat::set_error(HEAT_ERR_NOMEM, "heat_probe_grid_barrier: allocation failed");
  }
  cudaStream_t st = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  heat_status rc = HEAT_OK;
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&a) != cudaSuccess ||
      cudaEventCreate(&b) != cudaSuccess) {
    cudaGetLastError();
    rc = heat::set_error(HEAT_ERR_CUDA, "heat_probe_grid_barrier: stream or event creation failed");
  }
  const unsigned int grid = (unsigned int)(sms * blocks_per_sm);
  double best = 1e300;
  for (int t = -1; t < 3 && rc == HEAT_OK; ++t) {  // t = -1: warm-up
    heat::GridSync g{};
    g.limit_ns = 1000000000ull;  // 1 s per wait
    int zero = 0;
    if (cudaMemcpyAsync(gs, &g, sizeof(g), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(passed, &zero, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = heat::set_error(HEAT_ERR_CUDA, "heat_probe_grid_barrier: upload failed");
      break;
    }
    void* args[] = {&gs, &reps, &passed};
    cudaEventRecord(a, st);
    const cudaError_t le = cudaLaunchCooperativeKernel((const void*)k_barrier_rate, dim3(grid), dim3(128), args, 0, st);
    cudaEventRecord(b, st);
    int got = 0;
    if (le != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
        cudaMemcpy(&got, passed, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
      cudaGetLastError();
      rc = heat::set_error(HEAT_ERR_CUDA, "heat_probe_grid_barrier: launch failed");
      break;
    }
    if (got != (int)grid) {
      rc = heat::set_error(HEAT_ERR_TIMEOUT, "heat_probe_grid_barrier: a barrier wait ran out");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (t >= 0) best = std::min(best, (double)ms * 1e3 / reps);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (st) cudaStreamDestroy(st);
  cudaFree(gs);
  cudaFree(passed);
  if (rc == HEAT_OK) *us_per_barrier = best;
  return rc;
}

extern "C" heat_status heat_probe_fma_rate(int fp64, int reps, double* tflops) {
  if (!tflops || reps < 1 || (fp64 != 0 && fp64 != 1))
    return heat::set_error(HEAT_ERR_ARG, "heat_probe_fma_rate: need fp64 in {0, 1}, reps >= 1, tflops");
  return fp64 ? probe<double>(reps, tflops) : probe<float>(reps, tflops);
}
