// The inner CG iterations of a tick as ONE persistent kernel (k_cg_loop):
// every block stays resident (a cooperative launch, so that all blocks are
// on the GPU together) and runs, round after round, the work items of the
// warp-segment apply and then those of the pointwise update, with a grid
// barrier after each phase instead of a kernel boundary. The items are the
// same as those of k_apply_dot_w and k_update and run the same code
// (apply_w_item, update_item), so every result is bitwise the one of the
// replayed tick graph; only where the time goes changes: no launch, drain
// and ramp-up between the phases of an iteration.
//
// A round is one CG iteration of every member in PH_ITER (Algorithm 1's
// loop body, §3.3). The loop ends when no member stays in PH_ITER (each
// simulation's last update block reports whether it does, and the second
// barrier of the round combines the reports) or after `rounds` rounds; the
// next tick's k_open then takes the phase changes. The round limit is read
// from the barrier state, so that timing runs can lower it without a new
// graph.
//
// Every wait is bounded: a barrier wait that exceeds GridSync::limit_ns
// sets GridSync::abort and returns, and every other block's wait sees the
// flag and returns too, so the kernel ends and the host reports
// HEAT_ERR_TIMEOUT instead of the GPU hanging.
#pragma once

#include "tile_kernels.cuh"

namespace heat {

// Device state of the grid barrier (one per engine). The arrival counter,
// the word the waiting blocks poll and the abort flag sit on separate
// 128-byte lines, so the polls do not contend with the arrivals' atomics.
struct GridSync {
  unsigned int count;   // arrivals in bits 0-15, reported flags in bits 16-31
  unsigned int pad0_[31];
  unsigned int gen;     // (barrier generation << 1) | whether the last barrier saw a flag
  unsigned int pad1_[31];
  int abort;            // a wait ran out: every block leaves
  unsigned int extra;   // arrivals expected beyond the grid (a test hook: nonzero = no barrier completes)
  unsigned long long limit_ns;  // bound of one wait
  int rounds;           // rounds (CG iterations) one launch runs at most
  unsigned int pad2_[27];
};

__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier of the nb blocks of the launch. Each block arrives with
// a flag; `any` returns whether any block's flag was set. Returns false when
// the wait ran out or another block gave up (abort): the caller returns.
// Writes of the block before the barrier are visible to every block after
// it (a fence before the arrival, an acquire load after the wait).
__device__ __forceinline__ bool grid_barrier(GridSync* g, unsigned int nb, bool flag, bool& any) {
  __shared__ int s_res;  // bit 0: passed, bit 1: some block's flag was set
  __syncthreads();
  if (threadIdx.x == 0) {
    int res = 0;
    const unsigned int g0 = ld_acquire_gpu(&g->gen);  // the generation this barrier ends
    __threadfence();
    const unsigned int old = atomicAdd(&g->count, 1u + (flag ? 0x10000u : 0u));
    if ((old & 0xffffu) == nb - 1u + g->extra) {
      const bool f = ((old >> 16) + (flag ? 1u : 0u)) != 0u;
      atomicExch(&g->count, 0u);
      __threadfence();
      st_release_gpu(&g->gen, (g0 & ~1u) + 2u + (f ? 1u : 0u));
      res = 1 | (f ? 2 : 0);
    } else {
      const unsigned long long t0 = global_ns(), limit = g->limit_ns;
      for (unsigned int polls = 1;; ++polls) {
        const unsigned int gv = ld_acquire_gpu(&g->gen);
        if ((gv >> 1) != (g0 >> 1)) {
          res = 1 | ((gv & 1u) ? 2 : 0);
          break;
        }
        if ((polls & 63u) == 0u) {  // the abort flag and the clock, now and then
          if (ld_acquire_gpu(reinterpret_cast<const unsigned int*>(&g->abort)) != 0u) break;
          if (global_ns() - t0 > limit) {
            atomicExch(&g->abort, 1);
            break;
          }
        }
        __nanosleep(20);
      }
    }
    if (res && ld_acquire_gpu(reinterpret_cast<const unsigned int*>(&g->abort)) != 0u) res = 0;
    __threadfence();
    s_res = res;
  }
  __syncthreads();
  const int res = s_res;
  any = (res & 2) != 0;
  return (res & 1) != 0;
}

// cache_sim for a persistent kernel: after a grid barrier (stale) the
// cached simulation's control scalars are re-read even when the simulation
// is the same.
__device__ __forceinline__ void cache_sim_loop(const SimDev* __restrict__ sims, int sim, ItemCache& cache, int& cur,
                                               bool& stale) {
  if (sim != cur) {
    bool dep = true;  // no programmatic predecessor to wait for
    cache_sim(sims, sim, cache, cur, dep);
  } else if (stale) {
    __syncthreads();  // the previous item's users of the scalars are done
    if (threadIdx.x == 0) cache.c = load_ctl(cache.s.sc);
    __syncthreads();
  }
  stale = false;
}

// The persistent inner iteration of the FP32 paths on boxes of element E
// (the engine builds it for trilinear boxes) with the register-prefetch warp
// apply <SX, NY, WARPS>
// and the pointwise update of QPT groups per thread (VT = kPwThreads /
// (32 WARPS) update threads per thread of this block). work_aw / work_pw and
// nwork[2] / nwork[1] are the engine's apply and update work lists.
template <int P, int SX, int NY, int WARPS, int MINB, int QPT, int E>
__global__ void __launch_bounds__(32 * WARPS, MINB)
    k_cg_loop(const SimDev* __restrict__ sims, const int2* __restrict__ work_aw, const int2* __restrict__ work_pw,
              const int* __restrict__ nwork, GridSync* __restrict__ gs) {
  static_assert(P != P_FP64, "the persistent iteration runs the FP32 inner solve");
  static_assert(kPwThreads % (32 * WARPS) == 0, "update items must split evenly over the block");
  constexpr int VT = kPwThreads / (32 * WARPS);
  __shared__ double red[32];
  __shared__ ItemCache cache;
  int cur = -1;
  const int n_aw = nwork[2], n_pw = nwork[1], rounds = gs->rounds;
  const unsigned int nb = gridDim.x;
  for (int round = 0; round < rounds; ++round) {
    bool stale = true, any = false;
    for (int w = blockIdx.x; w < n_aw; w += gridDim.x) {
      const int2 wi = work_aw[w];
      cache_sim_loop(sims, wi.x, cache, cur, stale);
      if (cache.c.phase != PH_ITER) continue;
      apply_w_item<float, SX, NY, WARPS, 0, E, true>(cache.s, cache.c, wi.y, red, nullptr);
    }
    if (!grid_barrier(gs, nb, false, any)) return;
    stale = true;
    bool more = false;  // this block closed a simulation's iteration and it iterates on
    for (int w = blockIdx.x; w < n_pw; w += gridDim.x) {
      const int2 wi = work_pw[w];
      cache_sim_loop(sims, wi.x, cache, cur, stale);
      if (cache.c.phase != PH_ITER) continue;
      more |= update_item<float, P, QPT, VT, true>(cache.s, cache.c, wi.y, red);
    }
    if (!grid_barrier(gs, nb, more, any)) return;
    if (!any) break;
  }
}

}  // namespace heat
