// Internal host-side structures shared by the C ABI and the tick engine.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "heat.h"
#include "heat_dev.cuh"

struct heat_mesh {
  int nx, ny, nz;
  double origin[3], extent[3];
};

namespace heat {
struct Engine;
struct GridSync;
// The persistent inner iteration (loop_kernels.cuh): sims, apply and update
// work lists, their counts, the grid barrier state (with the round limit).
using LoopFn = void (*)(const SimDev*, const int2*, const int2*, const int*, GridSync*);
// Its instance for a register-prefetch warp-apply shape (segment width, rows,
// warps) and pointwise item size (groups per thread); nullptr if none.
LoopFn loop_kernel(int sx, int ny, int warps, int qpt);
}

struct heat_sim {
  const heat_mesh* mesh = nullptr;
  heat_bc bc{};
  heat_params prm{};
  cudaStream_t stream = nullptr;
  long long nn = 0, ne = 0;
  std::vector<void*> allocs;          // device buffers owned by the sim
  heat::SimDev dev{};                 // descriptor (host copy)
  heat::SimDev* d_dev = nullptr;      // descriptor (device copy, per-node kernels)
  heat::SimScalars* d_sc = nullptr;   // device scalars
  heat::SimScalars* h_sc = nullptr;   // pinned host mirror
  double* d_q6 = nullptr;
  double* d_qface[6] = {};            // per-element face flux densities in use (NULL: uniform)
  double* qface_buf[6] = {};          // their buffers (owned, in allocs)
  unsigned int* d_bad = nullptr;
  int iters_log_cap = 0;
  heat::Engine* eng = nullptr;        // single-simulation engine (lazy)
};

namespace heat {

heat_status set_error(heat_status st, const char* fmt, ...);
// Q1 element mass/stiffness entries of an hx*hy*hz box by corner XOR pattern.
void element_classes(double hx, double hy, double hz, double mhat[8], double khat[8]);
// The same element matrices' eigenvalues in the corners' Walsh basis, / 8.
void walsh_eigenvalues(double hx, double hy, double hz, double lam_m[8], double lam_k[8]);
// 8x8 mass (M, row-major by local corner) and stiffness (K) of an hx*hy*hz
// box split into six linear tetrahedra (heat.h HEAT_ELEM_P1).
void p1_box_matrices(double hx, double hy, double hz, double M[64], double K[64]);
heat_status sim_alloc(heat_sim* s, void** p, size_t bytes);
heat_status sim_upload_desc(heat_sim* s);
heat_status sim_read_scalars(heat_sim* s);
heat_status sim_write_scalars(heat_sim* s);
// Queue nsteps steps on a simulation (target, phase, counters; log capacity).
heat_status sim_prepare_steps(heat_sim* s, int nsteps);
// Device bytes a simulation of this size holds.
size_t sim_footprint(long long nn, long long ne);
// Statistics from the host copy of the scalars (after sim_read_scalars).
void sim_stats(const heat_sim* s, heat_step_stats* o);
// Recompute the flux vector F from the uniform face values and the
// per-element face arrays (asynchronous on the sim's stream).
heat_status sim_setup_flux(heat_sim* s);
// After the device coefficients changed: FP32 copy, Jacobi diagonal,
// Dirichlet lift, stored products invalidated; no host round trip (the
// caller guarantees valid coefficients).
heat_status sim_derive_async(heat_sim* s);

// Kernel tuning: warp-apply variant per precision (-1: block-tile apply) and
// segment tile size (nodes) per mesh-size bucket (size_bucket).
struct Tuning {
  int variant[3];
  int seg_nodes[3];
  int pw_quads[3];  // k_update: groups of 4 nodes per thread (1, 2 or 4), per precision
  int open_w[3];    // per precision: 1 runs k_open's passes in the warp-segment march (k_open_w)
  int loop[3];      // per precision: 1 runs a tick's CG iterations as one persistent kernel (k_cg_loop)
};
int size_bucket(long long nn);
int num_variants();
// {segment width, rows per thread, warps per block, has an FP64 kernel, cp.async stages,
//  fused iteration kernel}
bool variant_info(int v, int info[6]);
Tuning tuning_get();
heat_status tuning_set(const Tuning& t);
// Time CG iterations through the tick graph (engine_time_iterations) for
// every candidate (variant, segment size) on the simulations together (each
// must have run a step) and store the fastest in the table entries of their
// precision and of the first one's size bucket.
heat_status engine_autotune(heat_sim* const* sims, int nsims, int reps, int* best_variant, int* best_seg,
                            double* best_ms);
// yv[v] = A' vec64[v] for slots v < nslots on the sim's stream (the stored
// products a resumed FP32-path simulation needs; see k_product).
heat_status prime_products(heat_sim* s, int nslots);
// Mean ms per CG iteration over about `reps` iterations run through the
// engine's captured tick graph (as a solve runs them), every member kept
// iterating; leaves the members' solver state undefined.
heat_status engine_time_iterations(Engine* e, int reps, double* ms_per_iter);

// A set of simulations driven together by one captured tick graph (kernel
// choice from the tuning table, or from `tun` when given).
// headroom > 1 sizes the descriptor array and work lists for that many times
// the members' needs and the grids by those capacities, so that
// engine_set_members can change the members under the same captured graph.
heat_status engine_create(heat_sim* const* sims, int nsims, int precision, cudaStream_t stream, Engine** out,
                          const Tuning* tun = nullptr, double headroom = 1.0);
// Replace the members (same precision and element) without reallocating:
// HEAT_ERR_ARG when the set exceeds the engine's capacities (build a new
// engine then). New members' last-block counters are cleared; the graph is
// captured again only when the Chebyshev pass count or a grid changes.
heat_status engine_set_members(Engine* e, heat_sim* const* sims, int nsims);
void engine_destroy(Engine* e);
// Re-read the sims' descriptors (after a buffer or parameter change).
heat_status engine_refresh(Engine* e);
// Advance every sim of the engine by nsteps steps; stats[i] per sim (may be
// NULL). reset_counters clears the per-call counters first.
heat_status engine_step_all(Engine* e, int nsteps, heat_step_stats* stats, int reset_counters);
// Launch nticks ticks without waiting (the server drives its own loop).
heat_status engine_launch_ticks(Engine* e, int nticks);
// Phase of every simulation of the engine (host array of nsims ints); waits.
heat_status engine_read_phases(Engine* e, int* phases);
// Kernels launched so far by engine_launch_ticks / engine_step_all.
long long engine_launches(const Engine* e);
// Device bytes the engine needs for these simulations (work lists, partials).
size_t engine_footprint(long long nn, long long nx, long long ny, long long nz);
// Time reps CG iterations of the engine's first simulation (see heat_profile_iteration).
heat_status engine_profile(Engine* e, int reps, void* flush, size_t flush_bytes, double* ms_apply,
                           double* ms_update, double* bytes_apply, double* bytes_update);

}  // namespace heat

#define CUDA_TRY(call)                                                                               \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) {                                                                         \
      cudaGetLastError();                                                                            \
      return heat::set_error(HEAT_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
    }                                                                                                \
  } while (0)
