// The tick engine: a set of simulations advanced together by one captured
// CUDA graph of phase-gated kernels. One tick is
//   k_open, then iters_per_tick x (k_apply_dot, k_update),
// over device-side work lists of (simulation, operator tile) and
// (simulation, pointwise chunk) pairs. Each simulation carries its own phase,
// so simulations of different sizes, at different steps and iterations, share
// every launch; the host only replays the graph and polls a counter of
// unfinished simulations every few ticks (the paper's host reads the residual
// back after every iteration, §3.4.3).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "engine.h"
#include "loop_kernels.cuh"
#include "open_kernels.cuh"

namespace heat {

using TileFn = void (*)(const SimDev*, const int2*, const int*);

struct KernelSet {
  TileFn open, apply, update;
  int sx, sy;
  int open_threads, apply_threads;
  // warp-segment apply (FP32 paths); when set it replaces `apply`
  TileFn apply_w;
  int wsx, wny, wwarps;
  int pw_chunk;  // nodes per pointwise (k_update) work item
  int seg_nodes[3];  // warp-segment tile size per mesh-size bucket
  int apply_w_smem;  // dynamic shared memory of apply_w per block
  bool fused;        // apply_w is k_cg_iter: one kernel per CG iteration, no update kernel
  // Chebyshev passes: block form, and the warp form matching apply_w (which
  // then replaces it, on the same work list)
  TileFn cheb, cheb_w;
  // step-start and refinement passes in the warp-segment march (replaces
  // `open` when set), on their own segment geometry and work list
  TileFn open_w = nullptr;
  int owsx = 0, owny = 0, owwarps = 0;
  long long open_cap = 0;  // blocks of open_w resident on the GPU at once (0: unknown)
  // the CG iterations of a tick as one persistent kernel (replaces the
  // apply and update launches when set; FP32 paths, register-prefetch apply)
  LoopFn loop = nullptr;
};

// The warp-segment forms of k_open (tuning open_w): 32-lane segments of 2
// rows (shape 1) or 1 row (shape 2), 4 warps per block; double-float on the
// FP32 paths, FP64 on the FP64 path. Two rows hold twice the double-width
// values of a lane (254 registers, 2 blocks per SM); one row fits 168
// registers and 3 blocks per SM at the cost of more halo rows per output.
constexpr int kOpenSX = 32, kOpenWarps = 4;
static int open_w_rows(int shape) { return shape == 2 ? 1 : 2; }
static TileFn open_w_kernel(int prec, int shape) {
  if (shape == 2) {
    switch (prec) {
      case P_FP64: return k_open_w<P_FP64, kOpenSX, 1, kOpenWarps, 3>;
      case P_FP32_REFINED: return k_open_w<P_FP32_REFINED, kOpenSX, 1, kOpenWarps, 3>;
      default: return k_open_w<P_FP32_PLAIN, kOpenSX, 1, kOpenWarps, 3>;
    }
  }
  switch (prec) {
    case P_FP64: return k_open_w<P_FP64, kOpenSX, 2, kOpenWarps, 1>;
    case P_FP32_REFINED: return k_open_w<P_FP32_REFINED, kOpenSX, 2, kOpenWarps, 2>;
    default: return k_open_w<P_FP32_PLAIN, kOpenSX, 2, kOpenWarps, 2>;
  }
}

template <int P, int SX, int SY, int E = E_Q1>
static KernelSet make_set() {
  using T = typename std::conditional<P == P_FP64, double, float>::type;
  return {k_open<P, SX, SY, E>, k_apply_dot<T, SX, SY, E>, k_update<T, P, sizeof(T) == 4 ? 4 : 2>, SX, SY, SX * SY,
          SX * SY, nullptr, 0, 0, 0, pw_chunk(sizeof(T) == 4 ? 4 : 2), {512, 512, 512}, 0, false,
          k_cheb<T, SX, SY, E>, nullptr};
}

// Warp-segment apply variants the tuner chooses from: segment width, rows per
// lane, warps per block, cp.async stages (0: register prefetch); f64 is null
// where the FP64 registers or shared memory do not fit. Each kernel exists
// for both elements (the march differs, op_warp.cuh); index 0 trilinear
// boxes, 1 six-tetrahedra boxes.
struct WVariant {
  int sx, ny, warps, stages;
  TileFn f32[2], f64[2];
  int smem32, smem64;  // dynamic shared memory per block
  bool fused;          // FP32 only: the fused iteration kernel k_cg_iter
  TileFn cheb32[2], cheb64[2];  // Chebyshev passes of this segment shape (null: fused)
};
// One register-prefetch Chebyshev pass kernel per segment shape and type,
// bounded like that shape's register-prefetch apply (FP64: one block per SM).
template <class T, int SX, int NY, int W, bool ON, int E>
static constexpr TileFn chebfn() {
  if constexpr (!ON) {
    return nullptr;
  } else if constexpr (sizeof(T) == 8) {
    return k_cheb_w<double, SX, NY, W, 1, E>;
  } else {
    constexpr int MINB = (SX == 16 && NY == 2) ? 2 : ((SX == 32 && NY == 2) ? 4 : 3);
    return k_cheb_w<float, SX, NY, W, MINB, E>;
  }
}
template <class T, int SX, int NY, int W, int S, int MINB, bool ON, int E>
static constexpr TileFn wfn() {
  if constexpr (ON) return k_apply_dot_w<T, SX, NY, W, S, MINB, E>;
  else return nullptr;
}
template <int SX, int NY, int W, int S, int MINB, int MINB64>
static constexpr WVariant wv() {
  return {SX,
          NY,
          W,
          S,
          {wfn<float, SX, NY, W, S, MINB, true, E_Q1>(), wfn<float, SX, NY, W, S, MINB, true, E_P1>()},
          {wfn<double, SX, NY, W, S, MINB64, (MINB64 > 0), E_Q1>(),
           wfn<double, SX, NY, W, S, MINB64, (MINB64 > 0), E_P1>()},
          S ? 32 * W * async_stage_bytes<float, NY, (S ? S : 2)>() : 0,
          S ? 32 * W * async_stage_bytes<double, NY, (S ? S : 2)>() : 0,
          false,
          {chebfn<float, SX, NY, W, true, E_Q1>(), chebfn<float, SX, NY, W, true, E_P1>()},
          {chebfn<double, SX, NY, W, (MINB64 > 0), E_Q1>(), chebfn<double, SX, NY, W, (MINB64 > 0), E_P1>()}};
}
template <int SX, int NY, int W, int MINB>
static constexpr WVariant wv_fused() {
  return {SX, NY, W, 0, {k_cg_iter<SX, NY, W, MINB, E_Q1>, k_cg_iter<SX, NY, W, MINB, E_P1>}, {nullptr, nullptr},
          0,  0,  true, {nullptr, nullptr}, {nullptr, nullptr}};
}
// (segment width, rows, warps, stages, min blocks per SM for float / double,
// 0 = no double kernel)
static const WVariant kVariants[] = {
    wv<16, 4, 4, 0, 3, 0>(), wv<32, 4, 4, 0, 3, 0>(), wv<16, 2, 8, 0, 2, 1>(), wv<32, 2, 4, 0, 4, 1>(),
    wv<16, 4, 4, 3, 4, 0>(), wv<32, 4, 4, 3, 4, 0>(), wv<16, 2, 8, 3, 2, 1>(), wv<32, 4, 4, 3, 3, 0>(),
    wv<32, 4, 4, 4, 3, 0>(),     wv_fused<16, 4, 4, 2>(), wv_fused<32, 4, 4, 2>(), wv_fused<16, 4, 4, 3>(),
    wv_fused<32, 4, 4, 3>(),     wv_fused<16, 2, 8, 2>(), wv_fused<32, 2, 4, 4>(),
};
constexpr int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

// Process-wide tuning table, read when an engine is created: the warp apply
// variant per precision (-1: the block-tile apply) and the segment tile size
// per mesh-size bucket. Both are fixed per simulation size, so results stay
// bitwise identical alone and in batches built under the same table.
static Tuning g_tuning = {{-1, 0, 0}, {512, 512, 512}, {2, 4, 4}, {2, 2, 2}, {0, 0, 0}};
static std::mutex g_tuning_mu;

int num_variants() { return kNumVariants; }

bool variant_info(int v, int info[6]) {
  if (v < 0 || v >= kNumVariants) return false;
  info[0] = kVariants[v].sx;
  info[1] = kVariants[v].ny;
  info[2] = kVariants[v].warps;
  info[3] = kVariants[v].f64[0] != nullptr;
  info[4] = kVariants[v].stages;
  info[5] = kVariants[v].fused;
  return true;
}

int size_bucket(long long nn) { return nn < 200000 ? 0 : (nn < 4000000 ? 1 : 2); }

Tuning tuning_get() {
  std::lock_guard<std::mutex> lock(g_tuning_mu);
  return g_tuning;
}

heat_status tuning_set(const Tuning& t) {
  for (int p = 0; p < 3; ++p) {
    const int v = t.variant[p];
    if (v < -1 || v >= kNumVariants || (v >= 0 && p == P_FP64 && !kVariants[v].f64[0]))
      return set_error(HEAT_ERR_ARG, "tuning: bad variant %d for precision %d", v, p);
  }
  for (int p = 0; p < 3; ++p)
    if (t.pw_quads[p] != 1 && t.pw_quads[p] != 2 && t.pw_quads[p] != 4)
      return set_error(HEAT_ERR_ARG, "tuning: pointwise groups %d not 1, 2 or 4", t.pw_quads[p]);
  for (int p = 0; p < 3; ++p)
    if (t.open_w[p] < 0 || t.open_w[p] > 2)
      return set_error(HEAT_ERR_ARG, "tuning: open_w[%d] = %d not 0, 1 or 2", p, t.open_w[p]);
  for (int p = 0; p < 3; ++p)
    if (t.loop[p] < 0 || t.loop[p] > 1 || (p == P_FP64 && t.loop[p] != 0))
      return set_error(HEAT_ERR_ARG, "tuning: loop[%d] = %d not 0 or 1 (0 for FP64)", p, t.loop[p]);
  for (int b = 0; b < 3; ++b)
    if (t.seg_nodes[b] < 32 || t.seg_nodes[b] > (1 << 20))
      return set_error(HEAT_ERR_ARG, "tuning: segment size %d out of range", t.seg_nodes[b]);
  std::lock_guard<std::mutex> lock(g_tuning_mu);
  g_tuning = t;
  return HEAT_OK;
}

template <class T, int P>
static TileFn update_for(int qpt) {
  return qpt == 1 ? k_update<T, P, 1> : (qpt == 2 ? k_update<T, P, 2> : k_update<T, P, 4>);
}
static TileFn update_kernel(int prec, int qpt) {
  switch (prec) {
    case P_FP64: return update_for<double, P_FP64>(qpt);
    case P_FP32_REFINED: return update_for<float, P_FP32_REFINED>(qpt);
    default: return update_for<float, P_FP32_PLAIN>(qpt);
  }
}

static int sm_count();

// The kernels of precision prec under tuning table t. With Chebyshev passes
// (cheb) a fused variant is replaced by the register-prefetch variant of the
// same segment shape: the fused iteration has no place for the passes.
static KernelSet kernel_set(int prec, const Tuning& t, bool cheb = false, int elem = E_Q1) {
  const int ei = elem == E_P1 ? 1 : 0;
  int variant = t.variant[prec];
  if (cheb && variant >= 0 && variant < kNumVariants && kVariants[variant].fused) {
    const WVariant& f = kVariants[variant];
    int alt = -1;
    for (int v = 0; v < kNumVariants && alt < 0; ++v)
      if (!kVariants[v].fused && kVariants[v].stages == 0 && kVariants[v].sx == f.sx && kVariants[v].ny == f.ny &&
          kVariants[v].warps == f.warps)
        alt = v;
    variant = alt >= 0 ? alt : 0;
  }
  KernelSet k;
  if (elem == E_P1)
    k = prec == P_FP64 ? make_set<P_FP64, 16, 16, E_P1>()
                       : (prec == P_FP32_REFINED ? make_set<P_FP32_REFINED, 16, 16, E_P1>()
                                                  : make_set<P_FP32_PLAIN, 16, 16, E_P1>());
  else
    k = prec == P_FP64 ? make_set<P_FP64, 16, 16>()
                       : (prec == P_FP32_REFINED ? make_set<P_FP32_REFINED, 16, 16>()
                                                  : make_set<P_FP32_PLAIN, 16, 16>());
  if (variant >= 0 && variant < kNumVariants) {
    const WVariant& v = kVariants[variant];
    k.apply_w = prec == P_FP64 ? v.f64[ei] : v.f32[ei];
    if (k.apply_w) {
      k.wsx = v.sx;
      k.wny = v.ny;
      k.wwarps = v.warps;
      k.apply_w_smem = prec == P_FP64 ? v.smem64 : v.smem32;
      k.fused = v.fused;
      k.cheb_w = prec == P_FP64 ? v.cheb64[ei] : v.cheb32[ei];
      if (k.apply_w_smem > 0)
        cudaFuncSetAttribute(k.apply_w, cudaFuncAttributeMaxDynamicSharedMemorySize, k.apply_w_smem);
      // the persistent iteration: FP32 paths, trilinear boxes, register
      // prefetch, separate update, no Chebyshev passes
      if (t.loop[prec] && prec != P_FP64 && elem == E_Q1 && !cheb && !v.fused && v.stages == 0)
        k.loop = loop_kernel(v.sx, v.ny, v.warps, t.pw_quads[prec]);
    }
  }
  if (elem == E_Q1 && t.open_w[prec]) {
    k.open_w = open_w_kernel(prec, t.open_w[prec]);
    k.owsx = kOpenSX;
    k.owny = open_w_rows(t.open_w[prec]);
    k.owwarps = kOpenWarps;
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k.open_w, 32 * kOpenWarps, 0) == cudaSuccess && occ > 0)
      k.open_cap = (long long)sm_count() * occ;
    else
      cudaGetLastError();
  }
  for (int b = 0; b < 3; ++b) k.seg_nodes[b] = t.seg_nodes[b];
  const int qpt = t.pw_quads[prec];
  k.pw_chunk = pw_chunk(qpt);
  k.update = update_kernel(prec, qpt);
  return k;
}

// Number of simulations not yet DONE or FAILED.
__global__ void k_count_unfinished(const SimDev* __restrict__ sims, int nsims, int* out) {
  int c = 0;
  for (int i = threadIdx.x; i < nsims; i += blockDim.x) {
    const int ph = *(volatile const int*)&sims[i].sc->phase;
    c += (ph != PH_DONE && ph != PH_FAILED && ph != PH_IDLE) ? 1 : 0;
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
  __shared__ int red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    for (int w = 0; w < (int)((blockDim.x + 31) >> 5); ++w) t += red[w];
    *out = t;
  }
}

struct Engine {
  std::vector<heat_sim*> sims;
  int prec = 0;
  KernelSet ks{};
  cudaStream_t stream = nullptr;
  SimDev* d_sims = nullptr;
  int2* d_work_op = nullptr;
  int2* d_work_pw = nullptr;
  int2* d_work_aw = nullptr;  // warp-segment apply items
  long long cap_aw = 0;
  int grid_aw = 0;
  std::vector<int2> h_aw;
  int2* d_work_ow = nullptr;  // warp-segment open-pass items
  long long cap_ow = 0;
  int grid_ow = 0;
  std::vector<int2> h_ow;
  // [0] operator tiles, [1] pointwise chunks, [2] warp-apply items, [3] warp open-pass items
  int* d_nwork = nullptr;
  int* d_unfinished = nullptr;  // [2]: the two poll slots of engine_step_all
  int* h_unfinished = nullptr;  // [2], pinned
  cudaEvent_t poll_ev[2] = {nullptr, nullptr};
  double* d_partial = nullptr;
  long long cap_op = 0, cap_pw = 0, cap_partial = 0;
  int grid_op = 0, grid_pw = 0, iters_per_tick = 6;
  int elem = E_Q1;  // the members' finite element (one per engine)
  int ncheb = 0;    // Chebyshev passes per iteration in the tick: max over members of degree - 1
  int grid_ch = 0;  // grid of the pass kernel
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // persistent iteration (ks.loop): its barrier state and grid
  GridSync* d_sync = nullptr;
  int* h_abort = nullptr;
  int grid_loop = 0;
  long long launches = 0;  // kernels launched by the last engine_step_all
  int* d_phases = nullptr;
  int* h_phases = nullptr;
  int phases_cap = 0;
  std::vector<SimDev> h_sims;
  std::vector<int2> h_op, h_pw;
  long long cap_sims = 0;   // simulations the descriptor array holds
  bool grid_cap = false;    // grids sized by the capacities (members can change without a new graph)
};

// Host-side fault injection for tests of the server's recovery: the next
// g_fail_builds engine builds or membership updates return HEAT_ERR_NOMEM.
static std::atomic<int> g_fail_builds{0};
static bool injected_failure() {
  int n = g_fail_builds.load();
  while (n > 0)
    if (g_fail_builds.compare_exchange_weak(n, n - 1)) return true;
  return false;
}

// Kernels in one tick: k_open, then per iteration the Chebyshev passes and
// apply + update, or the fused kernel; or k_open and the persistent loop.
static int tick_launches(const Engine* e) {
  if (e->ks.loop) return 2;
  return 1 + (e->ncheb + (e->ks.fused ? 1 : 2)) * e->iters_per_tick;
}

// Rounds (CG iterations) one persistent launch runs at most: a solve's
// inner iterations normally end it first, at a phase change.
constexpr int kLoopRounds = 256;

// Test hook (heat_debug_loop_wait): arrivals the barrier expects beyond the
// grid, and the bound of one wait in ns (0: the engine's own bound).
static std::atomic<unsigned int> g_loop_extra{0};
static std::atomic<unsigned long long> g_loop_limit_ns{0};

// Barrier state for a fresh launch. One wait is bounded by 1 s plus 50 ns
// per node of the members (a phase of the largest batches takes far less),
// or by the test hook's bound; a launch runs at most `rounds` iterations.
static heat_status loop_sync_reset(Engine* e, int rounds = kLoopRounds) {
  if (!e->d_sync) return HEAT_OK;
  long long nodes = 0;
  for (const heat_sim* s : e->sims) nodes += s->nn;
  GridSync g{};
  g.extra = g_loop_extra.load();
  const unsigned long long hook = g_loop_limit_ns.load();
  g.limit_ns = hook ? hook : 1000000000ull + 50ull * (unsigned long long)nodes;
  g.rounds = rounds;
  CUDA_TRY(cudaMemcpyAsync(e->d_sync, &g, sizeof(g), cudaMemcpyHostToDevice, e->stream));
  CUDA_TRY(cudaStreamSynchronize(e->stream));
  return HEAT_OK;
}

// After a persistent launch gave up waiting (GridSync::abort): the members'
// iteration state is incomplete, so every member that has not finished
// fails with HEAT_ERR_TIMEOUT, and the barrier state is reset.
static heat_status loop_abort(Engine* e) {
  for (heat_sim* s : e->sims) {
    heat_status st = sim_read_scalars(s);
    if (st != HEAT_OK) return st;
    SimScalars* sc = s->h_sc;
    if (sc->phase != PH_DONE && sc->phase != PH_FAILED && sc->phase != PH_IDLE) {
      sc->status = HEAT_ERR_TIMEOUT;
      sc->phase = PH_FAILED;
    }
    sc->count = 0;
    st = sim_write_scalars(s);
    if (st != HEAT_OK) return st;
  }
  e->h_abort[0] = e->h_abort[1] = 0;
  return loop_sync_reset(e);
}

// Chebyshev passes the members need per iteration.
static int members_ncheb_of(heat_sim* const* sims, int nsims) {
  int n = 0;
  for (int i = 0; i < nsims; ++i) n = std::max(n, sims[i]->dev.cheb_m >= 2 ? sims[i]->dev.cheb_m - 1 : 0);
  return n;
}
static int members_ncheb(const Engine* e) { return members_ncheb_of(e->sims.data(), (int)e->sims.size()); }

// Operator tile geometry of one simulation: (SX-1) x (SY-1) node columns per
// tile, tz_len levels. tz_len trades z-halo work (3 extra levels per tile)
// against the number of tiles. It depends on the simulation's own mesh only
// (about kTileNodes output nodes per tile, at least 8 levels), so the tiles,
// and with them the order of every reduction, are the same whether the
// simulation runs alone or in a batch: its results are bitwise identical.
constexpr long long kTileNodes = 2048;
static void tile_geometry(SimDev& d, const KernelSet& ks) {
  d.ntx = (d.nx + 1 + ks.sx - 2) / (ks.sx - 1);
  d.nty = (d.ny + 1 + ks.sy - 2) / (ks.sy - 1);
  const int levels = d.nz + 1;
  const long long cols = (long long)d.ntx * d.nty;
  const long long want = std::max(1LL, d.nn / kTileNodes);
  int ntz = (int)std::max(1LL, std::min<long long>(levels, (want + cols - 1) / cols));
  ntz = std::min(ntz, std::max(1, levels / 8));
  d.tz_len = (levels + ntz - 1) / ntz;
  d.ntz = (levels + d.tz_len - 1) / d.tz_len;
  d.ntiles = d.ntx * d.nty * d.ntz;
  d.npw = (int)((d.nn + ks.pw_chunk - 1) / ks.pw_chunk);
  d.w_ntx = d.w_nty = d.w_ntz = d.w_tz = d.w_ntiles = d.w_items = 0;
  if (ks.apply_w) {
    // segment tiles of about seg output nodes, at least 4 levels (2 extra levels per tile)
    const int seg = ks.seg_nodes[size_bucket(d.nn)];
    d.w_ntx = (d.nx + 1 + ks.wsx - 3) / (ks.wsx - 2);
    d.w_nty = (d.ny + 1 + ks.wny - 1) / ks.wny;
    const int tz0 = std::max(4, std::min(levels, seg / ((ks.wsx - 2) * ks.wny)));
    d.w_ntz = (levels + tz0 - 1) / tz0;
    d.w_tz = (levels + d.w_ntz - 1) / d.w_ntz;
    d.w_ntiles = d.w_ntx * d.w_nty * d.w_ntz;
    const int spc = ks.wwarps * (32 / ks.wsx);
    d.w_items = (d.w_ntiles + spc - 1) / spc;
  }
  d.o_ntx = d.o_nty = d.o_ntz = d.o_tz = d.o_ntiles = d.o_items = 0;
  if (ks.open_w) {
    // about kOpenSegNodes output nodes per segment tile, at least 4 levels
    constexpr int kOpenSegNodes = 1024;
    d.o_ntx = (d.nx + 1 + ks.owsx - 3) / (ks.owsx - 2);
    d.o_nty = (d.ny + 1 + ks.owny - 1) / ks.owny;
    const long long cols = (long long)d.o_ntx * d.o_nty;
    const int spc = ks.owwarps * (32 / ks.owsx);
    const int tz_def = std::max(4, std::min(levels, kOpenSegNodes / ((ks.owsx - 2) * ks.owny)));
    auto items_for = [&](int tz) { return (cols * ((levels + tz - 1) / tz) + spc - 1) / spc; };
    int tz0 = tz_def;
    // A mesh whose passes fill at least half of the resident blocks in at
    // most two waves takes the tile height in [tz_def / 2, tz_def] whose
    // items fill the waves best (the 100^3 mesh: 404 items of 26 levels on
    // 456 resident blocks instead of 303 of 34). It depends on the mesh and
    // the GPU only, so a simulation's passes stay the same alone and in a batch.
    const long long cap = ks.open_cap, items_def = items_for(tz_def);
    if (cap > 0 && 2 * items_def >= cap && items_def <= 2 * cap) {
      double best = -1.0;
      for (int tz = tz_def; tz >= std::max(4, tz_def / 2); --tz) {
        const long long it = items_for(tz), waves = (it + cap - 1) / cap;
        const double eff = (double)it / (double)(waves * cap);
        if (eff > best + 1e-12) {
          best = eff;
          tz0 = tz;
        }
      }
    }
    d.o_ntz = (levels + tz0 - 1) / tz0;
    d.o_tz = (levels + d.o_ntz - 1) / d.o_ntz;
    d.o_ntiles = d.o_ntx * d.o_nty * d.o_ntz;
    d.o_items = (d.o_ntiles + spc - 1) / spc;
  }
}

static int sm_count() {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

static heat_status engine_upload(Engine* e) {
  e->h_sims.clear();
  e->h_op.clear();
  e->h_pw.clear();
  e->h_aw.clear();
  e->h_ow.clear();
  const int sms = sm_count();
  long long item_base = 0;
  for (size_t i = 0; i < e->sims.size(); ++i) {
    SimDev d = e->sims[i]->dev;
    tile_geometry(d, e->ks);
    d.fused = e->ks.fused ? 1 : 0;
    d.partial = e->d_partial + 4 * item_base;
    item_base += std::max(std::max(std::max(d.ntiles, d.npw), d.w_items), d.o_items);
    for (int t = 0; t < d.ntiles; ++t) e->h_op.push_back(make_int2((int)i, t));
    for (int t = 0; t < d.npw; ++t) e->h_pw.push_back(make_int2((int)i, t));
    for (int t = 0; t < d.w_items; ++t) e->h_aw.push_back(make_int2((int)i, t));
    for (int t = 0; t < d.o_items; ++t) e->h_ow.push_back(make_int2((int)i, t));
    e->h_sims.push_back(d);
  }
  if ((long long)e->h_op.size() > e->cap_op || (long long)e->h_pw.size() > e->cap_pw ||
      (long long)e->h_aw.size() > e->cap_aw || (long long)e->h_ow.size() > e->cap_ow ||
      item_base > e->cap_partial)
    return set_error(HEAT_ERR_ARG, "engine: work lists exceed their capacity");
  const int nwork[4] = {(int)e->h_op.size(), (int)e->h_pw.size(), (int)e->h_aw.size(), (int)e->h_ow.size()};
  CUDA_TRY(cudaMemcpyAsync(e->d_sims, e->h_sims.data(), sizeof(SimDev) * e->h_sims.size(), cudaMemcpyHostToDevice,
                           e->stream));
  CUDA_TRY(cudaMemcpyAsync(e->d_work_op, e->h_op.data(), sizeof(int2) * e->h_op.size(), cudaMemcpyHostToDevice,
                           e->stream));
  CUDA_TRY(cudaMemcpyAsync(e->d_work_pw, e->h_pw.data(), sizeof(int2) * e->h_pw.size(), cudaMemcpyHostToDevice,
                           e->stream));
  if (!e->h_aw.empty())
    CUDA_TRY(cudaMemcpyAsync(e->d_work_aw, e->h_aw.data(), sizeof(int2) * e->h_aw.size(), cudaMemcpyHostToDevice,
                             e->stream));
  if (!e->h_ow.empty())
    CUDA_TRY(cudaMemcpyAsync(e->d_work_ow, e->h_ow.data(), sizeof(int2) * e->h_ow.size(), cudaMemcpyHostToDevice,
                             e->stream));
  CUDA_TRY(cudaMemcpyAsync(e->d_nwork, nwork, sizeof(nwork), cudaMemcpyHostToDevice, e->stream));
  CUDA_TRY(cudaStreamSynchronize(e->stream));
  int occ_op = 1, occ_pw = 1, occ_aw = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_op, e->ks.apply, e->ks.apply_threads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_pw, e->ks.update, kPwThreads, 0);
  if (e->ks.apply_w)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_aw, e->ks.apply_w, 32 * e->ks.wwarps, e->ks.apply_w_smem);
  int occ_ch = 1;
  if (e->ks.cheb_w)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_ch, e->ks.cheb_w, 32 * e->ks.wwarps, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_ch, e->ks.cheb, e->ks.apply_threads, 0);
  int occ_ow = 1;
  if (e->ks.open_w)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_ow, e->ks.open_w, 32 * e->ks.owwarps, 0);
  if (e->ks.loop) {
    // every block resident at once (the launch is cooperative)
    int occ_loop = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_loop, (const void*)e->ks.loop, 32 * e->ks.wwarps, 0);
    if (occ_loop < 1) return set_error(HEAT_ERR_CUDA, "engine: the persistent iteration kernel does not fit an SM");
    e->grid_loop = sms * occ_loop;
  }
  // With grid_cap the grids cover the capacities, so a later member set that
  // fits them runs under the same captured graph (surplus blocks find no item).
  const long long items[4] = {e->grid_cap ? e->cap_op : nwork[0], e->grid_cap ? e->cap_pw : nwork[1],
                              e->grid_cap ? e->cap_aw : nwork[2], e->grid_cap ? e->cap_ow : nwork[3]};
  e->grid_ow = (int)std::max(1LL, std::min<long long>(items[3], (long long)sms * std::max(1, occ_ow)));
  e->grid_op = (int)std::max(1LL, std::min<long long>(items[0], (long long)sms * std::max(1, occ_op)));
  e->grid_pw = (int)std::max(1LL, std::min<long long>(items[1], (long long)sms * std::max(1, occ_pw)));
  e->grid_aw = (int)std::max(1LL, std::min<long long>(items[2], (long long)sms * std::max(1, occ_aw)));
  e->grid_ch = (int)std::max(1LL, std::min<long long>(e->ks.cheb_w ? items[2] : items[0],
                                                      (long long)sms * std::max(1, occ_ch)));
  return HEAT_OK;
}

// The apply kernel of an iteration and its launch shape / work list.
static void apply_launch(const Engine* e, TileFn* fn, int* grid, int* threads, const int2** work,
                         const int** nwork, int* smem) {
  *smem = 0;
  if (e->ks.apply_w) {
    *smem = e->ks.apply_w_smem;
    *fn = e->ks.apply_w;
    *grid = e->grid_aw;
    *threads = 32 * e->ks.wwarps;
    *work = e->d_work_aw;
    *nwork = e->d_nwork + 2;
  } else {
    *fn = e->ks.apply;
    *grid = e->grid_op;
    *threads = e->ks.apply_threads;
    *work = e->d_work_op;
    *nwork = e->d_nwork;
  }
}

static heat_status engine_capture(Engine* e) {
  if (e->gexec) {
    cudaGraphExecDestroy(e->gexec);
    e->gexec = nullptr;
  }
  if (e->graph) {
    cudaGraphDestroy(e->graph);
    e->graph = nullptr;
  }
  // Capture on a private stream (the legacy default stream cannot capture);
  // the instantiated graph is then launched on the engine's stream.
  cudaStream_t cap;
  CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  // Each kernel may launch while its predecessor finishes (programmatic
  // dependent launch); the kernels wait for the predecessor's results with
  // cudaGridDependencySynchronize after their static prologue.
  auto launch = [&](TileFn fn, int grid, int block, const int2* work, const int* nwork, int smem) -> cudaError_t {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = cap;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, (const SimDev*)e->d_sims, work, nwork);
  };
  TileFn afn;
  int agrid, athreads, asmem;
  const int2* awork;
  const int* anwork;
  apply_launch(e, &afn, &agrid, &athreads, &awork, &anwork, &asmem);
  cudaError_t err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (err == cudaSuccess) {
    cudaError_t lerr = e->ks.open_w
                           ? launch(e->ks.open_w, e->grid_ow, 32 * e->ks.owwarps, e->d_work_ow, e->d_nwork + 3, 0)
                           : launch(e->ks.open, e->grid_op, e->ks.open_threads, e->d_work_op, e->d_nwork, 0);
    if (e->ks.loop && lerr == cudaSuccess) {
      // one persistent launch for the tick's iterations: cooperative (all
      // blocks resident, which its grid barriers need), no early start
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(e->grid_loop);
      cfg.blockDim = dim3(32 * e->ks.wwarps);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = cap;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeCooperative;
      attr[0].val.cooperative = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      lerr = cudaLaunchKernelEx(&cfg, e->ks.loop, (const SimDev*)e->d_sims, (const int2*)e->d_work_aw,
                                (const int2*)e->d_work_pw, (const int*)e->d_nwork, e->d_sync);
    }
    for (int it = 0; it < (e->ks.loop ? 0 : e->iters_per_tick) && lerr == cudaSuccess; ++it) {
      for (int k = 0; k < e->ncheb && lerr == cudaSuccess; ++k) {
        if (e->ks.cheb_w) lerr = launch(e->ks.cheb_w, e->grid_ch, 32 * e->ks.wwarps, e->d_work_aw, e->d_nwork + 2, 0);
        else lerr = launch(e->ks.cheb, e->grid_ch, e->ks.apply_threads, e->d_work_op, e->d_nwork, 0);
      }
      if (lerr != cudaSuccess) break;
      lerr = launch(afn, agrid, athreads, awork, anwork, asmem);
      if (lerr == cudaSuccess && !e->ks.fused)
        lerr = launch(e->ks.update, e->grid_pw, kPwThreads, e->d_work_pw, e->d_nwork + 1, 0);
    }
    err = cudaStreamEndCapture(cap, &e->graph);
    if (err == cudaSuccess && lerr != cudaSuccess) err = lerr;
  }
  cudaStreamDestroy(cap);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return set_error(HEAT_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(err));
  }
  CUDA_TRY(cudaGraphInstantiate(&e->gexec, e->graph, 0));
  return HEAT_OK;
}

heat_status engine_create(heat_sim* const* sims, int nsims, int precision, cudaStream_t stream, Engine** out,
                          const Tuning* tun, double headroom) {
  *out = nullptr;
  if (nsims < 1 || !sims) return set_error(HEAT_ERR_ARG, "engine: no simulations");
  if (injected_failure()) return set_error(HEAT_ERR_NOMEM, "engine: build failure injected by the test hook");
  if (!(headroom >= 1.0) || headroom > 64.0) return set_error(HEAT_ERR_ARG, "engine: headroom must be in [1, 64]");
  Engine* e = new Engine();
  e->sims.assign(sims, sims + nsims);
  e->prec = precision;
  e->elem = sims[0]->dev.elem;
  for (int i = 1; i < nsims; ++i)
    if (sims[i]->dev.elem != e->elem) {
      delete e;
      return set_error(HEAT_ERR_ARG, "engine: the simulations of one batch must share the element type");
    }
  e->ncheb = members_ncheb(e);
  e->ks = kernel_set(precision, tun ? *tun : tuning_get(), e->ncheb > 0, e->elem);
  e->stream = stream;
  // capacities: the geometry is a function of each mesh, so compute it
  long long cap_op = 0, cap_pw = 0, cap_aw = 0, cap_ow = 0, cap_partial = 0;
  for (heat_sim* s : e->sims) {
    SimDev d = s->dev;
    tile_geometry(d, e->ks);
    cap_op += d.ntiles;
    cap_pw += d.npw;
    cap_aw += d.w_items;
    cap_ow += d.o_items;
    cap_partial += std::max(std::max(std::max(d.ntiles, d.npw), d.w_items), d.o_items);
  }
  if (cap_op > (1LL << 30) || cap_pw > (1LL << 30) || cap_aw > (1LL << 30) || cap_ow > (1LL << 30)) {
    delete e;
    return set_error(HEAT_ERR_ARG, "engine: too many work items");
  }
  auto grow = [&](long long c) { return (long long)std::ceil((double)c * headroom); };
  e->cap_sims = grow(nsims);
  e->grid_cap = headroom > 1.0;
  cap_op = grow(cap_op);
  cap_pw = grow(cap_pw);
  cap_aw = grow(cap_aw);
  cap_ow = grow(cap_ow);
  cap_partial = grow(cap_partial);
  e->cap_op = cap_op;
  e->cap_pw = cap_pw;
  e->cap_aw = cap_aw;
  e->cap_ow = cap_ow;
  e->cap_partial = cap_partial;
  heat_status st = HEAT_OK;
  auto fail = [&](heat_status s) {
    engine_destroy(e);
    return s;
  };
  if (cudaMalloc(&e->d_sims, sizeof(SimDev) * e->cap_sims) != cudaSuccess ||
      cudaMalloc(&e->d_work_op, sizeof(int2) * cap_op) != cudaSuccess ||
      cudaMalloc(&e->d_work_pw, sizeof(int2) * cap_pw) != cudaSuccess ||
      cudaMalloc(&e->d_work_aw, sizeof(int2) * std::max(1LL, cap_aw)) != cudaSuccess ||
      cudaMalloc(&e->d_work_ow, sizeof(int2) * std::max(1LL, cap_ow)) != cudaSuccess ||
      cudaMalloc(&e->d_nwork, sizeof(int) * 4) != cudaSuccess ||
      cudaMalloc(&e->d_unfinished, 2 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&e->d_partial, sizeof(double) * 4 * cap_partial) != cudaSuccess ||
      cudaMallocHost(&e->h_unfinished, 2 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&e->d_sync, sizeof(GridSync)) != cudaSuccess ||
      cudaMallocHost(&e->h_abort, 2 * sizeof(int)) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->poll_ev[0], cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&e->poll_ev[1], cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return fail(set_error(HEAT_ERR_NOMEM, "engine: device allocation failed"));
  }
  // the per-sim counters used by the last-block reductions start at zero
  for (heat_sim* s : e->sims) {
    st = sim_read_scalars(s);
    if (st != HEAT_OK) return fail(st);
    s->h_sc->count = 0;
    st = sim_write_scalars(s);
    if (st != HEAT_OK) return fail(st);
  }
  st = engine_upload(e);
  if (st != HEAT_OK) return fail(st);
  e->h_abort[0] = e->h_abort[1] = 0;
  st = loop_sync_reset(e);
  if (st != HEAT_OK) return fail(st);
  st = engine_capture(e);
  if (st != HEAT_OK) return fail(st);
  *out = e;
  return HEAT_OK;
}

void engine_destroy(Engine* e) {
  if (!e) return;
  cudaStreamSynchronize(e->stream);
  if (e->gexec) cudaGraphExecDestroy(e->gexec);
  if (e->graph) cudaGraphDestroy(e->graph);
  cudaFree(e->d_sims);
  cudaFree(e->d_work_op);
  cudaFree(e->d_work_pw);
  cudaFree(e->d_work_aw);
  cudaFree(e->d_work_ow);
  cudaFree(e->d_nwork);
  cudaFree(e->d_unfinished);
  cudaFree(e->d_partial);
  if (e->d_sync) cudaFree(e->d_sync);
  if (e->h_abort) cudaFreeHost(e->h_abort);
  if (e->h_unfinished) cudaFreeHost(e->h_unfinished);
  for (cudaEvent_t ev : e->poll_ev)
    if (ev) cudaEventDestroy(ev);
  if (e->d_phases) cudaFree(e->d_phases);
  if (e->h_phases) cudaFreeHost(e->h_phases);
  delete e;
}

heat_status engine_refresh(Engine* e) {
  const int g_op = e->grid_op, g_pw = e->grid_pw, g_aw = e->grid_aw, g_ch = e->grid_ch;
  // a member's preconditioner may have changed: the passes per iteration, and
  // with them the kernel set (no fused iteration with passes) and the graph
  const int nch = members_ncheb(e);
  const bool recapture = nch != e->ncheb;
  for (const heat_sim* s : e->sims)
    if (s->dev.elem != e->elem) return set_error(HEAT_ERR_ARG, "engine: a member changed its element type");
  if ((nch > 0) != (e->ncheb > 0)) {
    const KernelSet ks = kernel_set(e->prec, tuning_get(), nch > 0, e->elem);
    bool same_shape = ks.wsx == e->ks.wsx && ks.wny == e->ks.wny && ks.wwarps == e->ks.wwarps &&
                      ks.pw_chunk == e->ks.pw_chunk && (ks.apply_w != nullptr) == (e->ks.apply_w != nullptr);
    for (int b = 0; b < 3; ++b) same_shape = same_shape && ks.seg_nodes[b] == e->ks.seg_nodes[b];
    if (!same_shape)  // the work lists were sized for the old shape
      return set_error(HEAT_ERR_ARG, "engine: the tuning table changed since the engine was built; rebuild it");
    e->ks = ks;
  }
  e->ncheb = nch;
  heat_status st = engine_upload(e);
  if (st != HEAT_OK) return st;
  st = loop_sync_reset(e);
  if (st != HEAT_OK) return st;
  if (recapture || !e->gexec || e->grid_op != g_op || e->grid_pw != g_pw || e->grid_aw != g_aw || e->grid_ch != g_ch)
    return engine_capture(e);
  return HEAT_OK;
}

heat_status engine_set_members(Engine* e, heat_sim* const* sims, int nsims) {
  if (injected_failure()) return set_error(HEAT_ERR_NOMEM, "engine: update failure injected by the test hook");
  if (nsims < 1 || !sims || nsims > e->cap_sims) return set_error(HEAT_ERR_ARG, "engine: member set exceeds capacity");
  long long op = 0, pw = 0, aw = 0, ow = 0, part = 0;
  for (int i = 0; i < nsims; ++i) {
    const heat_sim* s = sims[i];
    if (s->prm.precision != e->prec || s->dev.elem != e->elem)
      return set_error(HEAT_ERR_ARG, "engine: a member's precision or element differs from the engine's");
    SimDev d = s->dev;
    tile_geometry(d, e->ks);
    op += d.ntiles;
    pw += d.npw;
    aw += d.w_items;
    ow += d.o_items;
    part += std::max(std::max(std::max(d.ntiles, d.npw), d.w_items), d.o_items);
  }
  if (op > e->cap_op || pw > e->cap_pw || aw > e->cap_aw || ow > e->cap_ow || part > e->cap_partial)
    return set_error(HEAT_ERR_ARG, "engine: member set exceeds the work-list capacity");
  // the last-block counters of newly added members start at zero
  for (int i = 0; i < nsims; ++i) {
    heat_sim* s = sims[i];
    if (std::find(e->sims.begin(), e->sims.end(), s) != e->sims.end()) continue;
    heat_status st = sim_read_scalars(s);
    if (st != HEAT_OK) return st;
    s->h_sc->count = 0;
    st = sim_write_scalars(s);
    if (st != HEAT_OK) return st;
  }
  e->sims.assign(sims, sims + nsims);
  return engine_refresh(e);
}

heat_status engine_step_all(Engine* e, int nsteps, heat_step_stats* stats, int reset_counters) {
  int max_iter = 1, max_outer = 1, poll = 32;
  if (e->ks.loop) {  // the barrier bound and the test hook as they are now
    heat_status st = loop_sync_reset(e);
    if (st != HEAT_OK) return st;
  }
  for (heat_sim* s : e->sims) {
    CUDA_TRY(cudaStreamSynchronize(s->stream));
    heat_status st = sim_read_scalars(s);
    if (st != HEAT_OK) return st;
    SimScalars* sc = s->h_sc;
    sc->target = sc->step + nsteps;
    sc->phase = PH_OPEN;
    sc->status = ST_OK;
    sc->count = 0;
    if (reset_counters) {
      sc->iters_total = 0;
      sc->outer_total = 0;
      sc->steps_total = 0;
      sc->max_iters_step = 0;
    }
    st = sim_write_scalars(s);
    if (st != HEAT_OK) return st;
    max_iter = std::max(max_iter, s->prm.max_iter);
    max_outer = std::max(max_outer, s->prm.max_outer);
    poll = std::min(poll, s->prm.poll_period);
  }
  // the persistent form polls after as many graph launches as the tick form
  const int ticks_per_poll = std::max(1, poll / e->iters_per_tick);
  // Every tick advances each unfinished simulation by at least one CG
  // iteration or one phase change, so this bound is never reached by a
  // healthy solve; it turns a logic error into HEAT_ERR_TIMEOUT.
  const long long max_ticks = (long long)nsteps * (max_iter + 2LL * max_outer + 4) + 64;
  long long ticks = 0;
  e->launches = 0;
  // Batch b of ticks_per_poll ticks ends with a count of the unfinished
  // members (and the persistent loop's abort flag) copied to slot b & 1 and
  // an event. The first batch is waited for at once (a short call leaves no
  // idle ticks behind); from then on batch b is queued before the host waits
  // for batch b - 1, so the GPU does not idle while the host polls. At most
  // one batch of idle ticks runs after the last member finishes.
  for (long long b = 0;; ++b) {
    const int slot = (int)(b & 1);
    for (int t = 0; t < ticks_per_poll; ++t) CUDA_TRY(cudaGraphLaunch(e->gexec, e->stream));
    ticks += ticks_per_poll;
    e->launches += (long long)ticks_per_poll * tick_launches(e) + 1;
    k_count_unfinished<<<1, 256, 0, e->stream>>>(e->d_sims, (int)e->sims.size(), e->d_unfinished + slot);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(e->h_unfinished + slot, e->d_unfinished + slot, sizeof(int), cudaMemcpyDeviceToHost,
                             e->stream));
    if (e->ks.loop)
      CUDA_TRY(cudaMemcpyAsync(e->h_abort + slot, &e->d_sync->abort, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    CUDA_TRY(cudaEventRecord(e->poll_ev[slot], e->stream));
    long long waited = -1;  // the batch whose counts are read now
    if (b == 0) waited = 0;
    else if (b >= 2) waited = b - 1;
    if (waited < 0) continue;  // batch 1 queued right after batch 0 was read
    const int ws = (int)(waited & 1);
    CUDA_TRY(cudaEventSynchronize(e->poll_ev[ws]));
    if (e->ks.loop && e->h_abort[ws]) {
      CUDA_TRY(cudaStreamSynchronize(e->stream));
      heat_status st = loop_abort(e);
      if (st != HEAT_OK) return st;
      break;
    }
    if (e->h_unfinished[ws] == 0) break;
    if (ticks > max_ticks) {
      cudaStreamSynchronize(e->stream);
      return set_error(HEAT_ERR_TIMEOUT, "engine: solve did not finish within %lld ticks", ticks);
    }
  }
  heat_status first_bad = HEAT_OK;
  for (size_t i = 0; i < e->sims.size(); ++i) {
    heat_sim* s = e->sims[i];
    CUDA_TRY(cudaMemcpyAsync(s->h_sc, s->d_sc, sizeof(SimScalars), cudaMemcpyDeviceToHost, e->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(e->stream));
  for (size_t i = 0; i < e->sims.size(); ++i) {
    const SimScalars* sc = e->sims[i]->h_sc;
    if (stats) {
      heat_step_stats& o = stats[i];
      o.steps = (int)sc->steps_total;
      o.status = sc->phase == PH_FAILED ? sc->status : HEAT_OK;
      o.iters = sc->iters_total;
      o.outer = sc->outer_total;
      o.max_iters_step = sc->max_iters_step;
      o.last_rel_residual = sc->rel_res;
      o.kernel_launches = e->launches;
    }
    if (sc->phase == PH_FAILED && first_bad == HEAT_OK) {
      first_bad = (heat_status)sc->status;
      set_error(first_bad, "simulation %zu failed at step %d: %s", i, sc->step + 1,
                heat_status_string((heat_status)sc->status));
    }
  }
  return first_bad;
}

__global__ void k_gather_phases(const SimDev* __restrict__ sims, int nsims, int* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nsims; i += gridDim.x * blockDim.x)
    out[i] = *(volatile const int*)&sims[i].sc->phase;
}

heat_status engine_launch_ticks(Engine* e, int nticks) {
  for (int t = 0; t < nticks; ++t) CUDA_TRY(cudaGraphLaunch(e->gexec, e->stream));
  e->launches += (long long)nticks * tick_launches(e);
  return HEAT_OK;
}

heat_status engine_read_phases(Engine* e, int* phases) {
  const int n = (int)e->sims.size();
  int* d = nullptr;
  if (!e->d_phases || e->phases_cap < n) {  // grown on first use
    if (e->d_phases) cudaFree(e->d_phases);
    if (e->h_phases) cudaFreeHost(e->h_phases);
    e->d_phases = nullptr;
    e->h_phases = nullptr;
    CUDA_TRY(cudaMalloc(&e->d_phases, sizeof(int) * n));
    CUDA_TRY(cudaMallocHost(&e->h_phases, sizeof(int) * n));
    e->phases_cap = n;
  }
  d = e->d_phases;
  if (e->ks.loop) {  // a persistent launch that gave up fails the unfinished members first
    CUDA_TRY(cudaMemcpyAsync(e->h_abort, &e->d_sync->abort, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
    CUDA_TRY(cudaStreamSynchronize(e->stream));
    if (*e->h_abort) {
      heat_status st = loop_abort(e);
      if (st != HEAT_OK) return st;
    }
  }
  k_gather_phases<<<(n + 255) / 256, 256, 0, e->stream>>>(e->d_sims, n, d);
  CUDA_TRY(cudaGetLastError());
  e->launches += 1;
  CUDA_TRY(cudaMemcpyAsync(e->h_phases, d, sizeof(int) * n, cudaMemcpyDeviceToHost, e->stream));
  CUDA_TRY(cudaStreamSynchronize(e->stream));
  std::memcpy(phases, e->h_phases, sizeof(int) * n);
  return HEAT_OK;
}

long long engine_launches(const Engine* e) { return e->launches; }

size_t engine_footprint(long long nn, long long nx, long long ny, long long nz) {
  // the largest work lists any precision's kernels need under the current table
  const Tuning t = tuning_get();
  long long op = 0, pw = 0, aw = 0, ow = 0;
  for (int p = 0; p < 3; ++p) {
    SimDev d{};
    d.nx = (int)nx;
    d.ny = (int)ny;
    d.nz = (int)nz;
    d.nn = nn;
    tile_geometry(d, kernel_set(p, t));
    op = std::max<long long>(op, d.ntiles);
    pw = std::max<long long>(pw, d.npw);
    aw = std::max<long long>(aw, d.w_items);
    ow = std::max<long long>(ow, d.o_items);
  }
  return (size_t)(sizeof(int2) * (op + pw + aw + ow) +
                  sizeof(double) * 4 * std::max(std::max(std::max(op, pw), aw), ow) + sizeof(SimDev) + 64);
}

// Reads a buffer larger than L2 so the next kernel starts cold. Reading (not
// writing) leaves clean lines, so no write-back lands in the timed kernel.
__global__ void k_flush_read(const uint4* __restrict__ p, size_t n, unsigned int* sink) {
  unsigned int acc = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const uint4 v = __ldcg(p + i);
    acc ^= v.x ^ v.y ^ v.z ^ v.w;
  }
  if (acc == 0x9e3779b9u) *sink = acc;  // keeps the loads alive; practically never taken
}

// r[i] = a hash of i mapped to [-1, 1); *delta += sum r[i]^2 pinv[i].
template <class T>
__global__ void k_profile_seed(T* __restrict__ r, const T* __restrict__ pinv, long long n, double* delta) {
  double acc = 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned int h = (unsigned int)i * 0x9E3779B1u;
    h ^= h >> 15;
    h *= 0x85EBCA77u;
    h ^= h >> 13;
    const T v = (T)((double)(h >> 8) * (1.0 / 8388608.0) - 1.0);
    r[i] = v;
    acc += (double)v * (double)v * (double)pinv[i];
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(delta, acc);
}

// Puts every member into the middle of an inner solve that cannot converge:
// a seeded, well-scaled residual (pseudo-random entries in [-1, 1)) with
// delta = r^T P^-1 r computed for it, phase ITER, restart. Timed iterations
// are then ordinary CG iterations whatever state the members were left in
// (a converged step leaves a residual near underflow).
static heat_status profile_arm(Engine* e, double* d_delta, std::vector<double>& h_delta) {
  heat_status st = HEAT_OK;
  if (e->ncheb > 0)
    return set_error(HEAT_ERR_ARG, "profiling and tuning time the Jacobi iteration: set cheb_degree to 0 for them");
  if (cudaMemsetAsync(d_delta, 0, sizeof(double) * e->sims.size(), e->stream) != cudaSuccess)
    return set_error(HEAT_ERR_CUDA, "profile: memset failed");
  for (size_t i = 0; i < e->sims.size(); ++i) {
    heat_sim* s = e->sims[i];
    const int g = (int)std::min<long long>((s->nn + 255) / 256, 4LL * sm_count());
    if (e->prec == P_FP64) {
      k_profile_seed<double><<<g, 256, 0, e->stream>>>(s->dev.r, s->dev.pinv, s->nn, d_delta + i);
    } else {
      st = sim_read_scalars(s);
      if (st != HEAT_OK) return st;
      const int slot = e->ks.fused ? (s->h_sc->cgs & 1) : 0;
      k_profile_seed<float><<<g, 256, 0, e->stream>>>(s->dev.rc32[slot], s->dev.pinv32, s->nn, d_delta + i);
    }
  }
  if (cudaMemcpyAsync(h_delta.data(), d_delta, sizeof(double) * e->sims.size(), cudaMemcpyDeviceToHost,
                      e->stream) != cudaSuccess ||
      cudaStreamSynchronize(e->stream) != cudaSuccess)
    return set_error(HEAT_ERR_CUDA, "profile: residual seeding failed");
  for (size_t i = 0; i < e->sims.size(); ++i) {
    heat_sim* s = e->sims[i];
    st = sim_read_scalars(s);
    if (st != HEAT_OK) return st;
    SimScalars* sc = s->h_sc;
    sc->phase = PH_ITER;
    sc->iter = 1;
    sc->iter_step = 0;
    sc->restart = 1;
    sc->thresh = -1.0;
    sc->thresh_in = -1.0;
    sc->count = 0;
    sc->delta = h_delta[i] > 0.0 ? h_delta[i] : 1.0;
    st = sim_write_scalars(s);
    if (st != HEAT_OK) return st;
  }
  return HEAT_OK;
}

static heat_status profile_check(Engine* e) {
  if (e->ks.loop) {
    CUDA_TRY(cudaMemcpy(e->h_abort, &e->d_sync->abort, sizeof(int), cudaMemcpyDeviceToHost));
    if (*e->h_abort) {
      heat_status st = loop_abort(e);
      return st != HEAT_OK ? st : set_error(HEAT_ERR_TIMEOUT, "profile: a persistent iteration's wait ran out");
    }
  }
  for (heat_sim* s : e->sims) {
    heat_status st = sim_read_scalars(s);
    if (st != HEAT_OK) return st;
    if (s->h_sc->phase != PH_ITER)
      return set_error(HEAT_ERR_BREAKDOWN, "profile: the iteration left PH_ITER (status %d)", s->h_sc->status);
  }
  return HEAT_OK;
}

heat_status engine_profile(Engine* e, int reps, void* flush, size_t flush_bytes, double* ms_apply,
                           double* ms_update, double* bytes_apply, double* bytes_update) {
  const int chunk = 40;  // below the inner-solve cap and the true-residual period
  cudaEvent_t ev[4 * chunk];
  for (int i = 0; i < 4 * chunk; ++i) CUDA_TRY(cudaEventCreate(&ev[i]));
  double ta = 0.0, tu = 0.0;
  heat_status st = HEAT_OK;
  double* d_delta = nullptr;
  std::vector<double> h_delta(e->sims.size(), 0.0);
  if (cudaMalloc(&d_delta, sizeof(double) * e->sims.size()) != cudaSuccess) {
    cudaGetLastError();
    st = set_error(HEAT_ERR_NOMEM, "profile: no room for the residual norms");
  }
  for (int done = 0; done < reps && st == HEAT_OK;) {
    const int c = std::min(reps - done, chunk);
    st = profile_arm(e, d_delta, h_delta);
    if (st != HEAT_OK) break;
    for (int i = 0; i < c; ++i) {
      if (flush) k_flush_read<<<sm_count() * 4, 256, 0, e->stream>>>((const uint4*)flush, flush_bytes / 16, (unsigned int*)e->d_unfinished);
      cudaEventRecord(ev[4 * i + 0], e->stream);
      {
        TileFn afn;
        int agrid, athreads, asmem;
        const int2* awork;
        const int* anwork;
        apply_launch(e, &afn, &agrid, &athreads, &awork, &anwork, &asmem);
        afn<<<agrid, athreads, asmem, e->stream>>>(e->d_sims, awork, anwork);
      }
      cudaEventRecord(ev[4 * i + 1], e->stream);
      if (flush && !e->ks.fused) k_flush_read<<<sm_count() * 4, 256, 0, e->stream>>>((const uint4*)flush, flush_bytes / 16, (unsigned int*)e->d_unfinished);
      cudaEventRecord(ev[4 * i + 2], e->stream);
      if (!e->ks.fused) e->ks.update<<<e->grid_pw, kPwThreads, 0, e->stream>>>(e->d_sims, e->d_work_pw, e->d_nwork + 1);
      cudaEventRecord(ev[4 * i + 3], e->stream);
    }
    if (cudaStreamSynchronize(e->stream) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      st = set_error(HEAT_ERR_CUDA, "profile: launch failed");
      break;
    }
    for (int i = 0; i < c; ++i) {
      float a = 0.f, u = 0.f;
      cudaEventElapsedTime(&a, ev[4 * i + 0], ev[4 * i + 1]);
      if (!e->ks.fused) cudaEventElapsedTime(&u, ev[4 * i + 2], ev[4 * i + 3]);
      ta += a;
      tu += u;
    }
    st = profile_check(e);
    done += c;
  }
  for (int i = 0; i < 4 * chunk; ++i) cudaEventDestroy(ev[i]);
  cudaStreamSynchronize(e->stream);
  cudaFree(d_delta);
  if (st != HEAT_OK) return st;
  *ms_apply = ta / reps;
  *ms_update = tu / reps;
  // algorithmic bytes: every vector and coefficient touched once per launch
  double ba = 0.0, bu = 0.0;
  for (heat_sim* x : e->sims) {
    const double n = (double)x->nn, ne = (double)x->ne;
    if (e->prec == P_FP64) {
      ba += n * (3 * 8 + 2 * 8) + ne * 16;    // r, P^-1, d_old in; d, q out; (rho_c, k)
      bu += n * (2 * 8 + 8 + 2 * 8 + 8 + 8);  // x in/out, d, r in/out, q, P^-1
    } else if (e->ks.fused) {
      ba += n * (6 * 4 + 5 * 4) + ne * 8;  // r, w, s, P^-1, p, e in; r', s', w', p, e out; (rho_c, k)
    } else {
      ba += n * (3 * 4 + 2 * 4) + ne * 8;
      bu += n * (2 * 4 + 4 + 2 * 4 + 4 + 4);
    }
  }
  *bytes_apply = ba;
  *bytes_update = bu;
  return HEAT_OK;
}

heat_status prime_products(heat_sim* s, int nslots) {
  constexpr int SX = 16, SY = 16, TZ = 8;
  const SimDev& d = s->dev;
  const int ntx = (d.nx + 1 + SX - 2) / (SX - 1), nty = (d.ny + 1 + SY - 2) / (SY - 1);
  const int ntz = (d.nz + 1 + TZ - 1) / TZ;
  const long long grid = (long long)ntx * nty * ntz;
  if (grid > (1LL << 31) - 1) return set_error(HEAT_ERR_ARG, "prime_products: mesh too large");
  for (int v = 0; v < nslots; ++v) {
    if (d.elem == E_P1)
      k_product<SX, SY, E_P1><<<(unsigned)grid, SX * SY, 0, s->stream>>>(s->d_dev, d.vec64[v], d.yv[v], ntx, nty, TZ);
    else
      k_product<SX, SY><<<(unsigned)grid, SX * SY, 0, s->stream>>>(s->d_dev, d.vec64[v], d.yv[v], ntx, nty, TZ);
  }
  CUDA_TRY(cudaGetLastError());
  return HEAT_OK;
}

heat_status engine_time_iterations(Engine* e, int reps, double* ms_per_iter) {
  // 40 iterations per timed chunk: below the inner cap, and on small meshes
  // short of the point where a seeded residual has converged to rounding
  constexpr int kChunk = 40;
  const int per_tick = e->ks.loop ? kChunk : e->iters_per_tick;
  const int chunk_ticks = e->ks.loop ? 1 : std::max(1, kChunk / e->iters_per_tick);
  if (e->ks.loop) {
    heat_status st = loop_sync_reset(e, kChunk);
    if (st != HEAT_OK) return st;
  }
  cudaEvent_t a, b;
  CUDA_TRY(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return set_error(HEAT_ERR_CUDA, "timing: event creation failed");
  }
  heat_status st = HEAT_OK;
  double* d_delta = nullptr;
  std::vector<double> h_delta(e->sims.size(), 0.0);
  if (cudaMalloc(&d_delta, sizeof(double) * e->sims.size()) != cudaSuccess) {
    cudaGetLastError();
    st = set_error(HEAT_ERR_NOMEM, "timing: no room for the residual norms");
  }
  double ms = 0.0;
  long long iters = 0;
  for (int done = 0; done < reps && st == HEAT_OK;) {
    const int ticks = std::min(chunk_ticks, std::max(1, (reps - done + per_tick - 1) / per_tick));
    st = profile_arm(e, d_delta, h_delta);
    if (st != HEAT_OK) break;
    cudaEventRecord(a, e->stream);
    for (int t = 0; t < ticks && st == HEAT_OK; ++t)
      if (cudaGraphLaunch(e->gexec, e->stream) != cudaSuccess) st = set_error(HEAT_ERR_CUDA, "timing: graph launch failed");
    cudaEventRecord(b, e->stream);
    if (cudaEventSynchronize(b) != cudaSuccess) st = set_error(HEAT_ERR_CUDA, "timing: synchronisation failed");
    if (st != HEAT_OK) break;
    float t = 0.f;
    cudaEventElapsedTime(&t, a, b);
    ms += t;
    st = profile_check(e);
    if (st != HEAT_OK) break;
    // iterations actually run (profile_arm cleared iter_step; every member iterates alike)
    const long long n = e->sims[0]->h_sc->iter_step;
    iters += n;
    done += (int)std::max(1LL, n);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(d_delta);
  if (e->ks.loop) {
    const heat_status st2 = loop_sync_reset(e);
    if (st == HEAT_OK) st = st2;
  }
  if (st != HEAT_OK) return st;
  *ms_per_iter = ms / (double)std::max(1LL, iters);
  return HEAT_OK;
}

// Segment sizes (output nodes per warp-segment tile) for table t's warp
// apply of precision prec on these simulations whose work items fill whole
// waves of resident blocks: for each count of waves, the largest levels per
// tile that keep the items within it, kept when the waves are at least 85%
// full; at most four, fewest waves first. Empty for the block-tile apply.
static std::vector<int> wave_segments(heat_sim* const* sims, int nsims, int prec, const Tuning& t, int bucket) {
  std::vector<int> out;
  const KernelSet ks = kernel_set(prec, t, members_ncheb_of(sims, nsims) > 0, sims[0]->dev.elem);
  if (!ks.apply_w) return out;
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, ks.apply_w, 32 * ks.wwarps, ks.apply_w_smem) != cudaSuccess ||
      occ < 1) {
    cudaGetLastError();
    return out;
  }
  const long long cap = (long long)sm_count() * occ;
  const int per_level = (ks.wsx - 2) * ks.wny;
  const int levels = sims[0]->dev.nz + 1;
  long long best_items_for_waves[5] = {0, 0, 0, 0, 0};
  int best_seg_for_waves[5] = {0, 0, 0, 0, 0};
  for (int tz0 = levels; tz0 >= 4; --tz0) {
    const int seg = tz0 * per_level;
    if (seg > (1 << 20)) continue;
    KernelSet k2 = ks;
    k2.seg_nodes[bucket] = seg;
    long long items = 0;
    for (int i = 0; i < nsims; ++i) {
      SimDev d = sims[i]->dev;
      tile_geometry(d, k2);
      items += d.w_items;
    }
    const long long waves = (items + cap - 1) / cap;
    if (waves < 1 || waves > 4) continue;
    if (items > best_items_for_waves[waves]) {  // the fullest last wave, largest tiles on ties
      best_items_for_waves[waves] = items;
      best_seg_for_waves[waves] = seg;
    }
  }
  for (int w = 1; w <= 4; ++w)
    if (best_seg_for_waves[w] && best_items_for_waves[w] >= (long long)(0.85 * (double)(w * cap)))
      out.push_back(best_seg_for_waves[w]);
  return out;
}

heat_status engine_autotune(heat_sim* const* sims, int nsims, int reps, int* best_variant, int* best_seg,
                            double* best_ms) {
  static const int kSegs[] = {256, 512, 1024, 2048};
  const int prec = sims[0]->prm.precision;
  const int bucket = size_bucket(sims[0]->nn);
  const Tuning base = tuning_get();
  Tuning best = base;
  double best_t = 1e300;
  heat_status st = HEAT_OK;
  // each warp variant's best time over the fixed segment sizes
  std::vector<double> vbest(kNumVariants, 1e300);
  for (int v = -1; v < kNumVariants && st == HEAT_OK; ++v) {
    if (v >= 0 && prec == P_FP64 && !kVariants[v].f64[0]) continue;
    for (int si = 0; si < (v < 0 ? 1 : 4) && st == HEAT_OK; ++si) {
      Tuning t = base;
      t.variant[prec] = v;
      if (v >= 0) t.seg_nodes[bucket] = kSegs[si];
      Engine* e = nullptr;
      st = engine_create(sims, nsims, prec, sims[0]->stream, &e, &t);
      if (st != HEAT_OK) break;
      // CG iterations as the solve runs them: the captured tick graph
      double ms = 0.0;
      st = engine_time_iterations(e, 8, &ms);  // warm-up
      if (st == HEAT_OK) st = engine_time_iterations(e, reps, &ms);
      engine_destroy(e);
      if (st == HEAT_OK && v >= 0) vbest[v] = std::min(vbest[v], ms);
      if (st == HEAT_OK && ms < best_t) {
        best_t = ms;
        best = t;
      }
    }
  }
  // then wave-aligned segment sizes for the two fastest warp applies: the levels
  // per segment tile whose total work items fill the resident blocks
  // (SMs x blocks per SM) best, a few waves at most (a launch whose last
  // wave is partly empty leaves SMs idle: on the 100^3 mesh 338 items on
  // 456 resident blocks run three blocks on some SMs and two on the others)
  int top[2] = {-1, -1};
  for (int v = 0; v < kNumVariants; ++v) {
    if (vbest[v] >= 1e300) continue;
    if (top[0] < 0 || vbest[v] < vbest[top[0]]) {
      top[1] = top[0];
      top[0] = v;
    } else if (top[1] < 0 || vbest[v] < vbest[top[1]]) {
      top[1] = v;
    }
  }
  for (int v : top) {
    if (v < 0 || st != HEAT_OK) continue;
    Tuning tv = base;
    tv.variant[prec] = v;
    for (int seg : wave_segments(sims, nsims, prec, tv, bucket)) {
      if (st != HEAT_OK) break;
      bool tried = false;
      for (int k : kSegs) tried = tried || k == seg;
      if (tried) continue;
      Tuning t = tv;
      t.seg_nodes[bucket] = seg;
      Engine* e = nullptr;
      st = engine_create(sims, nsims, prec, sims[0]->stream, &e, &t);
      if (st != HEAT_OK) break;
      double ms = 0.0;
      st = engine_time_iterations(e, 8, &ms);
      if (st == HEAT_OK) st = engine_time_iterations(e, reps, &ms);
      engine_destroy(e);
      if (st == HEAT_OK && ms < best_t) {
        best_t = ms;
        best = t;
      }
    }
  }
  // then the pointwise kernel's item size with the chosen apply
  const Tuning chosen = best;
  for (int qpt : {1, 2, 4}) {
    if (st != HEAT_OK || qpt == chosen.pw_quads[prec]) continue;
    Tuning t = chosen;
    t.pw_quads[prec] = qpt;
    Engine* e = nullptr;
    st = engine_create(sims, nsims, prec, sims[0]->stream, &e, &t);
    if (st != HEAT_OK) break;
    double ms = 0.0;
    st = engine_time_iterations(e, 8, &ms);
    if (st == HEAT_OK) st = engine_time_iterations(e, reps, &ms);
    engine_destroy(e);
    if (st == HEAT_OK && ms < best_t) {
      best_t = ms;
      best = t;
    }
  }
  // then the persistent iteration with each item size (FP32 paths, where
  // the chosen apply has a persistent form)
  const Tuning chosen2 = best;
  for (int qpt : {1, 2, 4}) {
    if (st != HEAT_OK || prec == P_FP64) break;
    Tuning t = chosen2;
    t.loop[prec] = 1;
    t.pw_quads[prec] = qpt;
    if (!kernel_set(prec, t, members_ncheb_of(sims, nsims) > 0, sims[0]->dev.elem).loop) continue;
    Engine* e = nullptr;
    st = engine_create(sims, nsims, prec, sims[0]->stream, &e, &t);
    if (st != HEAT_OK) break;
    double ms = 0.0;
    st = engine_time_iterations(e, 8, &ms);
    if (st == HEAT_OK) st = engine_time_iterations(e, reps, &ms);
    engine_destroy(e);
    if (st == HEAT_OK && ms < best_t) {
      best_t = ms;
      best = t;
    }
  }
  if (st != HEAT_OK) return st;
  st = tuning_set(best);
  if (st != HEAT_OK) return st;
  *best_variant = best.variant[prec];
  *best_seg = best.seg_nodes[bucket];
  *best_ms = best_t;
  return HEAT_OK;
}

}  // namespace heat

extern "C" heat_status heat_debug_loop_wait(unsigned int extra_arrivals, double limit_s) {
  if (extra_arrivals > 1u || !(limit_s >= 0.0) || limit_s > 60.0)
    return heat::set_error(HEAT_ERR_ARG, "heat_debug_loop_wait: need extra_arrivals in {0, 1}, 0 <= limit_s <= 60");
  heat::g_loop_extra.store(extra_arrivals);
  heat::g_loop_limit_ns.store((unsigned long long)(limit_s * 1e9));
  return HEAT_OK;
}

extern "C" heat_status heat_debug_fail_engine_builds(int n) {
  if (n < 0) return heat::set_error(HEAT_ERR_ARG, "heat_debug_fail_engine_builds: n must be >= 0");
  heat::g_fail_builds.store(n);
  return HEAT_OK;
}
