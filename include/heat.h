/*
 * heat.h -- C ABI of the GB300 assembly-free transient heat solver.
 *
 * The library solves the theta-scheme step system of transient heat flow
 * (§3.1), divided by dt:
 *
 *     [M/dt + theta K] U^n = [M/dt - (1 - theta) K] U^{n-1} + F^n,
 *
 * on a structured mesh of nx*ny*nz congruent trilinear (Q1) box elements with
 * per-element coefficients rho*C and k (§3.2, "fixed grid"). M and K are never
 * assembled: every product with A = M/dt + theta K is computed element by
 * element from the closed-form Q1 element matrices (the assembly operator of
 * §3.2 Eq. 1, read degree-of-freedom by degree-of-freedom). Each step is solved
 * by Jacobi-preconditioned conjugate gradients (Algorithm 1, §3.3), entirely on
 * one GPU.
 *
 * Conventions (all entry points):
 *   - element (i,j,k), id = i + nx*(j + ny*k); node (i,j,k), id = i + (nx+1)*(j +
 *     (ny+1)*k): x fastest (§4.1). N = (nx+1)(ny+1)(nz+1) nodes, Ne = nx*ny*nz.
 *   - faces: 0 x=x0, 1 x=x1, 2 y=y0, 3 y=y1, 4 z=z0, 5 z=z1.
 *   - Dirichlet faces are an extension (the paper has flux faces only): their
 *     rows and columns are eliminated symmetrically; a node on several Dirichlet
 *     faces takes the value of the lowest face id.
 *   - "on_device" arguments: 0 = the pointer is host memory, 1 = device memory of
 *     the current CUDA device. Device pointers are read/written on the sim's
 *     stream; host pointers are copied synchronously.
 *   - Every call returns heat_status. On error nothing is half-applied: the sim
 *     keeps its previous state. heat_last_error() gives a thread-local message.
 *   - Ownership: the library owns every device buffer it allocates; input arrays
 *     are copied and stay the caller's; outputs go into caller buffers.
 *   - Threading: one sim per thread (and per stream); the server is locked
 *     internally.
 */
#ifndef HEAT_H
#define HEAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct heat_mesh heat_mesh;
typedef struct heat_sim heat_sim;
typedef struct heat_batch heat_batch;
typedef struct heat_server heat_server;
typedef struct heat_slab heat_slab;

typedef enum {
  HEAT_OK = 0,
  HEAT_ERR_ARG = 1,           /* bad argument (null, size, range, mismatch) */
  HEAT_ERR_NOMEM = 2,         /* device memory or HBM budget exhausted */
  HEAT_ERR_CUDA = 3,          /* a CUDA runtime call failed */
  HEAT_ERR_NOT_CONVERGED = 4, /* max_iter reached; last iterate kept */
  HEAT_ERR_NONFINITE = 5,     /* NaN/Inf in inputs or in a CG scalar */
  HEAT_ERR_TIMEOUT = 6,       /* a bounded wait gave up */
  HEAT_ERR_BUSY = 7,          /* no free slot / ticket not finished */
  HEAT_ERR_BREAKDOWN = 8      /* CG breakdown: d^T A d <= 0 */
} heat_status;

typedef enum {
  HEAT_FP64 = 0,         /* operator, vectors and dots in FP64 */
  HEAT_FP32_REFINED = 1, /* FP32 operator/vectors, FP64 dots; outer refinement
                            on FP64 vectors, its residual operator in
                            double-float (pairs of floats, ~48 bits) */
  HEAT_FP32_PLAIN = 2    /* FP32 operator/vectors, FP64 dots, no refinement */
} heat_precision;

/* Solver parameters. heat_params_default() fills the defaults in brackets. */
typedef struct {
  double theta;      /* theta of the theta-scheme, 0 < theta <= 1   [0.5] (§3.1) */
  double dt;         /* time step, > 0                              [1e-3] */
  double rtol;       /* stop when r^T P^-1 r <= rtol^2 b^T P^-1 b   [1e-10] */
  int max_iter;      /* CG iterations per step (all kinds), >= 1     [20000] */
  int resid_period;  /* true residual r = b - A x every this many
                        iterations (Algorithm 1 uses 50), >= 1       [50] */
  int poll_period;   /* CG iterations queued between host polls      [32] */
  int precision;     /* heat_precision                               [HEAT_FP64] */
  double inner_rtol; /* FP32_REFINED: inner solve tolerance relative
                        to its own right-hand side                   [1e-5] */
  int max_outer;     /* FP32_REFINED: refinement sweeps per step     [40] */
  int inner_max_iter; /* FP32_REFINED: CG iterations per inner solve;
                         a restart loses the Krylov space, so stiff
                         systems want long inner solves, >= 1        [2000] */
  int cheb_degree;   /* preconditioner: 0 or 1 the Jacobi diagonal of
                        Algorithm 1; m in [2, HEAT_CHEB_MAX_DEGREE]
                        the Chebyshev polynomial z = p_m(D^-1 A) D^-1 r
                        (m - 1 extra operator passes per CG iteration,
                        fewer iterations). The stopping test stays
                        r^T P^-1 r of Algorithm 1. The FP32 fused
                        iteration kernels are not used with it.      [0] */
  double cheb_ratio; /* Chebyshev interval [lam_hi / ratio, lam_hi] of
                        D^-1 A, lam_hi an element-wise Gershgorin bound
                        (see heat_cheb_interval), > 1                [10] */
  int element;       /* heat_element: the finite element on each box of
                        the mesh                                     [HEAT_ELEM_Q1] */
} heat_params;

/* Finite elements on the structured box mesh. Coefficients are per box in
 * both cases (the same heat_set_coeffs layout). */
typedef enum {
  HEAT_ELEM_Q1 = 0, /* one trilinear hexahedron per box (§3.2's fixed grid) */
  HEAT_ELEM_P1 = 1  /* six linear tetrahedra per box, all sharing the box
                       diagonal from its lowest to its highest corner (the
                       split of §4.1): for each ordering (a, b, c) of the
                       axes, corners 0, e_a, e_a + e_b, 7. Face loads
                       integrate the linear functions of the boundary
                       triangles. Every kernel variant of the tuning
                       table has a P1 form. */
} heat_element;

#define HEAT_CHEB_MAX_DEGREE 8

/* Boundary conditions (§3.1 strong form: k dT/dn = f on the sides). */
typedef struct {
  uint32_t dirichlet_faces;  /* bit f set: face f has fixed temperature */
  double dirichlet_value[6]; /* value on each Dirichlet face */
  double flux[6];            /* inward heat flux f on each face (ignored on
                                Dirichlet faces); enters F (§3.1) */
  int flux_steps;            /* F^n = F for steps n <= flux_steps, 0 after;
                                < 0: on for every step */
} heat_bc;

/* Per-call statistics. */
typedef struct {
  int steps;                /* time steps completed by the call */
  int status;               /* heat_status of the last step */
  long long iters;          /* CG iterations (inner + outer) over the call */
  long long outer;          /* refinement sweeps over the call (FP32_REFINED) */
  int max_iters_step;       /* most CG iterations in one step */
  double last_rel_residual; /* sqrt(r^T P^-1 r / b^T P^-1 b) at the last exit */
  long long kernel_launches; /* kernels of this library launched by the call */
} heat_step_stats;

void heat_params_default(heat_params* p);

/* Structured mesh on [origin, origin + extent] split into nx*ny*nz boxes
 * (§4.1: domain divisions per dimension). nx, ny, nz >= 1, extent > 0. */
heat_status heat_create_mesh(int nx, int ny, int nz, const double origin[3],
                             const double extent[3], heat_mesh** out);
void heat_destroy_mesh(heat_mesh* mesh);
/* N and Ne of a mesh (either pointer may be NULL). */
heat_status heat_mesh_sizes(const heat_mesh* mesh, long long* n_nodes, long long* n_elems);

/* A simulation on `mesh` (kept by reference: the mesh must outlive the sim).
 * cuda_stream: a cudaStream_t, or NULL for the legacy default stream. The sim
 * starts with rho_c = k = 1 and U^0 = 0 (Dirichlet nodes at their values). */
heat_status heat_sim_create(const heat_mesh* mesh, const heat_bc* bc,
                            const heat_params* params, void* cuda_stream,
                            heat_sim** out);
void heat_destroy_sim(heat_sim* sim);

/* Per-element coefficients rho*C (> 0) and k (> 0), Ne values each, element
 * order (§3.2: constant per element). Rebuilds the Jacobi diagonal and the
 * Dirichlet lift. HEAT_ERR_NONFINITE/ARG on NaN/Inf or non-positive values
 * (checked for host input; device input is checked on the device). */
heat_status heat_set_coeffs(heat_sim* sim, const double* rho_c, const double* k,
                            int on_device);

/* Copy the per-element coefficients out (Ne values each, element order;
 * host or device buffers). Returns after the copy. */
heat_status heat_get_coeffs(heat_sim* sim, double* rho_c, double* k, int on_device);

/* Change dt / theta / tolerances / precision / preconditioner between steps. */
heat_status heat_set_params(heat_sim* sim, const heat_params* params);

/* The interval [lam_lo, lam_hi] of the Chebyshev preconditioner (params
 * cheb_degree >= 2): lam_hi = max over elements e of
 * sum_p |rho_c_e Mhat[p] / dt + theta k_e Khat[p]| / (rho_c_e Mhat[0] / dt +
 * theta k_e Khat[0]), the element-wise Gershgorin bound of the spectrum of
 * D^-1 A (Mhat, Khat: the rows of the Q1 element matrices of §3.2), and
 * lam_lo = lam_hi / cheb_ratio. Recomputed whenever the coefficients or the
 * parameters change. HEAT_ERR_ARG when the preconditioner is off. */
heat_status heat_cheb_interval(heat_sim* sim, double* lam_lo, double* lam_hi);

/* Set the current temperature U (N values, node order) and restart the time
 * history (the next step extrapolates from U alone). Dirichlet nodes are
 * overwritten with their face values. */
heat_status heat_set_state(heat_sim* sim, const double* u, int on_device);
/* Copy the current temperature U^n (N values) out. */
heat_status heat_get_state(heat_sim* sim, double* u, int on_device);

/* Checkpoint / resume. heat_get_history copies U^n and U^{n-1} (N values
 * each; u_prev2 may be NULL) and the number of completed steps n (used by the
 * flux schedule); *have_prev = 0 when U^{n-1} is not defined (no step since the
 * last heat_set_state). heat_set_history restores them (u_prev2 == NULL: no
 * history): a simulation resumed this way continues bitwise identically to
 * one that was never interrupted. Dirichlet nodes are overwritten with their
 * values. */
heat_status heat_get_history(heat_sim* sim, double* u_prev, double* u_prev2, int* step, int* have_prev,
                             int on_device);
heat_status heat_set_history(heat_sim* sim, const double* u_prev, const double* u_prev2, int step,
                             int on_device);

/* Advance nsteps time steps (Algorithm 1 per step, x0 = 2U^{n-1} - U^{n-2}).
 * stats may be NULL. Returns the first failing step's status, if any. */
heat_status heat_step(heat_sim* sim, int nsteps, heat_step_stats* stats);
/* heat_step, then copy U^n to host u_out (may be NULL). */
heat_status heat_solve_transient(heat_sim* sim, int nsteps, double* u_out,
                                 heat_step_stats* stats);
/* Number of completed steps, and the CG iterations of step s (0-based, of the
 * last heat_step call); iters may be NULL. */
heat_status heat_step_iterations(heat_sim* sim, int s, int* iters);

/* ---- batches --------------------------------------------------------------
 * Many independent simulations advanced together (the paper's inverse
 * problem runs thousands of forward solves on one precomputed mesh geometry
 * with varying coefficients, §3.2, §5.3). Every kernel launch of a batch step
 * carries all member simulations: sizes, coefficients, boundary conditions
 * and iteration counts may all differ. Each member's reductions run in the
 * same order as when it is stepped alone, so its results are bitwise
 * identical to heat_step on the same simulation.
 *   sims: nsims >= 1 distinct simulations with the same precision; they stay
 *     owned by the caller and must not be stepped otherwise (or destroyed)
 *     while the batch exists.
 *   cuda_stream: stream of the batch's work (NULL: legacy default stream).
 * heat_batch_step advances every member by nsteps steps; stats (nsims entries,
 * or NULL) receives per-member statistics. It returns the first failing
 * member's status; the other members complete their steps. */
heat_status heat_batch_create(heat_sim* const* sims, int nsims, void* cuda_stream, heat_batch** out);
heat_status heat_batch_step(heat_batch* batch, int nsteps, heat_step_stats* stats);
void heat_destroy_batch(heat_batch* batch);

/* ---- serving --------------------------------------------------------------
 * A request loop for transient simulations that arrive over time (the
 * inverse problem's stream of forward solves, §5.3). A worker thread owns the
 * GPU: it admits pending requests in arrival order while their device
 * footprint fits the HBM budget and a slot is free (first fit: a request that
 * does not fit does not block smaller ones behind it), keeps each admitted
 * simulation resident until its last step, and advances all admitted
 * simulations together in every kernel launch (continuous batching:
 * simulations join and leave between ticks, at any point of the others'
 * solves). A simulation's results do not depend on what it shares the GPU
 * with: they are bitwise identical to heat_step on the same inputs. */
typedef struct {
  int nx, ny, nz;            /* mesh, as heat_create_mesh */
  double origin[3], extent[3];
  const double* rho_c;       /* host, Ne values (copied by heat_submit) */
  const double* k;           /* host, Ne values (copied by heat_submit) */
  const double* u0;          /* host, N values, or NULL for zero (copied) */
  heat_bc bc;
  heat_params params;
  int nsteps;                /* time steps to run, >= 1 */
} heat_request;

typedef struct {
  long long submitted, completed, failed;
  int active, pending;
  size_t hbm_in_use, hbm_budget;  /* bytes of admitted simulations / budget */
  long long kernel_launches;      /* kernels launched by the worker */
  double dof_cg_iters;            /* sum over completed requests of N * CG iterations */
} heat_server_stats;

/* hbm_budget_bytes: device memory the admitted simulations may hold in total;
 * max_active >= 1: simulations admitted at once; cuda_stream: the worker's
 * stream (NULL: the worker creates a non-blocking one). The calling thread's
 * current device is used. */
heat_status heat_server_create(size_t hbm_budget_bytes, int max_active, void* cuda_stream,
                               heat_server** out);
/* Queue a request (inputs are copied; NaN/Inf or non-positive coefficients
 * and requests larger than the whole budget are rejected here). */
heat_status heat_submit(heat_server* srv, const heat_request* req, uint64_t* ticket);
/* *done = 1 once the request finished (successfully or not). */
heat_status heat_poll(heat_server* srv, uint64_t ticket, int* done);
/* Wait up to timeout_s seconds (HEAT_ERR_TIMEOUT after that) for a request;
 * then copy its final state (N values, host; may be NULL), statistics and
 * latency (submit to completion, seconds; may be NULL) and forget the
 * ticket. Returns the request's own status. */
heat_status heat_wait(heat_server* srv, uint64_t ticket, double timeout_s, double* u_out,
                      heat_step_stats* stats, double* latency_s);
heat_status heat_server_get_stats(heat_server* srv, heat_server_stats* out);
/* Stops the worker; requests not yet finished are abandoned. */
void heat_destroy_server(heat_server* srv);
/* Testing hook for the server's recovery (no counterpart in the paper): the
 * next n engine builds or engine membership updates, of any server, batch or
 * simulation in the process, fail with HEAT_ERR_NOMEM before touching the
 * GPU, as a failed device allocation would. When the set a server wants to
 * run cannot be built, the requests admitted in that round are refused with
 * that status and the requests already running continue undisturbed. n = 0
 * clears the hook. */
heat_status heat_debug_fail_engine_builds(int n);
/* Testing hook for the bounded waits of the persistent iteration (tuning
 * loop): engines built or refreshed afterwards expect extra_arrivals (0 or 1)
 * arrivals at each grid barrier beyond their grid, so with 1 no barrier ever
 * completes, and bound one wait by limit_s seconds (0: the engine's own
 * bound of 1 s plus 50 ns per node). A wait that runs out ends the kernel;
 * the step then fails with HEAT_ERR_TIMEOUT and the GPU context stays
 * usable. HEAT_ERR_ARG unless extra_arrivals is 0 or 1 and
 * 0 <= limit_s <= 60. heat_debug_loop_wait(0, 0) restores the defaults. */
heat_status heat_debug_loop_wait(unsigned int extra_arrivals, double limit_s);

/* ---- operator-level entry points (device pointers, sim stream) ---------- */

/* y = A' x with A = M/dt + theta K (§3.2: A = M + theta dt K scaled by 1/dt),
 * A' = A with Dirichlet rows and columns replaced by the identity. FP64. */
heat_status heat_apply(heat_sim* sim, const double* x, double* y);
/* Same operator in FP32 (the refined path's inner operator). */
heat_status heat_apply_f32(heat_sim* sim, const float* x, float* y);
/* General element-wise product y = sum_e A_e^T (sa*rho_c_e*Mhat + sb*k_e*Khat) A_e x
 * without Dirichlet elimination (§3.2 Eq. 1), FP64: (sa, sb) = (1/dt, theta)
 * gives A, (1/dt, theta-1) gives L, (1, 0) gives M, (0, 1) gives K. */
heat_status heat_apply_general(heat_sim* sim, double sa, double sb, const double* x,
                               double* y);
/* Jacobi diagonal P = diag(A') (§3.3; P = 1 on Dirichlet rows), FP64, N values. */
heat_status heat_diagonal(heat_sim* sim, double* p);
/* Right-hand side of step n (1-based) from U^{n-1} = u_prev (§3.1):
 * b = L u_prev + F^n - A_{.D} g on free rows, b = g on Dirichlet rows. FP64. */
heat_status heat_rhs(heat_sim* sim, int n, const double* u_prev, double* b);
/* Face flux vector F (flux on), FP64, N values. */
heat_status heat_flux_vector(heat_sim* sim, double* f);

/* ---- the coefficient inverse problem (§5.3) -------------------------------
 * §5.3 recovers a corrosion depth from surface temperatures: a heat source on
 * the front face, the face's temperature after the heating time compared
 * with noisy camera data, Metropolis-Hastings over the depth. These calls
 * give the pieces on the device and a driver that runs many chains at once,
 * every proposal's forward solve in one batch. */

/* Non-uniform heat flux on one face: q holds one flux density per element
 * face of `face` (0..5 = x=0, x=Lx, y=0, y=Ly, z=0, z=Lz), ordered with the
 * lower tangential index fastest (face x: (j,k), face y: (i,k), face z:
 * (i,j)). It replaces that face's uniform heat_bc flux; each node gets
 * q*area/4 from each adjacent element face (the integral of the bilinear
 * shape function, §3.1). The flux schedule (flux_steps) is unchanged.
 * q = NULL restores the uniform value. Host or device input (copied). */
heat_status heat_set_face_flux(heat_sim* sim, int face, const double* q, int on_device);

/* A corrosion profile of depth `depth` (§5.3, the parabolic boundary of a
 * gusset-plate crevice): seen from the rear face y = origin_y + Ly, the
 * corrosion reaches depth(z) = depth * (1 - ((z - z0) / half_width)^2) for
 * |z - z0| < half_width, and is the same along x. An element whose centroid
 * (x_c, y_c, z_c) has (y_rear - y_c) < depth(z_c) takes the corroded
 * material, every other element the sound one. Centroids and the test are
 * evaluated in FP64 in exactly this operation order, without fused
 * multiply-adds:
 *   z_c = oz + (k + 0.5)*hz, t = (z_c - z0)/half_width, d = depth*(1 - t*t),
 *   y_c = oy + (j + 0.5)*hy, corroded = |t| < 1 and (y_rear - y_c) < d. */
typedef struct {
  double z0, half_width;        /* apex height and half-width of the parabola */
  double rho_c_sound, k_sound;  /* material outside the corrosion, > 0 */
  double rho_c_corr, k_corr;    /* corroded material, > 0 */
} heat_corrosion;
/* Sets the coefficients from the profile on the device (no host round trip);
 * otherwise as heat_set_coeffs. depth >= 0. */
heat_status heat_set_coeffs_corrosion(heat_sim* sim, const heat_corrosion* geom, double depth);

/* Log-likelihood of camera data on one face (§5.3: i.i.d. Gaussian pixel
 * noise): *loglik = -1/2 sum_i ((U_i - data_i) / sigma)^2 over the face's
 * nodes, U the current state. data: device, one value per face node with the
 * lower tangential index fastest ((ny+1)*(nz+1) values for an x face, etc.).
 * loglik: device, one double, written asynchronously on the sim's stream
 * (a fixed-order sum: the same inputs give the same bits). */
heat_status heat_face_loglik(heat_sim* sim, int face, const double* data, double sigma, double* loglik);

/* Metropolis-Hastings over the corrosion depth with nchains chains that
 * advance together; every chain's proposal is solved in one batch.
 *   mesh: nx, ny, nz, origin, extent of the plate; bc: its boundary
 *   conditions; params: the solver parameters; nsteps: time steps of the
 *   heating period, starting from U = u0 (uniform). flux_face / flux_q: the
 *   source as in heat_set_face_flux (host array). obs_face: the observed face;
 *   data: host, one value per face node; sigma: noise std. depth_max: the
 *   uniform prior's upper end (lower end 0). */
typedef struct {
  int nx, ny, nz;
  double origin[3], extent[3];
  heat_bc bc;
  heat_params params;
  int nsteps;
  double u0;
  int flux_face;
  const double* flux_q;
  heat_corrosion geom;
  int obs_face;
  const double* data;
  double sigma;
  double depth_max;
  int nchains;
} heat_mh_config;
typedef struct heat_mh heat_mh;
heat_status heat_mh_create(const heat_mh_config* cfg, void* cuda_stream, heat_mh** out);
void heat_mh_destroy(heat_mh* mh);
/* Log-likelihoods of nchains depths (one forward solve each, all in one
 * batch). depths, loglik: host, nchains values. */
heat_status heat_mh_loglik(heat_mh* mh, const double* depths, double* loglik);
/* niter Metropolis-Hastings steps of every chain from `state` (host, nchains
 * depths; updated in place) with log-likelihoods `state_ll` (host, nchains;
 * NULL: computed first). Random draws are inputs: normals and uniforms hold
 * niter*nchains values (iteration-major). Proposal depth' = depth +
 * step * normal (rounded as a product, then a sum); a proposal outside
 * [0, depth_max] is rejected (its chain's batch slot re-solves the current
 * depth, whose result is discarded); otherwise it is accepted when
 * log(uniform) < ll' - ll. Outputs per
 * iteration and chain (iteration-major, host, may be NULL): the chain's depth
 * and log-likelihood after the step and whether it accepted. */
heat_status heat_mh_run(heat_mh* mh, int niter, double step, const double* normals, const double* uniforms,
                        double* state, double* state_ll, double* depth_trace, double* ll_trace,
                        int* accepted);
/* Forward solves and CG iterations (all kinds, as heat_step_stats.iters) run
 * by the driver so far (either pointer may be NULL). */
heat_status heat_mh_stats(const heat_mh* mh, long long* solves, long long* cg_iters);

/* ---- one simulation split into z-slabs -------------------------------------
 * The partitioned form of the dual-GPU split of §4.4 (Table 1 of §5.2 times
 * it): the element layers of the mesh are cut into nslabs contiguous ranges
 * along z and each slab keeps its own buffers for the node layers it owns plus
 * one ghost node layer per neighbour. Every slab lives on the current GPU.
 * Operator passes of a slab read only its own buffers; the kernels that write
 * a slab's lowest or highest owned layer of a vector an operator pass reads
 * (x, u = P^-1 r, Algorithm 1's d) store those values into the neighbour's
 * ghost layer too (one node layer per interface and vector). Every CG scalar
 * is summed per slab in tile order and then over slabs in slab order.
 * FP64, trilinear boxes, Jacobi preconditioner. Two iteration forms:
 *   merged = 1: the Chronopoulos-Gear form of CG, whose two inner products
 *     (r.P^-1 r and (A u).u) come from one reduction per iteration.
 *   merged = 0: Algorithm 1 (§3.3), two reductions per iteration (d.q and
 *     r.P^-1 r).
 * Both recompute r = b - A x every resid_period iterations, and when the
 * recurrence residual meets the stopping rule; a step closes on that true
 * residual only (as heat_step's FP64 path). The stopping rule,
 * the right-hand side, the initial guess and the Dirichlet and flux handling
 * are those of heat_step (§3.1, Algorithm 1).
 *
 * heat_slab_plan: the partition only (host, no GPU): first_layer[s] for
 *   s = 0..nslabs is the first node layer slab s owns,
 *   floor(s (nz + 1) / nslabs), and first_layer[nslabs] = nz + 1. Slab s owns
 *   node layers [first_layer[s], first_layer[s+1]). Needs
 *   1 <= nslabs <= min(nz + 1, 4096); else HEAT_ERR_ARG. */
heat_status heat_slab_plan(int nz, int nslabs, int* first_layer);
/* mesh, bc: as heat_sim_create. prm: precision HEAT_FP64, element
 * HEAT_ELEM_Q1, cheb_degree < 2 (else HEAT_ERR_ARG); poll_period is the
 * number of iterations queued between host polls. cuda_stream: the stream
 * of every launch and copy (NULL: legacy default stream). The library owns
 * every buffer; heat_slab_info reports their bytes. */
heat_status heat_slab_create(const heat_mesh* mesh, const heat_bc* bc, const heat_params* prm, int nslabs,
                             int merged, void* cuda_stream, heat_slab** out);
/* Host arrays of Ne values each, element order: rho*C > 0 and k > 0, finite
 * (else HEAT_ERR_ARG and nothing changes). Copies each slab's element layers
 * (its owned ones and the layer below its first owned node layer) and
 * derives P^-1, the Dirichlet lift and the face loads. Synchronous. */
heat_status heat_slab_set_coeffs(heat_slab* slab, const double* rho_c, const double* k);
/* Host array of N node values, node order: the state U^0 (Dirichlet nodes
 * take their face values). Resets the step count. Synchronous. */
heat_status heat_slab_set_state(heat_slab* slab, const double* u);
/* Host array of N values: the current state, gathered from the owned layers
 * of every slab. */
heat_status heat_slab_get_state(heat_slab* slab, double* u);
/* Advance nsteps time steps (the host polls the device phase every
 * poll_period iterations). Errors as heat_step: HEAT_ERR_NOT_CONVERGED,
 * HEAT_ERR_NONFINITE or HEAT_ERR_BREAKDOWN leave the state at the last
 * completed step; stats (may be NULL) as heat_step_stats. */
heat_status heat_slab_step(heat_slab* slab, int nsteps, heat_step_stats* stats);
/* CG iterations of each step of the last heat_slab_step call (at most cap
 * written to out, host; *n = the number logged). */
heat_status heat_slab_step_iterations(heat_slab* slab, int* out, int cap, int* n);
/* nslabs, the partition (nslabs + 1 ints, may be NULL) and the device bytes
 * of the slabs' vectors and coefficients (may be NULL). */
heat_status heat_slab_info(const heat_slab* slab, int* nslabs, int* first_layer, long long* device_bytes);
void heat_destroy_slab(heat_slab* slab);

/* ---- allocation-free operator call ---------------------------------------
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory: real-time loops that forbid allocation
 * after start-up, and hosts whose memory manager owns all device memory and
 * hands out only the buffers it was given. It computes y = A' x and
 * *xdoty = x . A' x on caller-owned device buffers, where A' is the step
 * matrix M/dt + theta K of trilinear boxes (heat_params.element = HEAT_ELEM_Q1
 * only; this call has no six-tetrahedra form) with Dirichlet rows and columns
 * replaced by the identity, as heat_apply computes it for such a simulation.
 * It allocates nothing: its reduction scratch (one partial sum per tile of
 * 32x4x8 nodes, and a counter) lives in a fixed file-scope device array of
 * (HEAT_NOALLOC_MAX_TILES + 32) doubles = 33,024 bytes that every GPU loading
 * the library holds until exit.
 *   nx, ny, nz, extent: the mesh, as in heat_create_mesh. At most
 *     HEAT_NOALLOC_MAX_TILES tiles, i.e. ceil((nx+1)/32)*ceil((ny+1)/4)*
 *     ceil((nz+1)/8) <= 4096 (for example 127^3 elements); larger meshes
 *     return HEAT_ERR_ARG without launching anything.
 *   dt, theta, dirichlet_faces: as in heat_params / heat_bc.
 *   coef: device, 2*Ne doubles, (rho_c, k) interleaved per element, element
 *     order, 16-byte aligned. x, y: device, N doubles. xdoty: device, 1 double.
 *     The library cannot check device buffer sizes: buffers shorter than
 *     these are read or written out of bounds.
 *   cuda_stream: stream of the launch (NULL: legacy default stream).
 * Calls share the scratch array and it keeps the last call's contents (the
 * call clears the counter it needs before its launch), so calls that overlap
 * on the GPU (other streams or host threads) race: the caller must serialise
 * them. The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. The call is asynchronous on cuda_stream. */
#define HEAT_NOALLOC_MAX_TILES 4096
heat_status heat_apply_dot_noalloc(int nx, int ny, int nz, const double extent[3], double dt,
                                   double theta, uint32_t dirichlet_faces, const double* coef,
                                   const double* x, double* y, double* xdoty, void* cuda_stream);

/* ---- measurement -------------------------------------------------------- */

/* Time `reps` CG iterations of the sim's current precision (the two tile
 * kernels of one iteration of Algorithm 1: apply+direction+dot, then
 * update+dot; or the one fused kernel, reported as the apply with
 * ms_update = 0) with CUDA events recorded on the sim's stream around each
 * launch. If flush != NULL, flush_bytes of it are overwritten before every
 * timed launch (to evict L2). Outputs the mean ms per launch of each kernel
 * and their algorithmic DRAM bytes per launch (vectors and coefficients each
 * touched once). Needs a prior heat_step on the sim; leaves its solver state
 * undefined (call heat_set_state before stepping again). */
heat_status heat_profile_iteration(heat_sim* sim, int reps, void* flush, size_t flush_bytes,
                                   double* ms_apply, double* ms_update,
                                   double* bytes_apply, double* bytes_update);
/* The same for every member of a batch at once (each launch carries all of
 * them); needs a prior heat_batch_step and leaves the members' solver state
 * undefined. */
heat_status heat_batch_profile_iteration(heat_batch* batch, int reps, void* flush, size_t flush_bytes,
                                         double* ms_apply, double* ms_update,
                                         double* bytes_apply, double* bytes_update);

/* Fused multiply-add throughput of the current GPU (fp64 = 1: FP64, 0: FP32),
 * TFLOP/s (2 flops per FMA), the best of `reps` timed launches of a kernel
 * whose threads run independent register-only FMA chains. The ceiling the
 * FP64 operator passes are measured against: on this GPU FP64 arithmetic,
 * not memory traffic, bounds them (§5.1 runs the paper's kernels in FP64). */
heat_status heat_probe_fma_rate(int fp64, int reps, double* tflops);
/* Microseconds one grid barrier of the persistent iteration (tuning loop)
 * takes on its own: a cooperative launch of blocks_per_sm 128-thread blocks
 * per SM passes `reps` barriers (best of three launches). Every wait is
 * bounded by 1 s (HEAT_ERR_TIMEOUT if one runs out). HEAT_ERR_ARG unless
 * 1 <= blocks_per_sm <= the blocks that fit an SM and 1 <= reps <= 100000. */
heat_status heat_probe_grid_barrier(int blocks_per_sm, int reps, double* us_per_barrier);

/* ---- kernel tuning ------------------------------------------------------ */

/* The process-wide table the kernel choice of every engine comes from; it is
 * read when a simulation's engine (first heat_step after a change of
 * precision), a batch or a server is built, and engines built earlier keep
 * their kernels. The choice depends on the precision and on each mesh's own
 * node count only, so a simulation gives bitwise the same results alone and in
 * any batch built under the same table.
 *   variant[p]: for heat_precision p, the warp-segment apply kernel variant
 *     (0 .. heat_tuning_num_variants()-1) or -1 for the block-tile apply.
 *     Default {-1, 0, 0}.
 *   seg_nodes[b]: output nodes per warp-segment tile for meshes of bucket b
 *     (N < 200000, N < 4000000, larger); 32 .. 2^20, default 512.
 *   pw_quads[p]: for heat_precision p, groups of 4 nodes each thread of the
 *     pointwise update kernel handles (1, 2 or 4; default {2, 4, 4}).
 *   open_w[p]: for heat_precision p, how the step-start and refinement
 *     residual passes run (§3.1's right-hand side, the true residual of
 *     Algorithm 1 and of the refinement): 0 in block tiles, 1 in the
 *     warp-segment march with two-row segments, 2 with one-row segments
 *     (default {2, 2, 2}; trilinear boxes only, six-tetrahedra boxes always
 *     use block tiles). On trilinear boxes the passes of the A operator read
 *     each element's precomputed Walsh-pair coefficients.
 *   loop[p]: for heat_precision p, how the CG iterations of a tick run:
 *     0 as an apply launch and an update launch per iteration, 1 as ONE
 *     persistent cooperative kernel that runs the same work items with a
 *     grid barrier after each phase, until no simulation of the engine is
 *     still iterating or 256 iterations (results bitwise the same; every
 *     barrier wait is bounded, and a wait that runs out fails the
 *     unfinished simulations with HEAT_ERR_TIMEOUT). Only for the FP32
 *     paths (loop[HEAT_FP64] must be 0) with a register-prefetch variant
 *     (stages 0, not fused) on trilinear boxes without Chebyshev passes;
 *     elsewhere the flag is ignored. Default {0, 0, 0}. */
typedef struct heat_tuning {
  int variant[3];
  int seg_nodes[3];
  int pw_quads[3];
  int open_w[3];
  int loop[3];
} heat_tuning;
int heat_tuning_num_variants(void);
/* Shape of variant v: segment width in nodes along x (one lane per node),
 * node rows along y per lane, warps per block, whether an FP64 kernel exists,
 * how its loads travel (0 = plain loads one level ahead into registers,
 * S >= 2 = each thread's own cp.async copies S-1 levels ahead into an S-stage
 * ring in shared memory), and whether it is a fused iteration (FP32 paths
 * only: one kernel per CG iteration in the Chronopoulos-Gear arrangement of
 * PCG, which forms both inner products of an iteration in one reduction,
 * instead of an apply kernel and an update kernel). Any output may be NULL.
 * HEAT_ERR_ARG for an unknown v. */
heat_status heat_tuning_variant(int v, int* seg_width, int* rows, int* warps, int* has_fp64, int* stages,
                                int* fused);
heat_status heat_tuning_get(heat_tuning* t);
/* HEAT_ERR_ARG (table unchanged) for an unknown variant, a variant without
 * an FP64 kernel in variant[HEAT_FP64], or a segment size out of range. */
heat_status heat_tuning_set(const heat_tuning* t);
/* Time CG iterations of this simulation as a solve runs them (the captured
 * tick graph of its engine, about `reps` iterations after 8 warm-up ones,
 * every iteration on a seeded residual that does not converge) for every
 * candidate (block tile; each variant with a segment size of 256, 512, 1024
 * or 2048 nodes; then, for the two fastest variants, the segment sizes whose work
 * items fill whole waves of resident blocks best; then the pointwise item
 * sizes and the persistent iteration) on this simulation's mesh and
 * precision, and store the
 * fastest in the table entries of that precision and of the mesh's size
 * bucket. Outputs the resulting table and the winner's mean ms per iteration
 * (either may be NULL). Needs a prior heat_step; leaves the simulation's solver state
 * undefined (call heat_set_state or heat_set_history before stepping again);
 * its next heat_step builds its engine under the new table. */
heat_status heat_autotune(heat_sim* sim, int reps, heat_tuning* best, double* best_ms);
/* The same over all members of a batch at once (every candidate's launches
 * carry all of them; the segment size is stored for the first member's size
 * bucket); needs a prior heat_batch_step, leaves the members' solver state
 * undefined and rebuilds the batch's engine under the new table. A failure
 * to rebuild leaves the batch unusable (destroy it). */
heat_status heat_batch_autotune(heat_batch* batch, int reps, heat_tuning* best, double* best_ms);

/* ---- compiled-in index checks (the library built with HEAT_CHECK) -------
 * No GPU sanitizer runs on the target machines, so the library can be built
 * a second time with HEAT_CHECK defined (build.py, checked=True, giving
 * lib/libheatgb_check.so): its operator kernels test every node and element
 * index they form against the simulation's bounds, skip an access that
 * would fall outside and count it. heat_checks_compiled() says which build
 * is loaded (1: checked); heat_check_violations gives a simulation's count
 * since it was created (always 0 in the normal build). */
int heat_checks_compiled(void);
heat_status heat_check_violations(heat_sim* sim, unsigned int* count);

const char* heat_last_error(void);
const char* heat_status_string(heat_status s);

#ifdef __cplusplus
}
#endif

#endif /* HEAT_H */
