/*
 * sdcheat.h -- C ABI of the GB300 IMEX multi-rate SDC heat solver.
 *
 * The library advances the fully coupled transient FEM heat equation of a
 * fixed stand and a stock sliding on it (Sec. 2 of Naumann, Ruprecht,
 * Wensch, arXiv:1707.03581) with the implicit-explicit multi-rate spectral
 * deferred correction method of Sec. 3 (Algorithm 1 = predictor,
 * Algorithm 2 = correction sweep):
 *
 *   M dT/dt = f^I(T) + f^E(T, t) + g,          (Eq. ivp)
 *   f^I(T)  = (A + B_env) T = -K T              slow, implicit (diffusion + Robin)
 *   g       = b_env                             slow source (environment)
 *   f^E     = M_B(t) T + C_B(t) T + b(t)        fast, explicit (contact + friction)
 *
 * All compute runs in CUDA kernels for sm_103a; this header carries no
 * C++ or PyTorch types. Conventions shared by every call:
 *
 *  - Every call returns an sdc_status. On error the context stays valid and
 *    sdc_last_error() describes the failure. Nothing is partially applied
 *    unless stated.
 *  - Host arrays passed in are read during the call and copied; the caller
 *    keeps ownership. Device arrays the library creates are owned by the
 *    context and freed by sdc_destroy().
 *  - A context is not thread safe; use one context per host thread/stream.
 *  - DOF numbering: stand nodes 0..n_stand-1, then stock nodes.
 *  - Units: SI (m, s, W, J, K or degC consistently).
 */
#ifndef SDCHEAT_H
#define SDCHEAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sdc_ctx sdc_ctx;

typedef enum {
    SDC_OK = 0,
    SDC_ERR_ARG = -1,            /* invalid argument (sizes, ids, geometry)            */
    SDC_ERR_OOM = -2,            /* a device allocation failed                         */
    SDC_ERR_CUDA = -3,           /* a CUDA runtime call failed                         */
    SDC_ERR_NOT_CONVERGED = -4,  /* a CG solve hit cg_max_iter before cg_rtol          */
    SDC_ERR_TIMEOUT = -5,        /* a bounded device wait gave up                      */
    SDC_ERR_STATE = -6           /* call out of order (e.g. step before assemble)      */
} sdc_status;

/* Standard quadrature nodes of one macro step (Sec. 3, "Single-rate SDC").
 * EQUI_NOLEFT: tau_m = t_n + m dt / M (the paper's choice);
 * RADAU_RIGHT: Radau IIA points (right end included);
 * LOBATTO: Gauss-Lobatto points (both ends; the zero-length first interval is
 * skipped, which leaves every result unchanged). */
typedef enum { SDC_NODES_EQUI_NOLEFT = 0, SDC_NODES_RADAU_RIGHT = 1, SDC_NODES_LOBATTO = 2 } sdc_nodes;

/* Arithmetic of the implicit solves. FP64: FP64 SpMV/CG throughout.
 * MIXED_FP32: FP64 iterative refinement around an FP32 SpMV/CG on the
 * correction; the state, right-hand sides, residuals, f^I/f^E evaluations
 * and quadratures stay FP64. */
typedef enum { SDC_FP64 = 0, SDC_MIXED_FP32 = 1 } sdc_precision;

#define SDC_MAX_SWEEPS 15

/* Diagnostics of one macro step. */
typedef struct {
    double t;                               /* simulated time after the step                  */
    int32_t sweeps;                         /* correction sweeps run (K)                      */
    int32_t n_solves;                       /* implicit solves in the step                    */
    int32_t cg_iters_total;                 /* CG iterations over all solves (inner for MIXED) */
    int32_t cg_iters_max;                   /* largest iteration count of one solve           */
    int32_t refinements_total;              /* outer refinement passes (MIXED only)           */
    int32_t status;                         /* sdc_status of the device-side checks           */
    int32_t kernel_launches;                /* CUDA kernels the step executed                 */
    double residual[SDC_MAX_SWEEPS + 1];    /* r^k, k = 0..K (Eq. residual), if enabled; else -1 */
    double heat_stand;                      /* sum_i m_i T_i over stand DOFs [J]              */
    double heat_stock;                      /* sum_i m_i T_i over stock DOFs [J]              */
    int32_t contact_cluster;                /* CTAs of the thread-block cluster that runs the
                                               contact substeps                               */
    int32_t pad_;
    double true_residual_max;               /* largest ||b - (m x + dtau K x)|| / ||b|| of the step's
                                               mixed-precision solves, with the FP64 operator, if
                                               enabled (sdc_set_diagnostics bit 1); else -1    */
} sdc_step_report;

/* Heat ledger (all FP64). */
typedef struct {
    double stored_stand;    /* sum_i m_i T_i, stand [J, relative to 0 degC]          */
    double stored_stock;    /* same, stock                                            */
    double friction_in;     /* int q(t) |Gamma_R| dt accumulated since set_temperature [J] */
    double t;               /* simulated time                                          */
} sdc_heat;

/* Device allocator hook: alloc(bytes, user) returns a device pointer or NULL;
 * free(ptr, user) releases it. Allocations happen only inside sdc_assemble,
 * sdc_set_scheme and the first sdc_step after either. */
typedef void* (*sdc_alloc_fn)(size_t bytes, void* user);
typedef void (*sdc_free_fn)(void* ptr, void* user);

/* ---------------------------------------------------------------- lifetime */

/* Create a context on CUDA device `device`, issuing all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). *out is set on success. */
sdc_status sdc_create(sdc_ctx** out, int device, void* cuda_stream);

/* Create a context on `device` that creates and owns a non-blocking CUDA
 * stream of its own (destroyed by sdc_destroy); for callers that need many
 * distinct streams, e.g. the members of a batch. */
sdc_status sdc_create_own_stream(sdc_ctx** out, int device);

/* The context's stream (a cudaStream_t), e.g. to order the caller's work after it. */
sdc_status sdc_get_stream(const sdc_ctx* ctx, void** stream);

/* Free every device and host resource of the context (NULL is a no-op). */
void sdc_destroy(sdc_ctx* ctx);

/* Text of the last error of this context (valid until the next call). */
const char* sdc_last_error(const sdc_ctx* ctx);

/* Route device allocations through alloc/free (e.g. a framework's caching
 * allocator). Must be called before sdc_assemble; NULL restores cudaMalloc. */
sdc_status sdc_set_allocator(sdc_ctx* ctx, sdc_alloc_fn alloc, sdc_free_fn free_fn, void* user);

/* ---------------------------------------------------------------- problem */

/* Mesh and material of one body (Sec. 2, Eq. heat-diffusion; the weak form
 * Eq. femContFix / femContMov). body: 0 = fixed stand, 1 = moving stock.
 * xyz: n_nodes x 3 row-major coordinates [m]. hex8: n_hex x 8 node ids
 * (0-based, per body), bottom face counter-clockwise then top face.
 * k_per_hex: n_hex conductivities [W/(m K)] or NULL for uniform k.
 * rho [kg/m^3], c [J/(kg K)]. SDC_ERR_ARG on bad ids or inverted elements
 * (detected in sdc_assemble). */
sdc_status sdc_set_body(sdc_ctx* ctx, int body, const double* xyz, int64_t n_nodes,
                        const int64_t* hex8, int64_t n_hex, const double* k_per_hex,
                        double k, double rho, double c);

/* Robin faces of one body (Sec. 2: environment / cooling / floor exchange,
 * B_env and b_env after Eq. femDiscr): n_faces x 4 node ids going around
 * each bilinear face; heat transfer coefficient h [W/(m^2 K)], T_env. */
sdc_status sdc_set_robin(sdc_ctx* ctx, int body, const int64_t* quad4, int64_t n_faces,
                         double h, double T_env);

/* One more group of Robin faces of a body, with its own heat transfer
 * coefficient and temperature (Sec. 2: B_env and b_env sum over the parts of
 * the boundary that exchange heat with the environment, the floor or cooling
 * equipment, each at its own temperature). sdc_set_robin replaces all groups
 * of the body with one; sdc_add_robin appends one. Same arguments. */
sdc_status sdc_add_robin(sdc_ctx* ctx, int body, const int64_t* quad4, int64_t n_faces,
                         double h, double T_env);

/* Contact between the stand's rail (stand_quads, per-body ids) and the stock
 * (stock_quads, per-body ids in the stock's reference position); Sec. 2,
 * Gamma_R(t), M_B, C_B (Eq. defCB) and b_X(t). Faces must be axis-aligned
 * rectangles in one common plane. The rail is insulated where it is not
 * covered. h_c: exchange coefficient alpha [W/(m^2 K)]; q0_peak: peak
 * friction flux [W/m^2], of which each body receives half. */
sdc_status sdc_set_contact(sdc_ctx* ctx, const int64_t* stand_quads, int64_t n_sq,
                           const int64_t* stock_quads, int64_t n_kq, double h_c, double q0_peak);

/* Rigid stock motion (the motion law of Sec. 5): displacement
 * d(t) = dir * (z0 + amp sin(2 pi t / period)), dir in the contact plane;
 * friction flux q(t) = q0_peak |cos(2 pi t / period)|. period = +inf gives a
 * resting stock with constant flux q0_peak. */
sdc_status sdc_set_motion(sdc_ctx* ctx, const double dir[3], double z0, double amp, double period);

/* Assemble K = -(A + B_env), the lumped mass m (row sums, Sec. 2) and
 * g = b_env for both bodies, build the contact tables and upload everything.
 * Allocates device memory. SDC_ERR_STATE if a body or the contact is missing. */
sdc_status sdc_assemble(sdc_ctx* ctx);

/* Time-stepping scheme (Sec. 3): node family, M standard nodes, P embedded
 * substeps per interval, K correction sweeps (<= SDC_MAX_SWEEPS), embedded
 * interpolation window (0 = min(M, P); P = the paper's literal weights),
 * macro step dt [s], CG relative tolerance ||r||_2 <= cg_rtol ||b||_2 and
 * iteration cap, precision of the implicit solves. */
sdc_status sdc_set_scheme(sdc_ctx* ctx, sdc_nodes nodes, int M, int P, int sweeps, int window,
                          double dt, double cg_rtol, int cg_max_iter, sdc_precision precision);

/* Diagnostics of each macro step, a bit set (costs extra passes):
 *  bit 0 (1): the FP64 SDC residual r^k of Eq. residual after the predictor and every sweep
 *             (MRSDC only; SDC_ERR_ARG with another stepper);
 *  bit 1 (2): the true residual of every mixed-precision implicit solve (Algorithms 1 and 2:
 *             (diag(m) + dtau K) x = b), ||b - (m x + dtau K x)||_2 / ||b||_2 with the FP64
 *             operator and iterate, after the refinement stopped on its carried residual;
 *             the step report's true_residual_max holds the largest. No effect on results. */
sdc_status sdc_set_diagnostics(sdc_ctx* ctx, int flags);

/* Time stepper of sdc_step.
 * SDC_STEPPER_MRSDC (default): IMEX multi-rate SDC (Algorithms 1 and 2).
 * SDC_STEPPER_SISDC: single-rate semi-implicit SDC (Sec. 3, the method MRSDC
 *   extends), with f^E only at the standard nodes and in the right-hand side of
 *   each interval's implicit stage: the IMEX Euler predictor and Eq. sdc_sweep
 *   with I_{m-1}^m = sum_j s_{m,j} F(T^k_j). The scheme's nodes, M, sweeps, dt and
 *   solver settings apply; its P only sets how many embedded geometry slots are
 *   formed (the end slots give f^E at the standard nodes), so P = 1 is cheapest.
 * SDC_STEPPER_IMPLICIT_EULER: fully implicit Euler with the contact coupling in
 *   the matrix (the comparison method of Sec. 1 and Sec. 5): one step of the
 *   scheme's dt solves (m + dt (K - L_E(t_{n+1}))) T_{n+1} = m T_n + dt (g +
 *   f^E(0, t_{n+1})) with FP64 Jacobi-PCG, where f^E(T, t) = f^E(0, t) + L_E(t) T.
 * Residual diagnostics (sdc_set_diagnostics) exist for MRSDC only; SDC_ERR_ARG. */
enum { SDC_STEPPER_MRSDC = 0, SDC_STEPPER_SISDC = 1, SDC_STEPPER_IMPLICIT_EULER = 2 };
sdc_status sdc_set_stepper(sdc_ctx* ctx, int stepper);

/* Execution mode. 0 (default): each macro step is one CUDA graph launch with
 * device-side CG loops. 1: the same kernels as plain launches, each CG loop
 * driven from the host (one small read-back per iteration); for profilers
 * that do not trace kernels inside conditional graph nodes, and for
 * debugging. Results are identical. */
sdc_status sdc_set_execution(sdc_ctx* ctx, int eager);

/* Placement of the contact substep loop's replicas of the contact temperatures:
 * 0 (default) = shared memory of each CTA of the loop's cluster when they fit,
 * else (with no sdc_set_contact_cluster cap) the grid-wide loop of 3 below, else global
 * memory; 1 = always global memory; 2 = global memory and gathers from
 * there. Global replicas are otherwise staged: after each substep one bulk copy brings
 * the whole replica into the CTA's shared memory when it fits (one buffer), and the
 * gathers read it there. 3 = the grid-wide loop: no cluster, one contact DOF a thread on
 * as many co-resident CTAs (a cooperative launch) as the interface needs, global replicas
 * published by a grid barrier with bounded waits (the step report's contact_cluster is then
 * its CTA count; if the device cannot hold them, the cluster forms are used). For tests and
 * tuning: results are identical; SDC_ERR_ARG outside 0..3. */
sdc_status sdc_set_contact_replicas(sdc_ctx* ctx, int global);

/* Side branches in the macro-step graph (1, default): the contact coupling
 * operator of the step and each interval's k_iface_prep, which do not depend
 * on the interval's implicit solve, run beside it instead of before or after
 * it. 0: one chain. Members of a batch (sdc_batch_add) run as one chain while
 * they are members: their concurrency comes from the batch. Results are
 * identical. */
sdc_status sdc_set_graph_branches(sdc_ctx* ctx, int on);

/* (SpMV, update) pairs in each body of the CG loops (the WHILE nodes of the step
 * graph, and the host-driven loop of eager execution), 1..8; 0 (default) = 3 on
 * grids of at most 2048 blocks of 256 rows, else 1. A body runs to its end after
 * the solve stops (its remaining launches return at once), so more pairs trade
 * loop iterations for such launches. Results are identical; SDC_ERR_ARG out of
 * range. */
sdc_status sdc_set_cg_unroll(sdc_ctx* ctx, int pairs);

/* Upper bound on the CTAs of the contact substep loop's thread-block cluster
 * (1..16; 0 = automatic). The loop takes the largest power of two within the
 * bound whose cluster fits on the device. For tuning and tests: results are
 * identical for every cluster size. */
sdc_status sdc_set_contact_cluster(sdc_ctx* ctx, int max_ctas);

/* Blocks a SM of the FP32 CG update's one-wave grid (mixed precision, grids of at most 2048
 * blocks of 256 rows); 0 (default) = as many as fit. Results are identical; SDC_ERR_ARG
 * outside 0..32. */
sdc_status sdc_set_update_blocks(sdc_ctx* ctx, int blocks_per_sm);

/* Launch options picked by sdc_autotune. */
typedef struct {
    int32_t cg_unroll;            /* (SpMV, update) pairs per CG loop body (sdc_set_cg_unroll)     */
    int32_t update_blocks_per_sm; /* FP32 update grid (sdc_set_update_blocks)                       */
    int32_t contact_cluster_cap;  /* cap on the contact loop's cluster (sdc_set_contact_cluster; 0 =
                                     automatic)                                                     */
    int32_t contact_cluster;      /* the cluster size that results                                 */
    int32_t contact_global;       /* 1: replicas in global memory (staged), 2: global, unstaged,
                                     3: grid-wide loop (sdc_set_contact_replicas)                  */
    int32_t graph_branches;       /* sdc_set_graph_branches                                        */
    int32_t trials;               /* option sets timed (0 when taken from the cache)               */
    int32_t cached;               /* 1: picks of an earlier context of the same shape              */
    int32_t skipped;              /* option sets the device could not run (skipped)                 */
    int32_t pad_;
    double ms_default;            /* ms per macro step with the options the context had (-1 cached)*/
    double ms_tuned;              /* ms per macro step with the picks (-1 cached)                   */
} sdc_tune_report;

/* Autotuner: picks the launch options above for this context from timed macro steps in
 * graph execution, and sets them. Each option set is timed on the same trial_steps macro
 * steps (0 = 3) from the context's current state, which is saved first and restored after,
 * so the call leaves T(t_n), the time and the heat ledger as they were. Coordinate descent
 * from the current options; a candidate must be 1 % faster to be taken, and one the device
 * cannot run (a contact cluster too small for the interface) is skipped. Every option leaves
 * results bitwise unchanged. Picks are cached in the process by the problem's shape
 * (device, DOFs, nonzeros, contact DOFs, precision, stepper, nodes, M, P, sweeps): later
 * contexts of that shape take them without trials. Needs sdc_set_temperature; allocates
 * n_dof doubles for the duration of the call; SDC_ERR_STATE in eager execution; rep may be
 * NULL. */
sdc_status sdc_autotune(sdc_ctx* ctx, int32_t trial_steps, sdc_tune_report* rep);

/* Polls of each bounded wait of the contact substep loop's exchange before it gives up
 * (0 = the default, 2^24). A loop whose wait gives up stops exchanging, drains the copies
 * still addressed to it and ends the step with SDC_ERR_TIMEOUT; the context stays usable.
 * For tests of that path (a budget of a few polls gives up on waits that would complete)
 * and for callers that prefer an early error to a long wait. SDC_ERR_ARG if polls < 0. */
sdc_status sdc_set_wait_limit(sdc_ctx* ctx, int64_t polls);

/* Measurement aid for eager execution (sdc_set_execution(ctx, 1)): when on,
 * every kernel launch of a step is bracketed by CUDA events on the
 * context's stream and each step waits for its launches, summing the
 * device time per kernel. Switching it (on or off) clears the sums. */
sdc_status sdc_set_kernel_timing(sdc_ctx* ctx, int on);

/* Per-kernel sums since timing was switched on: up to `capacity` entries of
 * names (static strings owned by the library), launch counts and total
 * device milliseconds; *n_kinds receives the number of kernels seen. Any
 * output array may be NULL. */
sdc_status sdc_get_kernel_times(sdc_ctx* ctx, int32_t capacity, const char** names, int32_t* launches,
                                double* ms_total, int32_t* n_kinds);

/* Initial state: T (host or device pointer of n_dof doubles) or, if T is
 * NULL, the uniform value T_uniform; simulated time t0. */
sdc_status sdc_set_temperature(sdc_ctx* ctx, const double* T, double T_uniform, double t0);

/* ---------------------------------------------------------------- stepping */

/* One macro step t_n -> t_n + dt: Algorithm 1 then K x Algorithm 2, as one
 * CUDA graph launch on the context's stream. If rep is non-NULL the call
 * waits for the step and fills *rep (and returns SDC_ERR_NOT_CONVERGED if a
 * solve hit its cap); if rep is NULL the step is only enqueued and device
 * errors surface at the next synchronising call. */
sdc_status sdc_step(sdc_ctx* ctx, sdc_step_report* rep);

/* Enqueue n_steps macro steps on the context's stream and return at once
 * (errors surface at the next waiting call, e.g. sdc_synchronize). */
sdc_status sdc_step_async(sdc_ctx* ctx, int64_t n_steps);

/* Enqueue n_steps macro steps back to back, then wait once; *last (if not
 * NULL) receives the report of the final step. */
sdc_status sdc_run_horizon(sdc_ctx* ctx, int64_t n_steps, sdc_step_report* last);

/* Wait for all enqueued work; returns the accumulated device status. */
sdc_status sdc_synchronize(sdc_ctx* ctx);

/* Non-blocking: *idle = 1 if every step enqueued on the context's stream has
 * finished, else 0. Errors of finished steps surface at the next waiting call. */
sdc_status sdc_poll(sdc_ctx* ctx, int* idle);

/* ---------------------------------------------------------------- batches
 * A batch runs the macro steps of several machines (contexts) concurrently on
 * one GPU, the batched workloads and the serving loop of this library. Each
 * member keeps its own device state and CUDA graph and must have its own
 * stream (sdc_create); a batch step enqueues the members' step graphs
 * round-robin so that their kernels and contact-loop clusters overlap on the
 * device. Members share nothing, so every result equals the member run alone,
 * bit for bit. The batch does not own its members: destroy them after
 * removing them or destroying the batch. */
typedef struct sdc_batch sdc_batch;

sdc_status sdc_batch_create(sdc_batch** out, int device);
void sdc_batch_destroy(sdc_batch* batch);
const char* sdc_batch_last_error(const sdc_batch* batch);

/* Add a ready context (assembled, scheme and temperature set) whose stream no
 * other member uses; *index receives its position (may be NULL). */
sdc_status sdc_batch_add(sdc_batch* batch, sdc_ctx* ctx, int32_t* index);

/* Remove a member (waits for its enqueued work); positions after it shift down. */
sdc_status sdc_batch_remove(sdc_batch* batch, sdc_ctx* ctx);

sdc_status sdc_batch_size(const sdc_batch* batch, int32_t* n);

/* Enqueue n_steps[i] macro steps of member i (NULL: one step each), round-robin
 * over the members; if wait != 0, wait for all and return the first error. */
sdc_status sdc_batch_step(sdc_batch* batch, const int64_t* n_steps, int wait);

/* Wait for every member; returns the first member error. */
sdc_status sdc_batch_synchronize(sdc_batch* batch);

/* Block-diagonal form of a batch (the batched layout of the stacked per-machine systems of
 * Eq. coupledFEM): on (1), the members that qualify run as one fused group, one CUDA graph
 * per batched macro step on a stream of the batch, in which the FP32 inner CG of every
 * mixed-precision implicit solve (Algorithms 1 and 2) is ONE launch of the SpMV and ONE of
 * the update per iteration over the concatenated rows of all members, with each member's
 * own dot products, step lengths and stop test (a member whose CG stopped returns at once),
 * and one launch of the refinement per pass; the rest of each member's step runs as its
 * own chain of that graph. Results are bitwise those of the members run alone. Qualify:
 * mixed precision, the MRSDC stepper, at most 2048 blocks of 256 rows, no diagnostics,
 * graph execution, and the scheme of the group's first member; the others keep their own
 * graphs. Fused members take equal step counts in sdc_batch_step (else SDC_ERR_ARG). Off
 * (0, the default): every member runs its own graph on its own stream. */
sdc_status sdc_batch_set_fused(sdc_batch* batch, int on);

/* Members in the fused group (0 when the batch is not fused or fewer than two qualify). */
sdc_status sdc_batch_fused_size(sdc_batch* batch, int32_t* n);

/* ---------------------------------------------------------------- results */

/* Device bytes the context holds (assembled system, state and scheme buffers). */
sdc_status sdc_get_footprint(const sdc_ctx* ctx, int64_t* bytes);

/* The MRSDC weight tables of a scheme on the unit step (Sec. 3: the standard-node weights
 * s_{m,j}, the embedded ones of Table 1 and the node positions), as sdc_set_scheme forms
 * them. Host only: no context and no device. Each output may be NULL; otherwise it is a
 * host array of float64, row-major, the caller's:
 *   c    [M+1]       node positions, c[0] = 0 (t_n), c[m] = tau_m;
 *   emb  [M][P+1]    embedded positions tau_{m,p} of interval m (p = 0 is tau_{m-1});
 *   S    [M][M]      s_{m,j};     Shat [M][P]     shat_{m,q};
 *   Stil [M][P][M]   stil_{m,p,j}; Semb [M][P][P] s_{m,p,q}
 * (interval, embedded and node indices from 0). window 0 = min(M, P). SDC_ERR_ARG for
 * arguments sdc_set_scheme refuses. */
sdc_status sdc_scheme_weights(sdc_nodes nodes, int M, int P, int window, double* c, double* emb, double* S,
                              double* Shat, double* Stil, double* Semb);

/* Column form of the stored matrix K (Eq. coupledFEM; sliced ELL of 32-row slices, read by
 * every SpMV of the implicit solves, f^I and the bulk endpoints):
 *   0 (default) = 16-bit offsets from each slice's smallest column when every slice spans at
 *     most 65,535 columns (2 bytes an entry instead of 4; a 27-point stencil numbered plane by
 *     plane spans about two node planes), else 32-bit columns; and the FP32 copy that the
 *     mixed-precision solves stream has implied columns when the matrix allows them: each
 *     slice's rows share one increasing table of relative columns (col - row), absent
 *     neighbours hold 0, and no column is stored (4 bytes an entry instead of 6). Allowed when
 *     every row's columns increase, a slice's table has at most 64 entries and the layout
 *     holds at most 1.25 times the entries of the offsets form: a mesh numbered plane by
 *     plane qualifies, a scrambled numbering does not;
 *   16 = as 0 without implied columns;
 *   32 = 32-bit columns always, no implied columns.
 * Takes effect at the next sdc_assemble. Results are identical in every form: each row's
 * products are summed in the same order. SDC_ERR_ARG for other values. */
sdc_status sdc_set_matrix_columns(sdc_ctx* ctx, int bits);

/* Bits of a column index in the assembled matrix: 16 or 32. SDC_ERR_STATE before
 * sdc_assemble. */
sdc_status sdc_get_matrix_columns(const sdc_ctx* ctx, int32_t* bits);

/* 1 when the assembled matrix's FP32 copy has implied columns (see sdc_set_matrix_columns),
 * else 0. SDC_ERR_STATE before sdc_assemble, SDC_ERR_ARG for a null pointer. */
sdc_status sdc_get_matrix_implied(const sdc_ctx* ctx, int32_t* implied);

/* Sizes: total DOFs, stand DOFs, stored nonzeros of K, contact DOFs. */
sdc_status sdc_get_sizes(const sdc_ctx* ctx, int64_t* n_dof, int64_t* n_stand, int64_t* nnz,
                         int64_t* n_contact);

/* Copy T(t_n) into out (host or device pointer, n == n_dof doubles). Waits. */
sdc_status sdc_get_temperature(sdc_ctx* ctx, double* out, int64_t n);

/* Borrowed device pointer to T(t_n); valid until the next step or destroy. */
sdc_status sdc_get_temperature_device(const sdc_ctx* ctx, const double** dptr);

/* Heat ledger after the last step (waits). */
sdc_status sdc_get_heat_totals(sdc_ctx* ctx, sdc_heat* out);

/* Copy the assembled system to host arrays: row_ptr (n_dof+1), col (nnz),
 * val (nnz) of K in CSR with sorted columns, mass (n_dof), genv (n_dof).
 * Any pointer may be NULL to skip it. */
sdc_status sdc_get_system(const sdc_ctx* ctx, int64_t* row_ptr, int64_t* col, double* val,
                          double* mass, double* genv);

/* ---------------------------------------------------------------- components
 * Single operations of the step on caller-owned device buffers of n_dof
 * doubles, run on the context's stream (asynchronous unless stated). */

/* y = m .* x + dtau K x (the implicit-stage operator of Algorithms 1 and 2). */
sdc_status sdc_apply_operator(sdc_ctx* ctx, double dtau, const double* x_dev, double* y_dev);

/* Stationary initial state (Sec. 5: the machine at rest, in thermal exchange
 * with the environment and cooling equipment only, 0 = f^I(T0) + g, i.e.
 * K T0 = b_env). Solves it with Jacobi-PCG in FP64 on the device, from the
 * current temperature (zero if none was set), to ||b_env - K T0||_2 <= rtol
 * ||b_env||_2, and makes T0 the temperature at time t0 (as sdc_set_temperature
 * does). K is nonsingular when every body has Robin faces with h > 0. Waits;
 * *iters receives the CG iterations (may be NULL). SDC_ERR_NOT_CONVERGED after
 * max_iter iterations (the state is then the last iterate). Uses n_dof doubles
 * of device memory for the duration of the call. */
sdc_status sdc_set_stationary_state(sdc_ctx* ctx, double t0, double rtol, int32_t max_iter, int32_t* iters);

/* Solve (diag(m) + dtau K) x = b with Jacobi-PCG in the scheme's precision;
 * x_dev holds the initial guess on entry. Waits; *iters receives the
 * iteration count (may be NULL). */
sdc_status sdc_solve(sdc_ctx* ctx, double dtau, const double* b_dev, double* x_dev, int32_t* iters);

/* Measurement aid for the implicit solves of Algorithms 1 and 2 (the CG of the implicit
 * stage; its arithmetic is that of sdc_solve): the device time of n_iters consecutive CG
 * iterations on (diag(m) + dtau K) x = b, b = g and x0 = T(t_n), in the scheme's precision
 * (FP32 inner iterations for SDC_MIXED_FP32), launched as one CUDA graph of the same kernels,
 * grids and launch order as a macro step's CG loop. The stop test is disabled so that every
 * iteration works; spmv_only != 0 launches only the SpMV kernel of each iteration. *ms
 * receives the milliseconds of the n_iters iterations (CUDA events on the context's stream
 * around that graph; an initial-residual kernel runs before the first event). If ms_spmv is
 * not NULL, the same iterations run again from the same start with event records around
 * every SpMV inside the graph, and *ms_spmv receives the sum of the SpMVs' durations. Uses
 * the step's work buffers, not T(t_n); waits. SDC_ERR_ARG unless 1 <= n_iters <= 4096 and
 * dtau > 0. Needs sdc_set_temperature. */
sdc_status sdc_time_cg_iterations(sdc_ctx* ctx, double dtau, int32_t n_iters, int32_t spmv_only, float* ms,
                                  float* ms_spmv);

/* f^E(T, t) on all DOFs (zero away from the contact): Sec. 2, the contact
 * and friction terms of Eq. femContFix / femContMov. */
sdc_status sdc_contact_flux(sdc_ctx* ctx, const double* T_dev, double t, double* fE_dev);


/* ---------------------------------------------------------------- allocation-free variant
 * The paper has no counterpart: this is a service for callers that must not
 * allocate device memory while they run. Examples are a monitoring hook
 * inside a real-time look-ahead loop, where a cudaMalloc/cudaFree would
 * implicitly synchronise the device and stall the steps in flight, and a
 * process that has handed all free device memory to another framework's
 * pool.
 *
 * heat_dev[0] = sum over stand DOFs of m_i T_i, heat_dev[1] = the same over
 * stock DOFs [J], for any temperature field T_dev (device, n_dof doubles) of
 * this context's model. Same reduction as the ledger behind
 * sdc_get_heat_totals. heat_dev is a device pointer to 2 doubles, written
 * asynchronously on the context's stream.
 *
 * The call allocates nothing. Its scratch is one fixed 512 KiB (+256 B) device
 * array inside the library, present on every GPU that loads the library
 * until the process exits. Limit: n_dof <= 8,388,608; larger models get
 * SDC_ERR_ARG with a message.
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * All calls on a device share the one array. Calls whose kernels overlap on
 * the GPU (other streams, other contexts) race on it and give wrong totals,
 * so serialise them, e.g. on one stream. */
sdc_status sdc_heat_totals_noalloc(sdc_ctx* ctx, const double* T_dev, double* heat_dev);

#ifdef __cplusplus
}
#endif

#endif /* SDCHEAT_H */
