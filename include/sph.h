/*
 * sph.h - C ABI of the GB300 grad-h SPH neighbour-loop library (libsph.so).
 *
 * The library computes, on one NVIDIA GB300 (sm_103a), the per-step hot path
 * of the grad-h SPH method described by Hubber, Rosotti & Booth (2018),
 * "GANDALF - Graphical Astrophysics code for N-body Dynamics And Lagrangian
 * Fluids" (arXiv:1709.04488):
 *   - neighbour search (Morton-key sort, leaf cells, a tree over the leaves),
 *   - the density / smoothing-length solve, Eqs. SPHRHO and HRHO, iterated by
 *     Newton-Raphson to convergence, with the grad-h term Omega, Eq. OMEGA,
 *   - pressure accelerations and energy rates, Eqs. GRADHMOMEQN and
 *     GRADHENEQN, with Monaghan (1997) viscosity and Wadsley (2008)
 *     conductivity, Eqs. MON97ARTVISC and MON97ENERGYDISS,
 *   - the CFL time-step, Eq. SPH_DT, and the global-step leapfrog
 *     kick-drift-kick, Eqs. LFKDK1 and LFKDK2.
 * The smoothing kernel is the M4 cubic spline (support 2h) or the M6
 * quintic spline (support 3h), the two kernels of Sec. 2.
 *
 * Conventions shared by every entry point
 *   - All functions return an int status: SPH_OK (0) or a negative SPH_E*
 *     code.  sph_last_error() returns a message for the calling thread's last
 *     failure.  No function aborts the process.
 *   - Device memory is owned by the caller (e.g. PyTorch tensors).  The library
 *     never allocates device memory; the caller passes particle arrays and a
 *     workspace whose size sph_workspace_bytes() reports.  Host memory passed
 *     in is only read during the call.  A context (sph_ctx) is a small host
 *     object that records pointers, sizes and the stream; it owns no device
 *     memory.
 *   - All work is enqueued on the caller's CUDA stream (a cudaStream_t passed
 *     as void*; NULL is the legacy default stream).  Unless the context was
 *     created with SPH_FLAG_ASYNC, each compute call synchronises that stream
 *     before returning so that it can report device-side errors; with
 *     SPH_FLAG_ASYNC it returns after enqueueing and sph_sync() reports them.
 *   - Particle arrays are structure-of-arrays, FP64, length n, in the caller's
 *     particle order, which the library never changes.
 */
#ifndef SPH_H
#define SPH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define SPH_OK 0
#define SPH_EINVAL -1       /* bad parameter, size or pointer                      */
#define SPH_EBOX -2         /* periodic box too small: 2h reached half a box side  */
#define SPH_ENOCONV -3      /* h-rho iteration did not converge for some particle  */
#define SPH_ENONFINITE -4   /* NaN or Inf met in inputs or results                 */
#define SPH_ETIMEOUT -5     /* a bounded device wait gave up                       */
#define SPH_ETOOBIG -6      /* request larger than the server's memory budget      */
#define SPH_EBUSY -7        /* server queue full                                   */
#define SPH_EAGAIN -8       /* result not ready yet                                */
#define SPH_ECUDA -9        /* a CUDA runtime call failed                          */
#define SPH_ENOSPACE -10    /* workspace too small                                 */

/* ---- parameters -------------------------------------------------------- */
#define SPH_EOS_ADIABATIC 0  /* P = (gamma-1) rho u, c = sqrt(gamma P / rho) (Sec. 2.1.1) */
#define SPH_EOS_ISOTHERMAL 1 /* P = cs^2 rho, c = cs; u is not evolved (Sec. 6.2)         */

#define SPH_PREC_FP64 0      /* every step in FP64 (the plain reference path)              */
#define SPH_PREC_MIXED 1     /* FP32 pair arithmetic; FP64 positions, centre differences, */
                             /* integration, accumulation of a and the global reductions  */

#define SPH_KERNEL_M4 0      /* M4 cubic spline, support 2h (Sec. 2)                      */
#define SPH_KERNEL_M6 1      /* M6 quintic spline, support 3h (Sec. 2)                    */

#define SPH_AC_WADSLEY 0     /* conductivity signal speed |v_ij . r_hat_ij| (Wadsley 2008)  */
#define SPH_AC_PRICE 1       /* conductivity signal speed sqrt(|P_i - P_j| / rho_bar) (Price) */

#define SPH_AV_CONSTANT 0          /* viscosity alpha_av everywhere                       */
#define SPH_AV_MORRIS_MONAGHAN 1   /* per-particle alpha, Morris & Monaghan (1997) switch  */
#define SPH_AV_CULLEN_DEHNEN 2     /* per-particle alpha, Cullen & Dehnen (2010) switch    */

#define SPH_FLAG_ASYNC 1u    /* compute calls return without synchronising the stream     */
#define SPH_FLAG_TIMING 2u   /* record CUDA events around the stages of every step        */

/* stages reported by sph_stage_times */
#define SPH_STAGE_KICK_DRIFT 0   /* half kick + drift + predictor                 */
#define SPH_STAGE_SORT 1         /* domain, Morton keys, radix sort, gather       */
#define SPH_STAGE_TREE 2         /* leaves, leaf boxes, tree levels              */
#define SPH_STAGE_DENSITY 3      /* density / h solve (incl. the slow path)      */
#define SPH_STAGE_REFIT 4        /* smoothing-sphere boxes                       */
#define SPH_STAGE_FORCES 5       /* accelerations, du/dt, signal speeds          */
#define SPH_STAGE_GRAVITY 6      /* direct-sum self-gravity (problems with gravity) */
#define SPH_STAGE_CLOSE 7        /* closing half kick, reductions, CFL step      */
#define SPH_NSTAGES 8

typedef struct {
    int periodic;          /* 1: periodic box [box_lo, box_lo + box_len) per axis; 0: isolated */
    double box_lo[3];
    double box_len[3];
    int eos;               /* SPH_EOS_*                                                */
    double gamma;          /* ratio of specific heats (adiabatic)                      */
    double cs_iso;         /* isothermal sound speed                                   */
    double eta;            /* h = eta (m/rho)^(1/3), Eq. HRHO; paper default 1.2       */
    double alpha_av;       /* viscosity strength alpha_AV (paper: 1)                   */
    double beta_av;        /* signal-speed factor beta_AV = 2 alpha_AV (Sec. 2.1.1)    */
    double alpha_ac;       /* conductivity strength alpha_AC (0 disables)              */
    double c_cfl;          /* Courant factor of Eq. SPH_DT (paper: ~0.2)               */
    double h_tol;          /* stop the h iteration when |dh|/h < h_tol (0: per precision)*/
    int h_max_iter;        /* iteration cap (0: 50)                                     */
    int precision;         /* SPH_PREC_*                                               */
    int kernel;            /* SPH_KERNEL_M4 (cubic spline, support 2h) or SPH_KERNEL_M6
                              (quintic spline, support 3h), Sec. 2; the M6 kernel is
                              W = g(q) / (120 pi h^3), g = (3-q)^5 - 6 (2-q)^5 + 15 (1-q)^5
                              with each term present while its bracket is positive.
                              With M6, eta ~ 1.0 gives ~113 neighbours.  Any other
                              value: SPH_EINVAL.                                    */
    int leaf_size;         /* particles per leaf, 8/16/32 (0: chosen by the autotuner) */
    int lanes_per_particle;/* 1/2/4/8 lanes of a warp per particle (0: autotuner)      */
    unsigned flags;        /* SPH_FLAG_*                                               */
    int tree_rebuild_every;/* sph_step/sph_run: sort and rebuild the leaves every k-th
                              step and only update the leaf and node boxes bottom-up in
                              between (Sec. 4.2, tree reuse); 0 or 1: every step.
                              Results do not depend on it beyond round-off; the tree's
                              efficiency does.  Batched steps always rebuild.       */
    int ac_signal;         /* artificial-conductivity signal speed (Sec. 2.1.1):
                              SPH_AC_WADSLEY |v_ij . r_hat_ij| (default) or SPH_AC_PRICE
                              sqrt(|P_i - P_j| / rho_bar_ij).  Any other value: SPH_EINVAL */
    int av_switch;         /* SPH_AV_CONSTANT (alpha_av everywhere, default) or
                              SPH_AV_MORRIS_MONAGHAN: one alpha per particle (state.alpha),
                              d alpha/dt = -(alpha - alpha_min) av_decay c / h
                              + max(-div v, 0) (alpha_av - alpha), integrated like u;
                              pair (i,j) uses alpha_ij = (alpha_i + alpha_j)/2 and
                              beta_ij = beta_av / alpha_av alpha_ij (Sec. 2.1.1 names the
                              Morris & Monaghan 1997 switch).  Requires alpha_av > 0,
                              0 <= alpha_min <= alpha_av, av_decay > 0 and non-NULL
                              state.alpha, state.dalpha; not accepted by the server.
                              SPH_AV_CULLEN_DEHNEN: alpha per particle from a shock
                              indicator (Cullen & Dehnen 2010): the force pass forms the
                              velocity gradient V = -(1/(Omega rho)) sum_j m_j v_ij (x)
                              grad_i W(h_i), D = tr V, the traceless shear S, R = (1/rho)
                              sum_j sign(D_j) m_j W(r_ij, h_i) (self included, signs of
                              the previous evaluation), xi = q^2/(q^2 + tr S S^T) with
                              q = 2 (1-R)^4 D; each step then sets A = xi max(-dD/dt, 0)
                              (dD/dt between the step's two force evaluations),
                              alpha_loc = alpha_av h^2 A / (v_sig^2 + h^2 A), and alpha =
                              alpha_loc where alpha < alpha_loc, else it decays towards it
                              with time constant h / (2 av_decay v_sig).  state.dalpha
                              holds D (input: the previous evaluation's, 0 at the start;
                              output: this one's).  Not with block time-steps.        */
    double alpha_min;      /* switch: floor alpha decays to (default 0.1)               */
    double av_decay;       /* switch: decay rate in units of c/h (default 0.1)          */
    int gravity;           /* 1: self-gravity, Eq. SPHSELFGRAV (Sec. 2.1.2): the kernel-
                              softened attraction -G sum_j m_j (phi'(r,h_i)+phi'(r,h_j))/2
                              r_hat over every particle of the problem plus the zeta term
                              of Eq. GRADHZETA over the neighbours.  Isolated problems and
                              the M4 kernel only (SPH_EINVAL otherwise).                 */
    double G;              /* gravitational constant (gravity; must be > 0)            */
    double grav_theta;     /* gravity: 0 (default) sums the attraction directly over
                              every pair, O(n^2); 0 < theta <= 1 walks the tree instead
                              (Sec. 4.2): a node is used through its monopole and
                              quadrupole moments when the squared distance from its
                              centre of mass to the leaf's box is at least l^2/theta^2
                              (l: distance from the centre of mass to the node box's
                              farthest corner) and no pair with it is softened (boxes
                              at least 2 max h apart); other nodes are opened, opened
                              leaves summed pair by pair.  Outside [0, 1]: SPH_EINVAL. */
    double c_grav;         /* gravity: acceleration condition of Eq. SPH_DTACCEL, the
                              step is also at most c_grav sqrt(h_i / |a_i|) (default 0.5;
                              must be > 0 with gravity)                                   */
    int block_levels;      /* hierarchical block time-steps (Sec. 2.1.4) for
                              sph_block_step: largest level L, 0..20 (0 = none, the
                              default).  With gravity the long range and the zeta
                              term follow the same active set, and the acceleration
                              condition enters each particle's step.                    */
    int block_gap;         /* block steps: limiter gap in levels (Saitoh & Makino):
                              a particle's step is at most 2^gap times its shortest
                              neighbour's (default 2; 1..20)                              */
} sph_params;

/* Caller-owned device arrays, FP64, length n, caller's particle order.
 * Inputs: x,y,z, vx,vy,vz, u, m, and h (the starting guess of the iteration;
 * h <= 0 asks for a default guess).  Outputs written by the library:
 * h, rho, omega, P, c (density solve), ax,ay,az, du (= du/dt), vsig (forces).
 * sph_step also advances x, v and u in place. */
typedef struct {
    double *x, *y, *z;
    double *vx, *vy, *vz;
    double *u, *m, *h;
    double *rho, *omega, *P, *c;
    double *ax, *ay, *az, *du, *vsig;
    double *alpha, *dalpha; /* viscosity switch only (else may be NULL): alpha per particle
                               (input, advanced by sph_step) and d alpha/dt (output of the
                               force evaluation)                                          */
} sph_state;

/* Per-call diagnostics (FP64 reductions over the particles, Sec. 2.1.1
 * conservation; counters of the work done). */
typedef struct {
    double mass;           /* sum m                                   */
    double momentum[3];    /* sum m v                                 */
    double energy;         /* sum m (v^2/2 + u)  (u only if adiabatic) */
    double force_sum[3];   /* sum m a                                 */
    double dEdt;           /* sum m (v.a + du/dt)                     */
    double dt_next;        /* C_CFL min h / v_sig (Eq. SPH_DT)         */
    double time;           /* simulated time advanced by sph_step     */
    int64_t steps;         /* steps taken                             */
    int64_t nr_iterations; /* Newton-Raphson iterations, summed        */
    int32_t nr_max;        /* largest iteration count of one particle */
    int32_t ngb_min, ngb_max; /* neighbours inside 2h (incl. self)     */
    double ngb_mean;
    int64_t density_pairs; /* in-range (i,j) pair evaluations, density pass, all iterations */
    int64_t force_pairs;   /* in-range (i,j) pair evaluations, force pass                  */
    int64_t candidates;    /* staged candidate pairs tested, both passes                   */
    int64_t fallback;      /* particles finished by the slow fallback path                 */
    int64_t leaves;        /* leaves built                                                  */
    int32_t status;        /* device-side status (SPH_OK or SPH_E*)                         */
    int32_t unconverged;   /* particles that met SPH_ENOCONV                                */
    int32_t walk_reused;   /* 1: the last force pass took its candidate leaves from the
                              density pass's walk; 0: it walked the tree itself            */
    int32_t wrap_leaves;   /* leaves of the last density + force passes whose pair vectors
                              needed minimum-image wraps (periodic; few particles per
                              box length)                                                  */
    int64_t grav_pairs;    /* gravity tree walk, last force pass: (i,j) pair terms summed  */
    int64_t grav_nodes;    /* gravity tree walk, last force pass: (i,node) multipole terms */
} sph_diag;

typedef struct sph_ctx sph_ctx;

/* Fill *p with the paper's defaults (eta 1.2, alpha_AV 1, beta_AV 2,
 * alpha_AC 1, C_CFL 0.2), periodic unit cube, adiabatic gamma 5/3, mixed
 * precision, autotuned launch shape. */
int sph_params_default(sph_params *p);

/* Bytes of device workspace a context of n particles needs (0 on bad input). */
size_t sph_workspace_bytes(int64_t n, const sph_params *p);

/* Create a context.  state: caller-owned device arrays (see sph_state);
 * workspace: device memory of at least sph_workspace_bytes(n, p) bytes,
 * 256-byte aligned, owned by the caller and reserved for this context until
 * sph_destroy.  stream: cudaStream_t as void*.  Validates the parameters
 * (SPH_EINVAL) and copies them.  n may be 0. */
int sph_setup(sph_ctx **out, const sph_params *p, int64_t n, const sph_state *state,
              void *workspace, size_t ws_bytes, void *stream);

/* Neighbour search and the density / smoothing-length solve (Eqs. SPHRHO,
 * HRHO, OMEGA) at the current positions, starting from state->h.  Writes h,
 * rho, omega, P, c.  SPH_ENOCONV if a particle failed to converge within
 * h_max_iter iterations (results for the others are valid); SPH_EBOX if 2h
 * reached half a periodic box side. */
int sph_density_h(sph_ctx *ctx);

/* Accelerations, du/dt and signal speeds (Eqs. GRADHMOMEQN, GRADHENEQN,
 * MON97ARTVISC, MON97ENERGYDISS, SPH_DT) from the current h, rho, omega, P, c
 * (run sph_density_h first).  Also updates the CFL time-step returned by
 * sph_diagnostics.dt_next. */
int sph_forces(sph_ctx *ctx);

/* One global-step kick-drift-kick (Eqs. LFKDK1/2): half kick and drift with
 * the stored a and du/dt, density solve and forces at the new positions with
 * the predicted v and u, closing half kick.  dt > 0 uses that step; dt <= 0
 * uses the CFL step computed by the previous force evaluation.  The state must
 * hold a valid force evaluation (sph_density_h + sph_forces once after setup).
 * If dt_used is not NULL the step is written there (this synchronises). */
int sph_step(sph_ctx *ctx, double dt, double *dt_used);

/* Take nsteps steps with the CFL time-step without host round trips (one
 * captured CUDA graph replayed nsteps times). */
int sph_run(sph_ctx *ctx, int nsteps);

/* One hierarchical block step (Sec. 2.1.4) of a context set up with
 * block_levels = L > 0: every particle goes from one synchronisation point to
 * the next, Delta t_MAX = min(max_i dt_i, 2^L min_i dt_i) later (dt_i the CFL
 * step of the last force evaluation).  A particle on level l steps by
 * Delta t_MAX / 2^l with its own kick-drift-kick; at every tick where some
 * particle's step ends all particles drift, and the particles whose step ends
 * get a new h and density and forces (from the positions and predicted v and
 * u of all), the closing half kick and the level and opening half kick of
 * their next step; the others keep the h, rho, omega, P and c of their last
 * solve.  Levels rise freely and fall by one
 * at a time where synchronised; Saitoh & Makino's limiter keeps each step
 * within 2^block_gap of the neighbours' (predictive: from the neighbours'
 * largest level at the last force pass; reactive: particles that take forces
 * shorten the steps of slower neighbours, which then end at the next tick of
 * their new level).  Needs a force evaluation first; leaves every particle
 * synchronised with fresh forces.  Tree reuse (tree_rebuild_every = k > 1):
 * the block starts from the context's leaves, the ticks at multiples of k
 * sort and build afresh and the others keep and refit them; the last tick
 * (2^L) always builds them.  Writes Delta t_MAX to *dtmax and the
 * number of particle force evaluations to *evals (either may be NULL).
 * The schedule lives on the device: on a stream that can be captured, the
 * first call captures one CUDA graph whose ticks are a conditional while
 * loop (no host round trip between ticks) and later calls replay it; on the
 * legacy default stream the host reads a loop flag after every tick.  In a
 * tick the pair kernels serve tasks of a leaf's particles whose step ends
 * rather than whole leaves: one particle with a whole warp in FP32 pairs
 * with the M4 kernel, up to 4 with 8 lanes each with M6 or self-gravity, 8
 * with 4 lanes in FP64.  Synchronises once at the end. */
int sph_block_step(sph_ctx *ctx, double *dtmax, int64_t *evals);

/* Capture the block step's graph now (see sph_block_step), so that the first
 * sph_block_step does not include the capture; nothing runs.  SPH_OK on the
 * legacy default stream, where nothing is captured.  SPH_EINVAL: ctx NULL or
 * set up without block_levels; SPH_ECUDA: capture or instantiation failed. */
int sph_block_prepare(sph_ctx *ctx);

/* Copy each particle's time-step level (int32, caller's order) into the
 * device array levels (n entries). */
int sph_block_levels(sph_ctx *ctx, int32_t *levels);

/* Wait for the context's queued work and report the device-side status. */
int sph_sync(sph_ctx *ctx);

/* Diagnostics of the last compute call (synchronises). */
int sph_diagnostics(sph_ctx *ctx, sph_diag *out);

/* Exact FP64 neighbour lists in CSR form, ids ascending (Sec. 4.2 tree walk
 * retrieves them per leaf).  kind 0: {j : |r_ij|^2 < (2 h_i)^2} including i;
 * kind 1: {j != i : |r_ij|^2 < (2 max(h_i,h_j))^2}.  h_in: device array of n
 * smoothing lengths to use (NULL: state->h).  Distances are formed in FP64 as
 * dx*dx + dy*dy + dz*dz without fused multiply-add, after the periodic minimum
 * image of each coordinate difference.  offsets (n+1 entries) and idx (cap
 * entries) are device arrays; *total receives the number of entries (if it
 * exceeds cap, idx holds the first cap and SPH_ENOSPACE is returned). */
int sph_neighbours(sph_ctx *ctx, int kind, const double *h_in, int64_t *offsets, int32_t *idx,
                   int64_t cap, int64_t *total);

/* Durations in milliseconds of the stages of the last step or compute call
 * (CUDA events on the context's stream; needs SPH_FLAG_TIMING, synchronises).
 * Stages that did not run report 0.  ms must hold SPH_NSTAGES doubles. */
int sph_stage_times(sph_ctx *ctx, double *ms);

/* Number of kernel launches one step makes (the kernel nodes of the captured
 * step graph; builds the graph if sph_run has not yet done so, which takes one
 * step).  Needs a non-default stream. */
int sph_step_kernel_count(sph_ctx *ctx, int *kernels);

/* Release the context (frees no caller memory). */
int sph_destroy(sph_ctx *ctx);

/* ---- batching: many independent problems in one launch set ------------- */
/* Bytes of device workspace for a batch of the given contexts. */
size_t sph_batch_workspace_bytes(sph_ctx *const *ctxs, int nctx);

/* Advance every context by nsteps CFL steps; each kernel of a step runs once
 * over all problems (work lists of (problem, leaf) items).  Every problem's
 * result equals the result of stepping it alone.  All contexts must use the
 * same precision and stream; workspace is caller-owned device memory of at
 * least sph_batch_workspace_bytes().  Synchronises; returns the first error
 * among the contexts (each context's own status: sph_sync or
 * sph_diagnostics).  A later sph_step of one context alone rebuilds its
 * leaves first. */
int sph_batch_step(sph_ctx *const *ctxs, int nctx, int nsteps, void *workspace, size_t ws_bytes);

/* A resident batch of contexts (the batched path of the many-problem
 * workloads): the problem tables are uploaded once at creation, and one
 * batched step (every kernel once over all problems: persistent work-queue
 * launches over (problem, leaf) items for the density and force passes)
 * runs eagerly the first time, is captured as a CUDA graph the second time
 * and replayed after that, with no host round trip between steps.  The contexts must have a
 * force evaluation, share precision and a non-default stream, and stay alive
 * and unchanged in size while the batch exists; workspace as for
 * sph_batch_step, reserved for the batch until sph_batch_destroy.
 * flags: SPH_FLAG_TIMING records CUDA events around the stages of each step
 * (sph_batch_stage_times).  Every problem's result equals stepping it alone.
 * No counterpart in the paper (its batches are OpenMP loops over one
 * problem's cells); the work unit, a leaf cell, is the paper's. */
typedef struct sph_batch sph_batch;
int sph_batch_create(sph_batch **out, sph_ctx *const *ctxs, int nctx, void *workspace, size_t ws_bytes,
                     unsigned flags);
/* Enqueue nsteps batched CFL steps (graph replays; asynchronous). */
int sph_batch_run(sph_batch *b, int nsteps);
/* Wait for the batch's work; writes each context's status to status[k]
 * (nctx entries, may be NULL) and returns the first error among them. */
int sph_batch_sync(sph_batch *b, int *status);
/* Stage durations (ms, SPH_NSTAGES doubles) of the last batched step. */
int sph_batch_stage_times(sph_batch *b, double *ms);
/* Kernel launches in one captured batched step (after the second step). */
int sph_batch_kernel_count(sph_batch *b, int *kernels);
int sph_batch_destroy(sph_batch *b);

/* ---- serving: continuous batching of independent runs ------------------ */
typedef struct {
    void *pool;            /* caller-owned device memory the server carves slots from */
    size_t pool_bytes;     /* admission budget (bytes of pool)                         */
    int max_slots;         /* concurrent problems (<= 4096)                            */
    int max_queue;         /* queued requests before SPH_EBUSY                         */
    void *stream;          /* cudaStream_t as void*                                    */
    int precision;         /* SPH_PREC_* for every request                             */
} sph_server_cfg;

typedef struct {
    int64_t n;             /* particles                                    */
    const double *x, *y, *z, *vx, *vy, *vz, *u, *m, *h; /* host arrays, copied at submit */
    sph_params params;     /* per-request physics (precision/flags ignored) */
    int nsteps;            /* CFL steps to take (>= 1; else SPH_EINVAL)     */
    double arrival;        /* arrival time on the server's clock (seconds) */
} sph_request;

typedef struct {
    int status;            /* SPH_OK or error                               */
    int64_t n;
    int steps_done;
    double arrival, admitted, completed; /* server-clock seconds             */
    double t_sim;          /* simulated time reached                         */
    double *x, *y, *z, *vx, *vy, *vz, *u, *h, *rho; /* host arrays of n, caller-owned, filled at poll (may be NULL) */
} sph_result;

typedef struct sph_server sph_server;

int sph_server_create(sph_server **out, const sph_server_cfg *cfg);
/* Queue a request; copies its host arrays.  SPH_ETOOBIG if it can never fit
 * the pool, SPH_EBUSY if the queue is full.  *ticket identifies it. */
int sph_server_submit(sph_server *s, const sph_request *req, uint64_t *ticket);
/* Drive the loop until now >= until (server clock) or all work is done:
 * admit queued requests whose arrival time has passed while slots and pool
 * memory allow, advance every resident problem by one batched step per tick,
 * retire finished ones.  virtual_clock != 0 advances the clock by the measured
 * GPU time of each tick instead of reading the wall clock. */
int sph_server_run(sph_server *s, double until, int virtual_clock);
/* Fetch a finished result (SPH_EAGAIN if not finished).  Host arrays in out
 * that are not NULL receive the final particle state. */
int sph_server_poll(sph_server *s, uint64_t ticket, sph_result *out);
/* Current server clock (seconds). */
double sph_server_clock(const sph_server *s);
int sph_server_destroy(sph_server *s);

/* ---- allocation-free entry point --------------------------------------- */
/* Density solve and force evaluation (what sph_density_h followed by
 * sph_forces compute) for callers that may not create device allocations of
 * their own, e.g. a host application that reserves all device memory in its
 * own pool, or a plug-in or real-time loop called from such a host.  The paper
 * has no counterpart: this is a property of the library, not of the method.
 *   - Allocates nothing: no cudaMalloc/cudaFree, no allocating library call.
 *     Its scratch memory is a fixed 24 MiB array compiled into the library,
 *     which every GPU that loads the library holds until the process exits.
 *   - n is at most 32768, whatever the options (precision, kernel,
 *     self-gravity by direct sum or tree walk; the FP64 tree walk's layout,
 *     the largest, takes about 22 MiB); larger n returns SPH_EINVAL with a
 *     message.  (A layout that did not fit would return SPH_ENOSPACE, before
 *     touching the device, naming the largest n that fits.)
 *   - The caller passes the particle arrays (inputs and outputs as in
 *     sph_state) and the stream; p as for sph_setup (SPH_FLAG_ASYNC skips the
 *     final synchronisation, and then no status is reported).
 *   - The first call on a device looks up the array's device address (a
 *     one-time set-up per device); make that first call before any stream
 *     capture.
 *   - All calls share the one array, which keeps the last call's contents:
 *     calls whose work overlaps on the GPU (other streams, other threads)
 *     race with each other and must be serialised by the caller. */
int sph_density_forces_noalloc(const sph_params *p, int64_t n, const sph_state *state, void *stream);

/* Launch-shape table for contexts whose params leave lanes_per_particle and
 * leaf_size at 0: a problem of n particles uses lanes[k] lanes per particle
 * (leaf size 32 / lanes[k]) for the first row k with n <= n_max[k]; sizes
 * beyond the last row, and every size when rows == 0 (the state at load
 * time), use the built-in rule (2 lanes up to 67023 particles, else 1: the
 * table the package's autotuner measured on GB300).
 * The table is process-wide and copied; it applies to contexts set up after
 * the call.  lanes[k] must be 1, 2, 4 or 8 and n_max must increase;
 * otherwise SPH_EINVAL and the table is unchanged.  At most 32 rows.  The
 * FP64 path clamps lanes to 2 or 4.  No counterpart in the paper: the
 * package's autotuner measures the table on the GPU and installs it. */
int sph_set_launch_table(const int64_t *n_max, const int32_t *lanes, int rows);

/* ---- hardware ceiling of the pair kernels ------------------------------ */
/* Measured fused multiply-add throughput of the current device: independent
 * FP32 (precision SPH_PREC_MIXED) or FP64 (SPH_PREC_FP64) chains on every SM,
 * 2 flop per fused multiply-add, one launch of about target_ms milliseconds
 * (0 < target_ms <= 10000) after short calibration launches, timed with CUDA
 * events on stream.  Writes TFLOP/s to *tflops and the timed launch's
 * duration to *ms (may be NULL).  Synchronises the stream.  Allocates no
 * device memory.  The pair arithmetic of the density and force passes is
 * bound by this pipe (no dense contraction), so it is the ceiling their
 * roofline fraction is taken against; the paper has no counterpart. */
int sph_alu_peak(int precision, double target_ms, double *tflops, double *ms, void *stream);

/* Message describing the calling thread's last error ("" if none). */
const char *sph_last_error(void);

/* Library version string. */
const char *sph_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SPH_H */
