/*
 * to.h -- C ABI of the GB300 batched trajectory-optimisation library (libto.so).
 *
 * The library solves many independent instances of the paper's finite-horizon
 * discrete optimal control problem (Sec. II, Eq. 1)
 *
 *     min_{X,U}  sum_{k=0}^{T-1} l_k(x_k, u_k) + l_T(x_T)
 *     s.t.       x_{k+1} = f_k(x_k, u_k),  k = 0..T-1,   x_0 = x_init,
 *
 * one per initial state, with iLQR: a DDP backward pass without second-order
 * dynamics terms whose value gradient V_x is also returned (Sec. II), Cholesky
 * of Q_uu with the LM term Q_uu + mu I only as a guard (Sec. IV-B),
 * eigenvalue clipping of the state- and control-cost Hessians,
 * S' = max(S, eps), Q_psd = sym(W diag(S') W^T) (Sec. IV-B), a parallel line
 * search over step sizes alpha_j = decay^j, and a fixed per-instance iteration
 * budget (Sec. IV-A).  The warm start is zero controls, caller-given controls,
 * or the actor policy rolled out through the dynamics (Sec. II).  The control
 * bound |u| <= u_max of Eq. 1 is not supported (u_max must be +inf).
 *
 * Conventions
 *   - Every function returns TO_OK (0) or a negative TO_ERR_* code; the
 *     message of the last error on the calling thread is tolast_error().
 *   - Host arrays are instance-major, row-major, float64.  The caller owns
 *     every host pointer; the library copies what it needs before returning
 *     (or, for asynchronous calls, before the call's stream work starts).
 *   - The library owns all device memory it allocates; tofree_batch and
 *     todestroy_problem release it.  Device pointers passed in by the caller
 *     stay owned by the caller.
 *   - Per-instance outcomes are reported in status[], not in return codes.
 *   - Horizons shorter than T_max are padded in outputs: U with 0, X with x_T
 *     repeated, V_x with 0.
 *   - The library is single-GPU: every call runs on the device current on the
 *     calling thread when the problem was created.
 */
#ifndef TO_H
#define TO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct to_problem_s* to_problem;
typedef struct to_batch_s* to_batch;

/* systems (Sec. V-A: point mass, manipulators; Sec. V-D: quadruped-shaped) */
enum {
  TO_SYS_POINTMASS2D = 1, /* n=4 [px,py,vx,vy], m=2, explicit Euler              */
  TO_SYS_PLANAR3 = 2,     /* planar 3-link arm, n=6, m=3, semi-implicit Euler     */
  TO_SYS_ARM7 = 3,        /* 7-DoF serial arm, n=14, m=7, semi-implicit Euler     */
  TO_SYS_QUAD18 = 4,      /* 6 virtual base joints + 4x3 legs, n=36, m=12, contact */
  TO_SYS_DUBINS = 5       /* jerk-controlled Dubins car, n=5, m=2, explicit Euler  */
};

/* arithmetic of the solve */
enum {
  TO_FP64 = 0, /* every step in float64                                        */
  TO_MIXED = 1 /* float32 rollouts, derivatives and Riccati products; the
                  Q_uu Cholesky in float32 when every pivot exceeds 2^-10 of
                  the largest diagonal entry (groups of 2 to 31 lanes,
                  clipped Hessians), else in float64 with the pivot test;
                  float64 line-search cost comparison; the refinement
                  residual of the gain solve and the cost accumulation are
                  float-float (about 48 significant bits)                     */
};

/* return codes */
enum {
  TO_OK = 0,
  TO_ERR_ARG = -1,      /* malformed argument (message says which)            */
  TO_ERR_CUDA = -2,     /* a CUDA runtime call failed                         */
  TO_ERR_BUDGET = -3,   /* request exceeds the HBM budget / batch capacity    */
  TO_ERR_TIMEOUT = -4,  /* a bounded wait ran out                             */
  TO_ERR_NOTREADY = -5, /* result not available yet (serving)                 */
  TO_ERR_UNSUPPORTED = -6
};

/* per-instance status (low 4 bits) and flags */
enum {
  TO_ST_CONVERGED = 1, /* relative cost decrease fell below tol_rel             */
  TO_ST_MAX_ITER = 2,  /* iteration budget used (or forced sequence ended)      */
  TO_ST_LS_FAIL = 3,   /* no step size decreased the cost; iterate kept         */
  TO_ST_NONFINITE = 4, /* the cost or a Cholesky became non-finite              */
  TO_ST_TIMEOUT = 5,   /* a bounded device wait ran out                         */
  TO_ST_FLAG_REG = 16  /* some Q_uu failed the pivot test and got mu I added    */
};

/*
 * Problem description.  params is the flat float64 vector of the system:
 *
 * TO_SYS_POINTMASS2D:
 *   [0] dt  [1] w_u  [2] bump amplitude  [3] bump sigma  [4] nb (<= 8)
 *   [5 .. 5+2nb) bump centres (x, y)  [5+2nb] w_pT  [6+2nb] w_vT
 *   l_k = w_u |u|^2 + sum_b amp exp(-|p - c_b|^2 / (2 sigma^2))
 *   l_T = w_pT |p|^2 + w_vT |v|^2
 *
 * TO_SYS_DUBINS (Sec. V-A's jerk-controlled Dubins car without the time
 * state; x = [px, py, theta, v, a], u = [omega, jerk]):
 *   [0] dt  [1] w_u  [2] bump amplitude  [3] bump sigma  [4] nb (<= 8)
 *   [5 .. 5+2nb) bump centres  [5+2nb] w_pT  [6+2nb] w_vT  [7+2nb] w_aT
 *   px+ = px + dt v cos(theta), py+ = py + dt v sin(theta),
 *   theta+ = theta + dt omega, v+ = v + dt a, a+ = a + dt jerk
 *   l_k = w_u |u|^2 + sum_b amp exp(-|p - c_b|^2 / (2 sigma^2))
 *   l_T = w_pT |p|^2 + w_vT v^2 + w_aT a^2
 *
 * Rigid-body systems (TO_SYS_PLANAR3, TO_SYS_ARM7, TO_SYS_QUAD18):
 *   header  [0] dt  [1..3] gravity vector (world)  [4] N joints  [5] a0 (first
 *           actuated joint; m = N - a0)  [6] n_sub (semi-implicit Euler
 *           substeps of dt/n_sub per knot, 0 means 1)  [7] 0
 *   body i  at 8 + 16 i: [0] parent (-1 root) [1] joint type (0 Rx, 1 Ry,
 *           2 Rz, 3 Px, 4 Py, 5 Pz) [2..4] joint offset in the parent frame
 *           [5] mass [6..8] centre of mass [9..11] diagonal inertia about the
 *           centre of mass [12..15] 0
 *   cost block at C = 8 + 16 N:
 *   PLANAR3 (gravity in the xy plane, joints Rz, links along +x):
 *     [C] w_tau [C+1] bump amplitude [C+2] sigma [C+3] nb (<= 2)
 *     [C+4..7] bump centres [C+8..9] target [C+10] w_ee [C+11] w_vT
 *     [C+12] end-effector body [C+13..15] end-effector point in that body
 *     l_k = w_tau |u|^2 + sum_b amp exp(-|ee(q) - c_b|^2 / (2 sigma^2))
 *     l_T = w_ee |ee(q) - target|^2 + w_vT |qd|^2
 *   ARM7 (the device model is compiled for this tree: a chain, body i the
 *     child of body i-1, joints Rz Ry Rz Ry Rz Ry Rz; other trees are
 *     rejected with TO_ERR_ARG):
 *     [C] w_tau [C+1] w_v [C+2..4] target [C+5] w_ee [C+6] w_vT
 *     [C+7] end-effector body (6) [C+8..10] end-effector point
 *     l_k = w_tau |u|^2 + w_v |qd|^2,  l_T = w_ee |ee(q) - target|^2 + w_vT |qd|^2
 *   QUAD18 (compiled for this tree, others rejected with TO_ERR_ARG: base
 *     joints Px Py Pz Rz Ry Rx as the chain of bodies 0..5, then four legs
 *     of three bodies each -- hip Rx on body 5, thigh Ry, calf Ry -- with
 *     foot f on the calf, body 8 + 3 f):
 *     [C] w_tau [C+1] z_nom [C+2] w_z [C+3] w_rpy [C+4] w_vx [C+5] vx target
 *     [C+6] terminal scale [C+7] contact stiffness k [C+8] damping d
 *     [C+9] softplus beta [C+10] n_feet (4) then per foot: body, point (3)
 *     contact force at each foot (world): F_z = k softplus_beta(-z)
 *       - d sigmoid(-beta z) zdot,  F_xy = -d sigmoid(-beta z) pdot_xy
 *     l_k = w_z (z - z_nom)^2 + w_rpy |(yaw,pitch,roll)|^2 + w_vx (xdot - vx*)^2
 *           + w_tau |u|^2,   l_T = scale * (state terms of l_k)
 *
 * actor_w (optional, float32): W1[256x36] b1[256] W2[256x256] b2[256]
 * W3[12x256] b3[12], u = W3 tanh(W2 tanh(W1 x + b1) + b2) + b3; only
 * TO_SYS_QUAD18 accepts it.  NULL selects the zero-control warm start.
 */
typedef struct {
  int sys;
  int n, m;          /* must match the system                                 */
  int T_max;         /* largest horizon any solve of this problem will use    */
  double dt;         /* must equal params[0]                                  */
  const double* params;
  size_t n_params;
  const float* actor_w;
  size_t n_actor_w;
  double u_max;      /* must be +inf                                          */
} to_problem_desc;

typedef struct {
  int max_iter;           /* iteration budget per instance (Sec. IV-A)         */
  double tol_rel;         /* stop when (J_old - J_new) / |J_old| < tol_rel     */
  double eps_clip;        /* eigenvalue floor eps (Sec. IV-B)                  */
  int n_alpha;            /* number of step sizes L (1..32)                    */
  double alpha_decay;     /* alpha_j = alpha_decay^j                           */
  int prec;               /* TO_FP64 or TO_MIXED                               */
  int refine;             /* mixed mode: one refinement step of the gain solve
                             with the residual formed in float-float (1: exact
                             FMA products, compensated sum, ~48 bits) or in
                             native float64 (2); 0 = none                     */
  const int* forced_alpha;/* test hook, host B x max_iter or NULL: iteration i of
                             instance b takes step index forced_alpha[b*max_iter+i]
                             with no test; -1 ends that instance's run          */
  int want_vx;            /* 1: one more backward pass at the returned iterate
                             gives V_x and the gains K, k there                */
  size_t hbm_budget_bytes;/* 0 = no limit; else tocreate_batch / tosolve_batch
                             refuse a workspace larger than this (TO_ERR_BUDGET) */
  int group_lanes;        /* threads per instance, one of the system's supported
                             sizes (1/8/16/32 point mass and Dubins car,
                             1/4/8/16/32 planar arm, 32 arm, 64/32
                             quadruped); 0 = the totune
                             choice, else the system's default.  1: one thread
                             per instance with every per-knot matrix in
                             registers; its line search tries one step size
                             at a time (the smallest j first), the others
                             min(group_lanes, 16) at once                     */
  int groups_per_block;   /* instances resident per CTA (group_lanes x
                             groups_per_block <= 256, a multiple of 32);
                             0 = the totune choice, else the default (64
                             threads per CTA for a non-default group size)   */
  int profile_phases;     /* 1: accumulate per-phase clock64 cycles (tracing;
                             see toget_phase_cycles); 0 = off                 */
  int reg;                /* TO_REG_CLIP (default): eigenvalue clipping of the
                             cost Hessians, mu I only as a Cholesky guard
                             (Sec. IV-B, the paper's GPU choice);
                             TO_REG_LM: the standard Levenberg-Marquardt
                             iLQR the paper compares against (Sec. IV-B):
                             no clipping, Q_uu + mu I with mu = 1e-6 at the
                             start, x10 and the backward pass redone when
                             the pivot test or the line search fails, /10
                             (not below 1e-8) after an accepted step;
                             mu > 1e10 stops the instance with LS_FAIL.
                             eps_clip is ignored                              */
  int stage_depth;        /* knots of look-ahead with which a group fetches
                             what it reads next (the backward pass's knot
                             record or stored derivative block, the forward
                             pass's record and gains) into registers: 1 or 2
                             (2 only where the system offers it: the planar
                             arm's groups of 4 or more lanes; else
                             TO_ERR_ARG); 0 = the totune choice, else 1.
                             The arithmetic is the same at every depth:
                             results agree to the rounding of the compiler's
                             multiply-add fusion, which may differ between
                             kernel instantiations                            */
} to_solver_opts;

/* to_solver_opts.reg */
enum { TO_REG_CLIP = 0, TO_REG_LM = 1 };

/* Defaults: max_iter 100, tol_rel 1e-8, eps_clip 1e-8, n_alpha 16,
 * alpha_decay 0.5, TO_MIXED, refine 1, no forcing, want_vx 0, no budget,
 * autotuned launch shape and staging depth. */
void to_default_opts(to_solver_opts* opts);

/* One instance family of the OCP of Sec. II, Eq. 1: the system's dynamics
 * f_k, running cost l_k and terminal cost l_T (params), the horizon bound
 * T_max and, optionally, the actor policy whose rollout is the warm start
 * (Sec. II; Sec. III-D for the policy's use as initial guess).
 * Validate the description, parse params into the system's device layout and
 * upload it (plus the actor weights).  Errors: TO_ERR_ARG (shape, layout or a
 * system whose joint structure the GPU model does not cover), TO_ERR_CUDA. */
int tocreate_problem(const to_problem_desc* desc, to_problem* out);
void todestroy_problem(to_problem p);

/* Allocate the device workspace of a batch able to hold B_max instances whose
 * horizons sum (over T+1) to at most knots_max.  Per knot it holds the knot
 * records of min(group_lanes, 16) + 1 trajectory slots, the gain record and,
 * for the planar arm and the rigid trees, a derivative scratch (the planar
 * arm's stored derivative block, 108 elements; the rigid trees' n_sub stored
 * substep primals, about 6 KB each in float32 for the quadruped); elements
 * are float64 or float32 by opts->prec.  Reusing one batch object for many
 * solves keeps allocation out of the solve.  Errors: TO_ERR_ARG,
 * TO_ERR_BUDGET (workspace above opts->hbm_budget_bytes), TO_ERR_CUDA. */
int tocreate_batch(to_problem p, int B_max, long long knots_max, const to_solver_opts* opts, to_batch* out);
void tofree_batch(to_batch b);

/* Solve B instances of Eq. 1 (Sec. II), one per initial state x_init, with
 * the iLQR iteration of Sec. II and Sec. IV-B (backward pass with clipped cost
 * Hessians and the Q_uu Cholesky, then the line search) under the
 * per-instance iteration budget of Sec. IV-A; the batched form is the paper's
 * TO of many problems at once on the GPU (Sec. IV).
 * x0: host B x n; T: host B horizons in [1, T_max];
 * U_init: host B x T_max x m initial controls or NULL (zero controls, or the
 * actor warm start when the problem has actor weights).  The work is enqueued
 * on cuda_stream (a cudaStream_t, NULL = the legacy default stream) and the
 * call returns once the host inputs are copied.  If *out is NULL a batch sized
 * for this call is created and returned; otherwise *out is reused and must
 * have enough capacity.  Errors: TO_ERR_ARG, TO_ERR_BUDGET, TO_ERR_CUDA. */
int tosolve_batch(to_problem p, int B, const double* x0, const int* T, const double* U_init,
                  const to_solver_opts* opts, void* cuda_stream, to_batch* out);

/* Same solve with inputs already in device memory: d_x0 (B x n float64),
 * d_T (B int32, each in [1, T_max]), d_U_init (B x T_max x m float64 or NULL),
 * d_forced (B x max_iter int32 or NULL; replaces opts->forced_alpha).  Sum of
 * (T+1) must not exceed the batch's knots_max (checked on the device: an
 * overflowing solve marks every instance TO_ST_NONFINITE and computes
 * nothing).  Nothing is copied between host and device. */
int tosolve_batch_device(to_batch b, int B, const double* d_x0, const int* d_T, const double* d_U_init,
                         const int* d_forced, const to_solver_opts* opts, void* cuda_stream);

/* The solution of the last solve (Sec. II): the optimised trajectories X, U
 * and final cost J of Eq. 1, and, with want_vx, the value gradient V_x of the
 * DDP backward pass at the returned iterate and its feedback gains K, the
 * outputs the paper hands to critic training (Sec. II).
 * Copy results of the last solve to the host (synchronises the batch's
 * stream).  X: B x (T_max+1) x n, U: B x T_max x m, J, iters, status: B;
 * Vx: B x (T_max+1) x n and K: B x T_max x m x n (need want_vx; may be NULL);
 * any output pointer may be NULL.  T_max is the problem's. */
int toget_trajectories(to_batch b, double* X, double* U, double* J, int* iters, int* status, double* Vx,
                       double* K);

/* Several systems in one persistent launch (spec batching pattern:
 * uneven horizons and systems share one launch; the paper batches one
 * system at a time, Sec. IV).  batches[i] (one per problem, each of a
 * different system among the 7-DoF arm, the planar arm and the point mass)
 * solves Bs[i] instances from device inputs d_x0[i] (Bs[i] x n float64) and
 * d_T[i] (Bs[i] int32 in [1, T_max]), with one option set (no forced steps,
 * want_vx, profiling or launch shape).  One horizon sort per member, then a
 * single kernel in which every CTA serves the 7-DoF arm's queue, then the
 * planar arm's, then the point mass's: a CTA that drains one system moves on
 * to the next while others still solve the previous one.  Each member's
 * arithmetic is its own solver's; results are read per batch with
 * toget_trajectories.  Errors: TO_ERR_ARG, TO_ERR_UNSUPPORTED (another
 * system, a repeated system, an unsupported option), TO_ERR_CUDA. */
int tosolve_systems(const to_batch* batches, const int* Bs, const double* const* d_x0, const int* const* d_T, int n,
                    const to_solver_opts* opts, void* cuda_stream);

/* Per-iteration record of the last solve: accepted step index (B x max_iter,
 * -1 after the last iteration) and cost (B x (max_iter+1), J_hist[b][0] is the
 * warm-start cost).  Either pointer may be NULL. */
int toget_history(to_batch b, int* alpha_idx, double* J_hist);

/* Critic targets of the last solve (Sec. II: for every state of every
 * optimised trajectory, the partial K-step cost-to-go that, with V_x from the
 * DDP backward pass, trains the critic):
 *     Vbar[b][k] = sum_{j=k}^{min(k+K, T_b)-1} l_j(x_j, u_j) + [k + K >= T_b] l_T(x_T)
 * for k = 0..T_b (the terminal knot gets l_T alone), 0 for k > T_b; the
 * state K steps ahead is X[b][min(k+K, T_b)].  Evaluated on the device in
 * float64 from the returned trajectories (one pass over the knots, then the
 * window sums).  Vbar: host B x (T_max+1).  V_x comes from
 * toget_trajectories of a solve with want_vx.  Synchronises the batch's
 * stream.  Errors: TO_ERR_ARG (K < 1, no solve), TO_ERR_CUDA. */
int toget_critic_targets(to_batch b, int K, double* Vbar);

/* Device-resident results of the last solve (no copy): J (float64, B),
 * iters and status (int32, B), in the batch's own memory. */
int toget_device_results(to_batch b, const double** d_J, const int** d_iters, const int** d_status);

/* Tracing: SM cycles the last solve (run with profile_phases = 1) spent per
 * phase, summed over warps: [0] queue / bookkeeping, [1] backward: knot
 * staging + derivatives, [2] backward: V A, V B and the Q terms, [3] backward:
 * Cholesky + gain solve, [4] backward: value update, [5] forward rounds
 * (parallel line search, warm-start rollout), [6] 0, [7] total.  out must
 * hold 8 values. */
int toget_phase_cycles(to_batch b, unsigned long long* out);

/* Number of kernels the last tosolve_batch / tosolve_batch_device launched. */
int tolast_launch_count(to_batch b);

/* Bounds-checked build.  The library built with -DTO_CHECKED (nvcc_build
 * checked=True: _lib/libto_checked.so; the Python binding loads it when the
 * environment sets TO_CHECKED=1) checks every computed index of the solver
 * kernel against the buffer it addresses: the instance index against the
 * batch (or the server's seats), the horizon against [1, T_max], every knot
 * record, gain record, V_x row and derivative-scratch row against the
 * batch's knot capacity, the trajectory slot against the line-search width,
 * and the iteration index of the step-size history, the forced sequence and
 * the caller's warm start against their sizes.  A violation is recorded per
 * problem and the access goes to the buffer's first element instead; the
 * solve's results are then meaningless, but nothing is read or written
 * outside an allocation.  The release build compiles the checks away.
 *
 * tobounds_checked: 1 in the checked build, 0 in the release build.
 * toget_bounds_report: after synchronising the device, out4 receives the
 * problem's report since its creation (or the last reset): [0] the number of
 * violations, [1] the first one's site (1 instance index, 2 serving seat,
 * 3 horizon, 4 knot record, 5 trajectory slot, 6 gain record, 7 V_x row,
 * 8 derivative scratch, 9 forced step, 10 warm start, 11 history), [2] its
 * index, [3] the limit it broke.  reset != 0 zeroes the report afterwards.
 * TO_ERR_UNSUPPORTED in the release build. */
int tobounds_checked(void);
int toget_bounds_report(to_problem p, long long* out4, int reset);

/*
 * Serving: continuous batching of single OCP requests (the paper's real-time
 * use, Sec. V-D).  A server holds, per problem, a pool of seats -- one
 * instance workspace each, as many as hbm_budget_bytes (split evenly over the
 * problems; 0 = 4 GiB) holds -- and a persistent solver kernel per problem
 * that takes newly published requests into free seats at every iteration
 * boundary, so requests arriving while others are on the GPU start at once
 * and overlap with them.  Trajectories and gains stay on the device.  Every
 * device wait is bounded: a kernel with nothing to do for ~1 ms leaves and
 * the next tosubmit / topoll relaunches it.  Each problem's kernel takes an
 * equal share of the GPU's resident CTAs.  opts applies to every request
 * (forced_alpha, want_vx and profile_phases are ignored).
 */
typedef struct to_server_s* to_server;
int toserver_create(const to_problem* problems, int n_problems, const to_solver_opts* opts, size_t hbm_budget_bytes,
                    to_server* out);
void toserver_destroy(to_server s);

/* Admit one request for problems[problem] (x0: host n float64, T in
 * [1, T_max]).  TO_ERR_BUDGET when no seat is free: poll and retry.  The
 * request id is valid until topoll returns TO_OK for it. */
int tosubmit(to_server s, int problem, const double* x0, int T, uint64_t* req_id);

/* TO_ERR_NOTREADY while the request runs; else its results (any pointer may
 * be NULL; X: (T_max+1) x n, U: T_max x m, padded like toget_trajectories),
 * latency_ms = time from tosubmit to completion seen by this call, and the
 * seat is freed. */
int topoll(to_server s, uint64_t req_id, double* X, double* U, double* J, int* iters, int* status,
           double* latency_ms);

int toserver_stats(to_server s, int* seats_total, int* seats_busy, long long* completed, size_t* hbm_bytes);

/* Replay a request trace in real time on the calling thread: request i
 * arrives arrival_s[i] seconds after the call (sorted ascending), for
 * problems[problem[i]] with horizon T[i] and initial state x0 + i*x0_stride.
 * Requests wait (in arrival order) for a free seat.  latency_ms[i] is the time
 * from the scheduled arrival to the result; J and status may be NULL.
 * TO_ERR_TIMEOUT if the trace is not done after timeout_s seconds. */
int toserve_replay(to_server s, int n_req, const double* arrival_s, const int* problem, const int* T,
                   const double* x0, int x0_stride, double* latency_ms, double* J, int* status, double timeout_s);

/*
 * Solve without allocating device memory.  The paper has no counterpart:
 * this is for callers that cannot call cudaMalloc while they run -- a
 * real-time control loop whose latency must stay bounded, code confined to a
 * fixed, pre-sized memory pool, or code running while other work is being
 * captured into a CUDA graph.
 *
 * The workspace comes from one static device array of
 * TO_NOALLOC_SCRATCH_BYTES (64 MiB) inside the library; every GPU that loads
 * the library holds it until the process exits.  It must fit
 * B * (T_max + 1) knot records of the problem plus per-instance bookkeeping;
 * a larger request returns TO_ERR_BUDGET and launches nothing.  Inputs and
 * outputs are the caller's device buffers: d_x0 (B x n float64), d_T (B int32
 * in [1, T_max]); d_J (B float64), d_iters, d_status (B int32); d_X
 * (B x (T_max+1) x n float64) and d_U (B x T_max x m float64) may be NULL.
 * opts may not set forced_alpha, want_vx or profile_phases
 * (TO_ERR_UNSUPPORTED).  The work is enqueued on cuda_stream; results are
 * ready when the stream reaches them.  A horizon outside [1, T_max] is found
 * on the device (the host never reads d_T): then every instance gets
 * TO_ST_NONFINITE, d_J is NaN, d_X and d_U (if given) are NaN, and nothing
 * else is computed.  The call must come from the device the problem was
 * created on (TO_ERR_ARG otherwise).
 *
 * The first call on each device looks up the array's device address (with
 * that device current), so make that first call before any stream capture.
 * Every call shares the one array: calls whose work overlaps on the GPU (two
 * streams, two host threads) race and corrupt each other; serialise them.
 */
#define TO_NOALLOC_SCRATCH_BYTES (64u << 20)
int tosolve_batch_noalloc(to_problem p, int B, const double* d_x0, const int* d_T, const to_solver_opts* opts,
                          void* cuda_stream, double* d_J, int* d_iters, int* d_status, double* d_X, double* d_U);

/*
 * Launch-shape autotuner.  The solver kernel's shape -- threads per instance
 * (group_lanes, from the system's supported set), instances per CTA
 * (groups_per_block) and the staging depth (stage_depth, where the system
 * offers more than one) -- trades per-instance parallelism against
 * occupancy, register pressure and load latency, and the best point differs
 * per system and precision.  totune times every valid shape on a calibration batch (host
 * x0: B x n, T: B; solved with *opts, whose max_iter may be smaller than the
 * production one) with CUDA events on a stream of its own, after one untimed
 * warm-up solve per shape.  The fastest shape is written into
 * opts->group_lanes / groups_per_block / stage_depth and cached in the
 * problem for opts->prec: later solves that leave all three at 0 use it.  rows (may be NULL)
 * receives up to max_rows measured shapes; *n_rows how many were measured.
 * The calibration batch should fill the GPU (several instances per SM) so
 * the choice holds for large batches.  With the environment variable
 * TO_TUNE_CACHE naming a file, the choice is also appended to that file and
 * a later call with the same key (system, sizes, T_max, batch size and mean
 * horizon in powers of two, precision, LM mode, GPU name and SM count, the
 * library's build time) takes it from there without timing: *n_rows is then
 * 1 and rows[0] the stored shape.  Errors: TO_ERR_ARG, TO_ERR_CUDA.
 */
typedef struct {
  int group_lanes, groups_per_block;
  int grid;               /* CTAs launched                                     */
  int ctas_per_sm;        /* resident CTAs per SM at this shape                */
  double ms;              /* device time of one solve of the calibration batch */
  int stage_depth;        /* staging depth of this shape                       */
} to_tune_row;
int totune(to_problem p, int B, const double* x0, const int* T, to_solver_opts* opts, to_tune_row* rows,
           int max_rows, int* n_rows);

/*
 * CUDA-graph solves of a multi-system batch.  One graph replays the whole
 * solve of n member batches (one per problem, member i solving B[i]
 * instances): per member, the host-to-device copies of x0 and T from pinned
 * staging that the graph owns, the horizon sort, the persistent solver
 * kernel, the gather of X and U (when want_traj) and the device-to-host
 * copies of X, U, J, iters and status into pinned staging.  The members'
 * branches are independent, so their kernels run at the same time, each
 * sized to its share of the resident CTAs (shares[i] / sum(shares); shares
 * NULL = equal).  Horizons may change between launches (the sort runs on the
 * device); B, the options and the member batches are fixed at capture.
 * opts may not set forced_alpha, want_vx or profile_phases
 * (TO_ERR_UNSUPPORTED).  The member batches must outlive the graph and must
 * not be used by other solves while a launch is in flight.
 */
typedef struct to_graph_s* to_graph;
int tograph_create(const to_batch* batches, const int* B, const double* shares, int n, const to_solver_opts* opts,
                   int want_traj, to_graph* out);
/* Pinned staging of member i: inputs to fill before tograph_launch (x0:
 * B x n, T: B) and outputs valid after tograph_sync (X: B x (T_max+1) x n and
 * U: B x T_max x m, NULL without want_traj; J, iters, status: B).  Any output
 * pointer argument may be NULL. */
int tograph_staging(to_graph g, int member, double** x0, int** T, double** X, double** U, double** J, int** iters,
                    int** status);
/* Enqueue one replay on cuda_stream (NULL = the graph's own stream). */
int tograph_launch(to_graph g, void* cuda_stream);
/* Wait for the last replay. */
int tograph_sync(to_graph g);
/* Kernels one replay launches. */
int tograph_launch_count(to_graph g);
void tograph_destroy(to_graph g);

/*
 * Biased-initial-condition ranking (Sec. III-C/D): from the second CACTO
 * iteration on, 10N candidate initial states are scored by the std-critic
 * network V^std (the predicted standard deviation of the critic) and the N
 * highest start the next TO batch.  The std-critic here is an MLP
 * n_in -> 256 -> 256 -> 1 with tanh hidden layers and a softplus output;
 * weights (float32, row-major out x in): W1[256 x n_in] b1[256]
 * W2[256 x 256] b2[256] W3[1 x 256] b3[1]; 1 <= n_in <= 64.
 * torank_candidates scores the C candidates x (host, C x n_in float64) on
 * the device in float32 and writes the indices of the N largest scores to
 * top_idx (host, N, ascending index order; a score tied with the N-th
 * largest is taken by the lower index; a non-finite score ranks last);
 * scores (host, C float32) may be NULL.  Synchronises cuda_stream.
 * Errors: TO_ERR_ARG (sizes, 1 <= N <= C), TO_ERR_CUDA.
 */
typedef struct to_ranker_s* to_ranker;
int toranker_create(int n_in, const float* weights, size_t n_weights, to_ranker* out);
int torank_candidates(to_ranker r, int C, const double* x, int N, int* top_idx, float* scores, void* cuda_stream);
void toranker_destroy(to_ranker r);

const char* tolast_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TO_H */
