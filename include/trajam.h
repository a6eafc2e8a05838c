/*
 * trajam: batched multi-convex trajectory optimization on B300 (sm_103a).
 *
 * C ABI of the alternating-minimization (AM) loop of "GPU Accelerated Batch
 * Multi-Convex Trajectory Optimization for a Rectangular Holonomic Mobile
 * Robot" (arXiv 2109.13030).  One handle describes one planning problem
 * (Sec. II-B, Eq. acc_cost - coll_multiagent): a horizon of q steps over T
 * seconds, a robot covered by m circles at body offsets r_i, n axis-aligned
 * elliptical obstacles with tracks x_j(t), y_j(t), and boundary conditions
 * shared by every trajectory of the batch.  A solve runs the AM iteration of
 * Sec. III-D on B trajectories at once, each started from its own initial
 * coefficients.
 *
 * Conventions
 *  - Every function returns AM_OK (0) or a negative AM_ERR_* code and never
 *    throws; am_last_error() gives a message for the calling thread.
 *  - The library keeps no caller pointer after a call.  An argument named
 *    `mem` says whether the caller's buffers are host (AM_HOST) or device
 *    (AM_DEVICE) memory; host buffers should be pinned for speed.  Inputs
 *    are read in stream order: a device buffer or a pinned host buffer
 *    passed to a call that queues work must stay unchanged until the stream
 *    has reached that work (a pageable host buffer is read before the call
 *    returns).
 *  - The handle owns all of its device memory.  Calls on one handle must not
 *    run concurrently from several host threads.
 *  - Work is queued on the CUDA stream passed to am_solve_batch (NULL = the
 *    legacy default stream); getters wait for that stream with a bounded
 *    wait (AM_ERR_TIMEOUT after 60 s).
 *  - Coefficients are degree-10 Bernstein control points (11 per polynomial)
 *    on t in [0, T], sampled at t_k = k T / (q - 1), k = 0..q-1 (Eq. param).
 *
 * Per-trajectory state layout (AM_STATE_FLOATS = 110 floats):
 *    [ 0, 44)  xi1 = (c_x, c_c, c_y, c_s)   Eq. reform_cost
 *    [44, 55)  xi2 = c_psi
 *    [55, 99)  lambda                        Table I
 *    [99,110)  lambda_psi
 */
#ifndef TRAJAM_H
#define TRAJAM_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define AM_API __attribute__((visibility("default")))
#else
#define AM_API
#endif

#define AM_OK 0
#define AM_ERR_ARG (-1)     /* invalid argument; nothing was changed        */
#define AM_ERR_CUDA (-2)    /* a CUDA call failed                            */
#define AM_ERR_BUDGET (-3)  /* device memory budget exceeded                 */
#define AM_ERR_TIMEOUT (-4) /* a bounded wait expired                        */
#define AM_ERR_NAN (-5)     /* the solve produced a non-finite value         */
#define AM_ERR_STATE (-6)   /* call out of order (e.g. solve before obstacles) */

#define AM_HOST 0
#define AM_DEVICE 1

/* Precision of the fused kernel's tensor-core contraction over the time grid
 * (R = F^T (g - F xi1)): AM_FP32 takes three TF32 products per product
 * (hi*hi + hi*lo + lo*hi, FP32 accuracy); AM_TF32 and AM_BF16 take one
 * product of operands rounded to TF32 or BF16 (the reduced-precision form);
 * AM_SPLIT_BF16 splits each operand into BF16 hi + lo (16 significant bits)
 * and takes three BF16 products of K = 16 (half the tensor-core
 * instructions of AM_FP32).  The position and heading steps are FP32 in
 * every form.  Groups run each problem in its own precision; the plain
 * kernel and the allocation-free entry run FP32 only. */
#define AM_FP32 0
#define AM_TF32 1
#define AM_BF16 2
#define AM_SPLIT_BF16 3

#define AM_KERNEL_FUSED 0   /* one launch runs every iteration (default)     */
#define AM_KERNEL_PLAIN 1   /* one launch per step, intermediates in memory  */
#define AM_KERNEL_LARGE 2   /* fused, 128 trajectories per CTA on tcgen05    */
#define AM_KERNEL_WARP 3    /* fused, two warps per trajectory, no block     */
                            /* barriers in the loop                          */
#define AM_KERNEL_AUTO 4    /* the fastest of the three fused kernels that   */
                            /* takes the problem (see AM_OPT_KERNEL)         */

#define AM_NV 11
#define AM_STATE_FLOATS 110
#define AM_MAX_Q 256
#define AM_MAX_M 4
#define AM_MAX_N 64

typedef struct am_problem am_problem;

typedef struct {
    int q;                 /* planning steps, 2..AM_MAX_Q                     */
    double T;              /* horizon in seconds, > 0                         */
    int degree;            /* Bernstein degree; must be 10                    */
    int m;                 /* robot circles, 1..AM_MAX_M                      */
    const double *r;       /* m body offsets r_i of the circle centres        */
    double r_c;            /* circle radius, added to every obstacle semi-axis */
    double v_max, a_max;   /* speed and acceleration bounds (Eq. acc_constraint) */
    double rho, rho_psi;   /* penalty weights (Eq. reform_bergman, update_lambda_psi) */
    double x_bc[6], y_bc[6], psi_bc[6];  /* value, 1st, 2nd derivative at t = 0, then at t = T */
    int precision;         /* AM_FP32 | AM_TF32 | AM_BF16                    */
    int alpha_mode;        /* 0: alpha = atan2(a yt, b xt); 1: atan2(yt, xt) */
    int psi_dual_sign;     /* 0: lam_psi -= rho_psi P^T (P xi2 - psi_t); 1: opposite */
    int cs_boundary;       /* 1: slack polynomials c, s carry boundary rows  */
} am_problem_desc;

/* Create a handle: builds the Bernstein basis, the boundary matrix A and the
 * constant parts of both KKT systems in FP64 on the host (Eq. over_1 - over_3,
 * zeta_1_sepration_3, compute_convex_surrogate).  The first CUDA call of the
 * process happens here, on the current device. */
AM_API int am_init_problem(const am_problem_desc *desc, am_problem **out);

/* Set the n obstacles (0 <= n <= AM_MAX_N): centre tracks xo, yo of n x q
 * floats (row j = obstacle j over the q steps) and semi-axes a, b of n floats
 * each, before inflation by r_c (Eq. coll_multiagent).  Re-forms the position
 * KKT inverse when n changes, since F^T F depends on n (Sec. IV-E). */
AM_API int am_set_obstacles(am_problem *h, int n, const float *xo, const float *yo, const float *a,
                     const float *b, int mem);

/* Replace the shared boundary conditions (the MPC re-plan of Sec. IV). */
AM_API int am_set_boundary(am_problem *h, const double x_bc[6], const double y_bc[6],
                    const double psi_bc[6]);

/* Run `iters` (>= 1) AM iterations on B (>= 1) trajectories.
 *  init         B x 3 x 11 floats: c_x, c_y, c_psi per trajectory (cold start,
 *               multipliers zero unless warm_lambda is given); NULL continues
 *               from the state the handle holds (warm start, same B).
 *  warm_lambda  NULL, or B x 55 floats: lambda (44) then lambda_psi (11).
 *  stream       cudaStream_t the work is queued on.
 * Results stay on the device until read with the getters. */
AM_API int am_solve_batch(am_problem *h, int B, const float *init, const float *warm_lambda, int iters,
                   void *stream, int mem);

/* Per-trajectory results of the last solve, each B floats (NULL to skip):
 * final residual ||F xi1 - g||_2, heading residual ||P xi2 - psi_t||_2, cost
 * sum_t xdd^2 + ydd^2 + psidd^2 (Eq. acc_cost), and the smallest ellipse
 * distance sqrt(xt^2/a^2 + yt^2/b^2) over circles, obstacles and steps.
 * Host outputs wait for the handle's stream.  When all four go to host
 * memory (and 4 B <= 2^22) they arrive through one copy into a pinned area
 * the handle allocates on first use and keeps; otherwise one copy per array. */
AM_API int am_get_results(am_problem *h, float *res, float *res_psi, float *cost, float *mind, int mem);

/* The best trajectory of the last solve: lowest cost among those whose
 * smallest ellipse distance is >= 0.99, else lowest cost overall; ties go to
 * the lower index (Fig. 1's best-cost trajectory).  coeffs gets c_x, c_y,
 * c_psi (33 floats, host memory).  Trajectories with a non-finite cost rank
 * last; when every one is non-finite the outputs are filled and the call
 * returns AM_ERR_NAN.  (Host inputs with a non-finite value are refused with
 * AM_ERR_ARG by am_set_obstacles and am_solve_batch; device inputs are not
 * scanned.) */
AM_API int am_get_best(am_problem *h, float coeffs[33], float *cost, float *residual, int *index);

/* Re-draw the coefficients of the B trajectories the handle holds as the
 * batch initialisation of Sec. IV: samples around the straight line between
 * the handle's current start and goal positions (control points 0..2 at the
 * start, 8..10 at the goal, 3..7 evenly spaced), with the interior points of
 * c_x and c_y perturbed by sigma L z, L the Cholesky factor of the inverse
 * of D2^T D2 restricted to points 3..7 (D2 the second-difference operator on
 * the 11 control points; scaled to a largest standard deviation of 1 m), z
 * standard normal.  c_psi is the straight line between the heading
 * boundary values and the slacks c, s start at cos, sin of its control
 * points.  The multipliers lambda, lambda_psi are kept (the MPC warm start of
 * Sec. IV).  Trajectory 0 takes no perturbation (z = 0), so a batch of one is
 * the straight line.  z comes from a counter-based generator: SplitMix64
 * (Steele, Lea and Flood, 2014) of (seed, trajectory, draw) gives two 53-bit
 * uniforms for one Box-Muller pair, so a seed fixes the draw on any device.
 * Queued on the handle's stream; requires a state (am_init_state or a solve)
 * and sigma finite and >= 0. */
AM_API int am_resample(am_problem *h, unsigned long long seed, float sigma, void *stream);

/* Re-time the B trajectories the handle holds by dt seconds (0 <= dt <= T):
 * each of a trajectory's five polynomials (c_x, c, c_y, s, c_psi) is
 * re-expressed on [dt, dt + T] (past T by extending the same polynomial), so
 * a warm-started re-plan (Sec. IV) continues every plan from where it is dt
 * later.  The new control points are c'_k = f(dt/T repeated 10 - k times,
 * 1 + dt/T repeated k times), f the blossom of the polynomial, evaluated on
 * the host in FP64 by de Casteljau steps; the device applies the resulting
 * 11 x 11 matrix.  The multipliers are kept.  Queued on the handle's stream;
 * requires a state. */
AM_API int am_shift(am_problem *h, double dt, void *stream);

/* Cross-entropy method planner on the handle's problem: the sampling-based
 * comparator of Sec. IV (Table IV; the paper runs it with 8k samples).  The
 * search space is z = control points 3..7 of c_x, c_y and c_psi (the others
 * come from the boundary conditions).  Each iteration draws `samples` z from
 * N(mu, Sigma) (counter-based normals as in am_resample, stream = iteration
 * x 2^24 + sample), scores them with
 *   J = sum_t (x''^2 + y''^2 + psi''^2) + w_coll sum_{t,i,j} max(0, 1 - d_ij)^2
 *       + w_bound sum_t (max(0, |v| - v_max)^2 + max(0, |a| - a_max)^2)
 * (d_ij the ellipse distance of circle i to the inflated obstacle j at step
 * t), and refits mu, Sigma to the `elites` lowest (ties to the lower index):
 * mu <- alpha mean + (1 - alpha) mu, Sigma <- alpha cov + (1 - alpha) Sigma
 * + reg I, cov normalised by the elite count.  Start: mu = the straight line
 * between the boundary positions and headings (or, with warm, control
 * points 3..7 of the plan warm re-timed by warm_dt as in am_shift), Sigma =
 * blockdiag(sigma_xy^2 C, sigma_xy^2 C, sigma_psi^2 C), C the covariance of
 * am_resample.  The result is the lowest J over all iterations.  Bounds:
 * 16 <= samples <= 8192, 2 <= elites <= min(samples, 1024), iters >= 1. */
typedef struct {
    int samples, elites, iters;
    float sigma_xy, sigma_psi;  /* initial spread (m, rad)                     */
    float alpha, reg;           /* smoothing in (0, 1]; covariance floor > 0   */
    float w_coll, w_bound;      /* penalty weights >= 0                        */
    unsigned long long seed;
    const float *warm;          /* nullable: 33 floats (c_x, c_y, c_psi), host */
    double warm_dt;             /* re-timing of warm, 0 <= warm_dt <= T        */
} am_cem_desc;
AM_API int am_cem_solve(am_problem *h, const am_cem_desc *d, void *stream);
/* Best plan of the last am_cem_solve (waits for it): coefficients (33), J and
 * its smallest ellipse distance. */
AM_API int am_cem_get_best(am_problem *h, float coeffs[33], float *cost, float *min_dist);
/* Samples (N x 15) and scores (N) of the last iteration, and mu (15) and
 * Sigma (15 x 15) after its refit (any output may be NULL; host memory). */
AM_API int am_cem_get_samples(am_problem *h, float *z, float *cost, float *mu, float *sigma);
/* Score `count` (1..8192) given plans (count x 33 floats, host) with J above:
 * cost and min_dist get count floats each (host). */
AM_API int am_cem_score(am_problem *h, int count, const float *coeffs, float w_coll, float w_bound,
                        float *cost, float *min_dist);

/* Scale the multipliers lambda, lambda_psi of the B trajectories the handle
 * holds by `factor` (finite, >= 0; 0 resets them), keeping their
 * coefficients: a re-plan that continues the kept plans with the previous
 * window's multipliers decayed.  Queued on the handle's stream; requires a
 * state. */
AM_API int am_scale_multipliers(am_problem *h, float factor, void *stream);

/* Evaluate a plan (c_x, c_y, c_psi: 33 floats, host) of horizon T at `count`
 * times t[i] (clamped to [0, T]): out[9 i ..] = x, x', x'', y, y', y'', psi,
 * psi', psi'' (derivatives in 1/s, 1/s^2; Eq. param).  Host arithmetic in
 * FP64, no device work. */
AM_API int am_plan_eval(const float coeffs[33], double T, int count, const double *t, double *out);

/* The same selection queued on `stream` without a wait: out gets 36 floats
 * {index, cost, residual, c_x, c_y, c_psi} in host (pinned) or device
 * memory when the stream reaches it.  A non-finite out[1] means every
 * trajectory was non-finite (am_get_best reports that as AM_ERR_NAN). */
AM_API int am_get_best_async(am_problem *h, float *out, int mem, void *stream);

/* Copy the B x AM_STATE_FLOATS state out of / into the handle. */
AM_API int am_get_state(am_problem *h, float *out, int mem);
AM_API int am_set_state(am_problem *h, int B, const float *in, int mem);

/* Per-iteration history: when enabled, solves record (res, res_psi, cost)
 * per trajectory and iteration; am_get_history copies B x iters x 3 floats. */
AM_API int am_set_history(am_problem *h, int enable);
AM_API int am_get_history(am_problem *h, float *out, int mem);

/* Options.  AM_OPT_KERNEL: AM_KERNEL_FUSED, AM_KERNEL_PLAIN,
 * AM_KERNEL_LARGE, AM_KERNEL_WARP or AM_KERNEL_AUTO.  AM_KERNEL_LARGE is the batch matrix form of Sec. III-E
 * (Eq. over_3) for large batches: one persistent CTA per SM runs every
 * iteration for tiles of 128 trajectories, with the position step, the
 * trajectory values, P^T delta and R as tcgen05 tensor-core products (three
 * TF32 products each, FP32 accuracy) accumulated in tensor memory.  It takes
 * the FP32 precision form, the default alpha form, q <= 128 and no history;
 * am_solve_batch returns AM_ERR_ARG (nothing launched) for anything else or
 * when the shape's operands exceed the shared memory of an SM.  Results
 * agree with AM_KERNEL_FUSED to FP32 rounding, not bit for bit.
 * AM_KERNEL_WARP runs the same iteration (Sec. III-D, steps 1-5) with two,
 * three or four warps per trajectory (q <= 128, 192, 256) for all
 * iterations: after the constants are staged the warps of a trajectory
 * synchronise only with each other, never with the other trajectories of
 * their CTA, which suits batches of a few trajectories per SM (the paper's
 * B = 1000).  Its contraction R is FP32 SIMT; it takes the FP32 precision
 * form, the default alpha form and cs_boundary (history included), and
 * am_solve_batch returns AM_ERR_ARG (nothing launched) for anything else.  Results agree with
 * AM_KERNEL_FUSED to FP32 rounding, not bit for bit.
 * AM_KERNEL_AUTO picks, per solve, AM_KERNEL_LARGE from B = 16384 on
 * (where it takes the problem), else AM_KERNEL_WARP where it takes the
 * problem, else AM_KERNEL_FUSED, with automatic tiles (AM_OPT_TILE is
 * ignored).  Groups and servers run a problem whose handle selects
 * AM_KERNEL_WARP or AM_KERNEL_AUTO on the warp-pair group kernels when its
 * form and shape fit them, every other problem on the small-tile ones; a
 * problem gives the same bits alone (with the kernel its handle selects
 * for that batch) and in a group.
 * AM_OPT_TILE: trajectories per CTA of the fused kernel (0 = automatic);
 * for AM_KERNEL_WARP, trajectories in flight per CTA: 1..8 for q <= 128,
 * 1..5 for q <= 192, 1..4 for q <= 256 (fewer where shared memory runs
 * out; am_solve_batch returns AM_ERR_ARG then).
 * AM_OPT_SELECT: the best-trajectory rule of am_get_best and of grouped
 * and served solves when no trajectory is collision-free.  AM_SELECT_COST
 * (default): the lowest cost (Fig. 1's rule applied to every trajectory);
 * AM_SELECT_CLEARANCE: the largest smallest ellipse distance, for a
 * receding-horizon loop, where the cheapest colliding plan is the worst one
 * to execute.  Collision-free trajectories always rank first, by cost.
 * Groups and servers read it when they are created or started.
 * AM_OPT_DIAG_STALL: diagnostic for failure-detection tests (no counterpart
 * in the paper).  While set, the fused kernel stages its constants without
 * issuing the copy, so its bounded device-side wait (about one second) runs
 * out; the kernel then records the failure in the handle's status word and
 * returns, the getters report AM_ERR_TIMEOUT, and the results are undefined.
 * The next solve after clearing it resets the status word. */
#define AM_OPT_KERNEL 1
#define AM_OPT_TILE 2
#define AM_OPT_DIAG_STALL 3
#define AM_OPT_SELECT 4
#define AM_SELECT_COST 0
#define AM_SELECT_CLEARANCE 1
AM_API int am_set_option(am_problem *h, int option, int value);

/* Stream used by calls that take none (am_set_obstacles, am_set_boundary,
 * getters); am_solve_batch also sets it to the stream it is given. */
AM_API int am_set_stream(am_problem *h, void *stream);

/* Number of kernels the last am_solve_batch launched. */
AM_API int am_last_solve_stats(am_problem *h, int *launches);

/* Allocation-free solve (no counterpart in the paper; an operational entry
 * point).  Runs the plain loop (AM_KERNEL_PLAIN's kernels) on caller-owned
 * device buffers and keeps every intermediate in a fixed 32 MiB area that is
 * part of the library's device image, so the call itself never allocates:
 * for callers that cannot call cudaMalloc at solve time -- a real-time
 * re-planning step whose budget cudaMalloc's unbounded, device-synchronising
 * latency would break, or code running under an allocator or a stream
 * capture that forbids raw allocations.
 *  h        a handle set up beforehand (am_init_problem, am_set_obstacles)
 *           on the device that is current now (else AM_ERR_ARG); only its
 *           device constants are read, its buffers are untouched.  The call
 *           orders itself after the handle's own stream, where the constants
 *           were uploaded (an event of the handle, recorded there and waited
 *           on; nothing is allocated).  While `stream` is being captured the
 *           caller must have ordered it after the handle's stream itself.
 *  state    device, B x AM_STATE_FLOATS, in/out (the cold-start state has
 *           xi1 = (c_x, cos c_psi, c_y, sin c_psi), lambda = 0).
 *  res, res_psi, cost, mind   device, B floats each (as am_get_results).
 * Returns AM_ERR_BUDGET, with the sizes in am_last_error(), when the batch
 * needs more than the fixed area holds (about 650 trajectories at q = 100,
 * m = 3, n = 10).  The first call on a device looks up the area's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  Later calls check the cached address
 * against the current context and look it up again after a device reset.  All calls in the process share the one
 * area: calls that overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  Nothing in the area needs to
 * start at zero: every word a call reads it has written earlier in the same
 * call. */
AM_API int am_solve_batch_noalloc(const am_problem *h, int B, float *state, float *res,
                                  float *res_psi, float *cost, float *mind, int iters,
                                  void *stream);

/* Loads a cold-start (or warm) state for B trajectories without solving, as
 * am_solve_batch does before its first iteration (init: B x 3 x 11
 * coefficients c_x, c_y, c_psi; warm_lambda: optional B x 55 lambda, lambda_psi).
 * Used to prepare the problems of a group. */
AM_API int am_init_state(am_problem *h, int B, const float *init, const float *warm_lambda,
                         void *stream, int mem);

/* Groups: many problems of different shapes (q, m, n, B) advanced by one
 * persistent launch (the uneven batching of many independent planning
 * problems, Sec. III-D applied per trajectory).  Each CTA takes (problem,
 * tile) work items from a counter, costliest tiles first, and stages a
 * problem's constants only when its next item belongs to another problem.
 * A group references its problems, which must outlive it; each problem keeps
 * its own state, results (am_get_results, am_get_best) and constants.  Every
 * problem needs a state (am_init_state or an earlier solve) before
 * am_group_solve.  On a non-default stream a solve is captured once into a
 * CUDA graph and replayed while the group, the iteration count, the block size
 * and the stream stay the same; changing a problem's batch size or obstacle
 * count needs a fresh group. */
typedef struct am_group am_group;
AM_API int am_group_create(am_problem *const *problems, int count, am_group **out);
/* Runs iters iterations of every problem of the group; asynchronous. */
AM_API int am_group_solve(am_group *g, int iters, void *stream);
/* Times the group's solve over the block sizes that fit every problem and
 * keeps the fastest; with problems on the warp-pair kernels, then over caps
 * on their trajectory slots per CTA (none, 7 .. 3) and keeps the fastest.
 * The problems' states are restored afterwards.  Writes the chosen block
 * size and the time per solve (ms) of the chosen settings. */
AM_API int am_group_autotune(am_group *g, int iters, void *stream, int *threads, float *ms);
/* AM_GOPT_THREADS: block size of the small-tile group kernels (0 = largest,
 * else a multiple of 32).
 * AM_GOPT_GRAPH: 1 = capture and replay on non-default streams (default).
 * AM_GOPT_WARP_SLOTS: at most this many trajectory slots per CTA in the
 * warp-pair group kernels (0 = as many as fit shared memory, the default;
 * else 1..AM_GROUP_MAX_WARP_SLOTS).
 * am_group_autotune sets AM_GOPT_THREADS and, when the group has problems
 * on the warp-pair kernels, AM_GOPT_WARP_SLOTS; am_group_get_option reads
 * any of them back. */
#define AM_GOPT_THREADS 1
#define AM_GOPT_GRAPH 2
#define AM_GOPT_WARP_SLOTS 3
#define AM_GROUP_MAX_WARP_SLOTS 8
AM_API int am_group_set_option(am_group *g, int option, int value);
AM_API int am_group_get_option(am_group *g, int option, int *value);
/* Restricts the following solves (and am_group_get_best) to the listed
 * problems, given by their position in am_group_create's array, each at most
 * once, in any order; count = 0 selects every problem again.  A captured
 * launch stays valid across changes of the list (the work list and its
 * length are uploaded before each replay). */
AM_API int am_group_set_active(am_group *g, const int *idx, int count);
/* Best trajectory of every active problem (Fig. 1's selection, per problem):
 * writes 36 floats per active problem, in the order of the active list:
 * {index, cost, residual, 33 coefficients c_x, c_y, c_psi}.  With host
 * memory the call waits (bounded) for the stream. */
AM_API int am_group_get_best(am_group *g, float *out, int mem, void *stream);
/* Launches issued by this group so far and work items of its last solve. */
AM_API int am_group_stats(am_group *g, int *launches, int *items);
AM_API void am_group_destroy(am_group *g);

/* ------------------------------------------------------------- serving
 * Re-planning service for the receding-horizon use of the method (Sec. IV:
 * each new plan starts from the previous one, warm-started, with few
 * iterations).  A scene is a problem whose state (xi, lambda) stays resident
 * on the device between requests.  A worker thread serves requests in
 * rounds: a round takes at most one pending request per scene (oldest
 * first) among the scenes not already in flight, applies each request's
 * updates (start state, obstacle tracks), advances the scenes by `iters`
 * iterations -- all of them in one grouped launch (AM_SRV_BATCHED; a round
 * of one request uses the scene's own kernel, and a round groups scenes
 * only when at least three requests are admissible, else it takes one and
 * the next goes to the next free lane), or one request per round
 * with the scene's own kernel (AM_SRV_SEQUENTIAL, the comparator) --
 * selects each scene's best trajectory and completes the requests.  Up to
 * `lanes` rounds are in flight at once, each on its own stream: the worker
 * issues a round without waiting for it, polls the rounds in flight, and
 * admits requests that arrive meanwhile into the next free lane, so their
 * work starts while earlier rounds are still on the GPU (continuous
 * batching).  A request's result does not depend on the round or lane it
 * was served in.
 *
 * Scenes are admitted while the device bytes they hold (am_scene_bytes)
 * stay within the budget; am_server_add_scene returns AM_ERR_BUDGET beyond
 * it, and am_server_submit returns AM_ERR_BUDGET when max_pending requests
 * are queued.  The server uses the scenes' handles from its own thread
 * between am_server_start and am_server_destroy: the caller must not use
 * them meanwhile, and destroys them after the server. */
#define AM_PENDING 1        /* am_server_poll: the request is not finished yet */
#define AM_SRV_BATCHED 0
#define AM_SRV_SEQUENTIAL 1

typedef struct {
    size_t budget_bytes;    /* device bytes all scenes together may hold      */
    int iters;              /* AM iterations per request                       */
    int mode;               /* AM_SRV_BATCHED | AM_SRV_SEQUENTIAL              */
    int max_batch;          /* requests per round (0 = up to one per scene);
                               a round takes several only when at least
                               three are admissible                          */
    int max_pending;        /* queue bound (0 = 65536)                         */
    int lanes;              /* rounds in flight (0 = 2 batched, 1 sequential;
                               at most 8); AM_SRV_SEQUENTIAL takes 1          */
} am_server_desc;

#define AM_REQ_GOAL 1       /* am_request.flags: replace the goal state        */
#define AM_REQ_RESAMPLE 2   /* am_request.flags: re-draw the batch (am_resample) */
#define AM_REQ_SHIFT 4      /* am_request.flags: re-time the batch by the advance (am_shift) */
#define AM_REQ_SCALE_LAMBDA 8  /* am_request.flags: scale the multipliers (am_scale_multipliers) */

typedef struct {
    int scene;              /* as returned by am_server_add_scene              */
    double advance;         /* > 0: the start state becomes the scene's last
                               best plan at t = advance s (position, velocity,
                               acceleration of x, y and psi)                   */
    const float *xo, *yo;   /* nullable: new obstacle centre tracks, n x q
                               each, host memory, copied by am_server_submit   */
    int flags;              /* AM_REQ_GOAL | AM_REQ_RESAMPLE | AM_REQ_SHIFT |
                               AM_REQ_SCALE_LAMBDA, applied after the advance
                               and the tracks, before the solve (a re-draw
                               supersedes a shift; the scaling comes last)    */
    double goal[9];         /* AM_REQ_GOAL: x, x', x'', y, y', y'', psi, psi',
                               psi'' at t = T                                   */
    unsigned long long seed;  /* AM_REQ_RESAMPLE: generator seed               */
    float sigma;            /* AM_REQ_RESAMPLE: perturbation scale (m)         */
    float lambda_scale;     /* AM_REQ_SCALE_LAMBDA: factor (finite, >= 0)      */
} am_request;

typedef struct {
    int status;             /* AM_OK or the error code of the request's round  */
    int index;              /* best trajectory of the scene                    */
    float cost, residual;
    float coeffs[33];       /* c_x, c_y, c_psi of the best trajectory          */
    double t_submit, t_start, t_done;  /* seconds, the server's steady clock  */
    long long round;        /* round that served the request                   */
    int batch;              /* requests in that round                          */
} am_result;

typedef struct am_server am_server;
AM_API int am_server_create(const am_server_desc *desc, am_server **out);
/* Admits a scene: loads its cold-start state (init: B x 3 x 11, as
 * am_solve_batch) and returns its number.  Before am_server_start only. */
AM_API int am_server_add_scene(am_server *s, am_problem *h, int B, const float *init, int mem,
                               int *scene);
/* Starts the worker thread (on the device current in the calling thread). */
AM_API int am_server_start(am_server *s);
/* Queues a request (thread-safe); returns its ticket.  Requests queued
 * before am_server_start are served from the first round on. */
AM_API int am_server_submit(am_server *s, const am_request *req, long long *ticket);
/* Waits up to timeout_ms for a request; AM_OK with its result (the ticket is
 * then forgotten), AM_PENDING if it is not finished, AM_ERR_ARG if unknown. */
AM_API int am_server_poll(am_server *s, long long ticket, am_result *out, int timeout_ms);
AM_API int am_server_stats(am_server *s, long long *rounds, long long *completed,
                           size_t *device_bytes);
/* Stops the worker after its current round; queued requests complete with
 * AM_ERR_STATE.  Does not destroy the scenes' handles. */
AM_API void am_server_destroy(am_server *s);
/* Device bytes a scene of this shape and batch holds (host arithmetic only). */
AM_API size_t am_scene_bytes(int q, int m, int n, int B);

AM_API void am_destroy(am_problem *h);
AM_API const char *am_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
