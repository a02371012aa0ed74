/*
 * hj.h -- C ABI of the GB300 (sm_103a) Hamilton-Jacobi safe-set library.
 *
 * The library computes the safe sets of Herbert, Choi et al., "Scalable
 * Learning of Safety Guarantees for Autonomous Systems using Hamilton-Jacobi
 * Reachability" (arXiv 2101.05916):
 *   - the value function of Sec. II-A, Eq. 1,
 *   - obtained by iterating the HJI variational inequality of Eq. 2 backward
 *     in time until convergence,
 *   - on one grid per decomposed subsystem (Sec. III-A),
 *   - warm-started from a previous value function (Sec. III-B),
 *   - or from a coarse-grid solution migrated to a finer grid (Sec. III-C).
 *
 * Sign convention.  Everything here uses W := -V and l := -c, where V and c
 * are the paper's value and constraint functions.  So:
 *   - l is positive inside the constraint set;
 *   - the safe set is {W >= 0};
 *   - the control maximises and the disturbance minimises;
 *   - the clamp of Eq. 2 reads W <- min(W, l).
 * Negate the results to get the paper's V.
 *
 * Discretisation (the paper names none; this is the textbook scheme):
 *   - Grid: uniform, n[i] nodes from lo[i] to hi[i] inclusive.  Row-major
 *     with the LAST axis fastest.  Values are FP32.  Ghost nodes continue
 *     each grid line linearly through its two outermost nodes.
 *   - Slopes: first-order upwind, ENO2 or WENO5 one-sided differences.
 *   - Hamiltonian: global Lax-Friedrichs numerical Hamiltonian, with bang-bang
 *     control and worst-case disturbance.
 *   - Time step: dt = cfl / sum_i(a_i / h_i), where a_i is the largest |f_i|
 *     over the grid and the input boxes.
 *   - Integration: TVD-RK3, then the clamp after each full step.
 *   - Stop: when max|W(t + check_dt) - W(t)| < tol, over every node or over
 *     the band |W| <= opts.band around the zero level set, optionally
 *     skipping opts.band_margin cells next to the faces of the grid box.
 *
 * Threading and memory:
 *   - Handles are not thread-safe.  Use one handle per thread, or serialise
 *     the calls.
 *   - Device memory belongs to the library.
 *   - Host arrays belong to the caller.  They are read or written only during
 *     the call.
 *   - Every call returns an hj_status.  On failure, hj_last_error() gives a
 *     thread-local message.
 *   - Nothing falls back to the CPU: with no usable CUDA device, every
 *     computing call returns HJ_ERR_CUDA.
 */
#ifndef HJ_H
#define HJ_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct hj_grid_s* hj_grid;

typedef enum {
  HJ_OK = 0,
  HJ_ERR_ARG = 1,           /* invalid argument (null pointer, bad size, out-of-grid query) */
  HJ_ERR_OOM = 2,           /* device allocation failed                                    */
  HJ_ERR_CUDA = 3,          /* a CUDA call failed, or no device                             */
  HJ_ERR_NOT_CONVERGED = 4, /* step cap or wall-time cap hit.  W is still the valid         */
                            /* finite-horizon value after the steps taken                   */
  HJ_ERR_STATE = 5,         /* e.g. warm solve with no prior, or dynamics/constraint unset  */
  HJ_ERR_ABORTED = 6,       /* cancelled between check windows                              */
  HJ_ERR_DIVERGED = 7       /* a non-finite value appeared in W                             */
} hj_status;

/* Dynamics f(x, u, d) (Sec. II-A).  The parameter vector is per model.
 *   HJ_DRIFT   any ndim 1..4.  f = d.  One disturbance input per axis.  No params.
 *   HJ_QUAD_Z  ndim 2, state (z, vz).  f = (vz, kT u - g + d).
 *              params = {kT, g, u_lo, u_hi}.  One disturbance input.
 *              This is the 2-D vertical quadcopter (Sec. V-A) and the z block
 *              of Eq. 3.
 *   HJ_QUAD_X4 ndim 4, state (p, v, th, w).
 *              f = (v, g tan th, -d1 th + w, -d0 th + n0 u), with the single
 *              disturbance d added to component `axis` (0 or 1).
 *              params = {g, d1, d0, n0, u_lo, u_hi, axis}.
 *              This is the x (or y) block of Eq. 3. */
enum { HJ_DRIFT = 0, HJ_QUAD_Z = 1, HJ_QUAD_X4 = 2 };

/* spatial schemes */
enum { HJ_FIRST = 1, HJ_ENO2 = 2, HJ_WENO5 = 5 };
/* clamp after each step: VI = min(W, l) (Eq. 2); MONOTONE = min(W, l, W_prev) */
enum { HJ_CLAMP_VI = 0, HJ_CLAMP_MONOTONE = 1 };
/* initial value: COLD = l (Eq. 2 terminal value); WARM = min(prior, l) (Sec. III-B) */
enum { HJ_COLD = 0, HJ_WARM = 1 };

#define HJ_MAX_DIM 4

typedef struct {
  int scheme;            /* HJ_FIRST, HJ_ENO2 or HJ_WENO5 (default WENO5)                 */
  double cfl;            /* Courant number (default 0.5)                                  */
  double dt;             /* > 0: fixed step instead of the CFL rule (default 0)           */
  double tol;            /* stop when the L-inf change over a window is below (1e-4)      */
  double check_dt;       /* window length in simulated seconds (default 0.1)              */
  long long max_steps;   /* step cap, 0 = none (default 1000000)                          */
  long long fixed_steps; /* > 0: run exactly this many steps and skip the stop test       */
  double max_wall_ms;    /* wall-time cap checked between windows, 0 = none               */
  int clamp;             /* HJ_CLAMP_VI (default) or HJ_CLAMP_MONOTONE                    */
  int use_graph;         /* 1: replay each window as a captured CUDA graph (default 1)    */
  double band;           /* > 0: the stop test watches only nodes with                    */
                         /* min(|W|, |W_window_start|) <= band, i.e. the band around the  */
                         /* zero level set that bounds the safe set (Sec. II-A).          */
                         /* 0 (default): every node.                                      */
  int autotune;          /* 1: pick the stage kernels' launch shape by timing (hj_autotune) */
                         /* once per grid shape before solving (default 0)                */
  int band_margin;       /* the stop test skips nodes closer than this many cells to a    */
                         /* face of an unconstrained axis (every axis for a ball), where  */
                         /* trajectories leave a truncated grid (default 0)               */
  double local_tol;      /* > 0: localized stepping (Sec. VI): after the first window,    */
                         /* only slabs whose value changed by more than local_tol in the  */
                         /* last window (nodes within band_margin of a free face do not   */
                         /* count; nodes outside the band do), and slabs close enough to  */
                         /* them for a change to arrive within the next window (the CFL   */
                         /* distance of a window along each slab axis, plus               */
                         /* local_margin slabs), step;                                    */
                         /* the others keep their value.  Slabs are the lines of the two  */
                         /* slowest axes of a 4-D grid, the first axis of a 2-D or 3-D    */
                         /* grid.  Stage values next to stepping slabs are recomputed on  */
                         /* rings of 1 and 2 stencil radii, so that every stepping node's */
                         /* update is the full solve's update of the current field.       */
                         /* Ignored with fixed_steps.  0 (default): off.                  */
  int local_margin;      /* extra reactivation margin in slabs (default 1)                */
} hj_solve_opts;

typedef struct {
  long long steps;   /* TVD-RK3 steps taken                                   */
  double t;          /* simulated backward time reached                       */
  double residual;   /* L-inf change over the last window                     */
  double dt;         /* step used                                             */
  double wall_ms;    /* host wall time of the call                            */
  int converged;     /* 1 if residual < tol                                   */
  long long windows; /* stop tests performed                                  */
  double stepped;    /* stage-kernel tiles run / tiles of full stepping (1 unless */
                     /* localized)                                               */
} hj_solve_stats;

/* Fill *o with the defaults listed above. */
void hj_default_opts(hj_solve_opts* o);

/* Create a grid of ndim (1..4) axes.  Axis i has n[i] >= 3 nodes spanning
 * [lo[i], hi[i]], with lo < hi.  The total node count must be below 2^31.
 * cuda_stream is a cudaStream_t, or NULL for the legacy default stream.  All
 * device work of this handle is ordered on that stream.  This call allocates
 * four FP32 fields (W, two RK stages, the window snapshot) of n[0]*..*n[ndim-1]
 * values each on the current device.
 * Errors: HJ_ERR_ARG on bad sizes, HJ_ERR_OOM, HJ_ERR_CUDA. */
hj_status hj_grid_create(hj_grid* out, int ndim, const int* n, const double* lo,
                         const double* hi, void* cuda_stream);
void hj_grid_destroy(hj_grid g);
hj_status hj_set_stream(hj_grid g, void* cuda_stream);

/* Dynamics of Sec. II-A (and Eq. 3 for the quadcopter blocks).  params has
 * nparams entries, laid out per model as in the model list above.
 * HJ_ERR_ARG on an unknown model, a wrong ndim or too few parameters. */
hj_status hj_set_dynamics(hj_grid g, int model, const double* params, int nparams);

/* Constraint set C of Sec. II-A, as the margin l = -c, where c is the signed
 * distance to C.  The safe region is the box lo[i] <= x_i <= hi[i].  An axis
 * with both bounds infinite is unconstrained.  Distances are in raw state
 * units:
 *   - inside the box, l is the distance to the nearest face;
 *   - outside it, l is minus the Euclidean distance to the box.
 * At least one axis must be constrained. */
hj_status hj_set_constraint(hj_grid g, const double* box_lo, const double* box_hi);
/* Alternative constraint: the safe region lies outside a ball.
 * l = |x - centre| - radius, with radius > 0. */
hj_status hj_set_constraint_ball(hj_grid g, const double* centre, double radius);
/* Constraint given as an array (Sec. II-A: c is the signed distance to the
 * constraint set C, for any C): l = -c at every node, positive where safe.
 *   - l holds npts floats, row-major as in hj_get_value; on_device = 1: a
 *     device pointer, 0: host memory.  The data is copied.
 *   - It replaces a box or ball; a later hj_set_constraint or
 *     hj_set_constraint_ball replaces it.
 *   - The clamp and the initial value read l at the node; migration
 *     (hj_prolong) reads the fine grid's l.
 *   - The band_margin option treats every axis as unconstrained.
 *   - Costs one extra 4-byte read per node in the last RK stage.
 * HJ_ERR_ARG on NULL or a non-finite value; after that rejection no
 * constraint is in force (solves fail with HJ_ERR_STATE until one is set). */
hj_status hj_set_constraint_field(hj_grid g, const float* l, int on_device);

/* Disturbance box D (Sec. II-C): d_j in [d_lo[j], d_hi[j]] for each of the
 * nd inputs.  Asymmetric intervals are allowed; they come from a GP
 * confidence interval.  nd must match the model: 1 for the quadcopter
 * blocks, ndim for HJ_DRIFT. */
hj_status hj_set_disturbance_bound(hj_grid g, const double* d_lo, const double* d_hi, int nd);

/* State-dependent disturbance box (Sec. II-C).  The GP gives a
 * delta-confidence interval D(x) at every state; this sets it node by node.
 *   - d_lo and d_hi hold nd * npts floats each, input-major: input j's
 *     field is [j * npts, (j + 1) * npts), with the nodes row-major as in
 *     hj_get_value.
 *   - on_device = 1: the pointers are device memory; 0: host memory.
 *     Either way the data is copied.
 *   - The field replaces the uniform box.  A later hj_set_disturbance_bound
 *     replaces the field.
 *   - Costs two extra reads per node and RK stage per disturbance input.
 *   - Warm starts stay exact while every interval of the prior lies inside
 *     the new one at every node.
 * HJ_ERR_ARG on NULL pointers, a bad nd, or a node where d_lo > d_hi or a
 * value is not finite.  After that last rejection no disturbance bound is in
 * force: solves fail with HJ_ERR_STATE until one is set again. */
hj_status hj_set_disturbance_field(hj_grid g, const float* d_lo, const float* d_hi, int nd,
                                   int on_device);

/* Translated prior.  The quadcopter blocks' f does not depend on the
 * position (axis 0), and a drift's on no axis, so when the constraint moves
 * by `shift` along such axes the fixed point moves with it.  This writes
 *   dst.W(x) = min(src.W(x - shift), l_dst(x))
 * by multilinear interpolation of src's value; where x - shift leaves src's
 * box, dst.W(x) = l_dst(x) (the cold start there).  The result is the prior
 * of a following HJ_WARM solve of dst.
 *   - src and dst are distinct grids with the same model and parameters; any
 *     resolution and box.
 *   - shift has ndim entries; it must be 0 on axes the dynamics depend on.
 *   - Exact (up to the grid's truncation near its faces) when the shifted
 *     constraint of src contains dst's and src's disturbance box lies in
 *     dst's (Sec. III-B's dominance, modulo the translation).
 * HJ_ERR_ARG on NULL, equal grids, other dynamics or a shift along a
 * non-invariant axis; HJ_ERR_STATE without a source value or target
 * constraint, or with a state-dependent disturbance bound on either. */
hj_status hj_translate(hj_grid src, hj_grid dst, const double* shift);

/* Iterate Eq. 2 to convergence.
 * Starting value:
 *   - HJ_COLD starts from l.
 *   - HJ_WARM starts from min(prior, l) (Sec. III-B).  The prior is the
 *     grid's current W: the last result, the last hj_set_value, or the last
 *     hj_prolong or hj_translate into this grid.
 * o may be NULL, which means the defaults.  s may be NULL.
 * On HJ_OK or HJ_ERR_NOT_CONVERGED the grid's W holds the result.
 * Returns:
 *   HJ_ERR_STATE    when dynamics, constraint or disturbance are unset, or
 *                   HJ_WARM is asked with no prior;
 *   HJ_ERR_DIVERGED when a non-finite value appears. */
hj_status hj_solve(hj_grid g, int mode, const hj_solve_opts* o, hj_solve_stats* s);

/* Solve several grids together (Sec. III-A: decomposed subsystems are
 * independent).  In each time step of all still-unconverged grids, the
 * grids of one kind (model, ndim, scheme) below 2^20 nodes share one fused
 * launch per RK stage, and larger grids get their own; each grid keeps its
 * own dt and stop test.  All grids
 * must be on the same device.  The work runs on the stream of gs[0].  modes,
 * opts and stats are arrays of ngrids entries.  opts may be NULL, or point to
 * a single entry when opts_count is 1.  Returns the first non-OK status, in
 * grid order; each grid's own status goes to status_out when that is
 * non-NULL. */
hj_status hj_solve_batch(hj_grid* gs, int ngrids, const int* modes, const hj_solve_opts* opts,
                         int opts_count, hj_solve_stats* stats, int* status_out);

/* Coarse-to-fine migration (Sec. III-C): fine.W = min(interp(coarse.W), l_fine),
 * where interp is multilinear interpolation of the coarse W at the fine nodes.
 * Both grids need the same ndim, and the fine box must lie inside the coarse
 * box.  The fine grid needs its constraint set first.  Afterwards an HJ_WARM
 * solve of the fine grid starts from the migrated value. */
hj_status hj_prolong(hj_grid coarse, hj_grid fine);

/* Copy a dense row-major FP32 field of npts values into W (a prior, or a
 * resume point), or W out of the library.  on_device = 1 means the pointer
 * is device memory on the grid's device; on_device = 0 means host memory.
 * Both calls return after the copy has completed. */
hj_status hj_set_value(hj_grid g, const float* src, int on_device);
hj_status hj_get_value(hj_grid g, float* dst, int on_device);

/* W (hj_query_value) or grad W (hj_query_gradient) at npts arbitrary states.
 * x is host memory with npts * ndim doubles, row-major (point-major).
 *   - Values are the multilinear interpolation of W.
 *   - Gradients are the multilinear interpolation of the node gradients.
 *     Node gradients are central differences, one-sided at the ends of an
 *     axis.  grad_out holds npts * ndim doubles.
 * The gradient gives the safety control u* = argmax_u grad W . f
 * (Sec. II-A, in the W convention).
 * HJ_ERR_ARG if a point lies outside the grid box. */
hj_status hj_query_value(hj_grid g, int npts, const double* x, double* v_out);
hj_status hj_query_gradient(hj_grid g, int npts, const double* x, double* grad_out);

/* Largest |f_i| over the grid and the input boxes, per axis.  These are the
 * Lax-Friedrichs coefficients, and the CFL dt follows from them.  Computed on
 * the device by a max-reduction.  alpha_out has ndim entries. */
hj_status hj_alpha(hj_grid g, double* alpha_out);

/* ------------------------------------------------------------------ server
 * Safety-update serving (Sec. II-C, Sec. III).  New disturbance bounds
 * arrive over time and each one triggers an update solve of one subsystem.
 * The server runs these solves with continuous batching:
 *   - Admission: a background worker admits queued requests in arrival
 *     order, whenever active slots and the HBM budget allow.  A request that
 *     does not fit is skipped for smaller later ones.
 *   - Stepping: all admitted requests advance together, one fused launch per
 *     RK stage (as hj_solve_batch), each with its own dt and stop test.
 *     A request that arrives while others run joins at the next round
 *     boundary.
 *   - Residency: each subsystem key keeps its latest converged value on the
 *     device.  A later HJ_WARM request with the same key warm-starts from it
 *     (Sec. III-B) only when the prior provably dominates the new fixed
 *     point.  That needs the same grid and model, every disturbance
 *     interval of the prior inside the new one, and the prior's constraint
 *     box containing the new one, and the VI clamp: under HJ_CLAMP_MONOTONE
 *     the solve's limit depends on its start, so such a request always
 *     solves cold.  Otherwise the request solves cold.  Priors whose box
 *     contains the new one only once moved are used only after
 *     hj_server_set_translated_starts(s, 1).
 *   - Memory: results stay on the device until hj_server_release.  Released
 *     results that are still a key's resident prior are evicted (least
 *     recently used first) when the budget is needed.
 * Handles are thread-safe: any host thread may submit, poll or wait. */
typedef struct hj_server_s* hj_server;

typedef struct {
  int ndim;
  int n[HJ_MAX_DIM];
  double lo[HJ_MAX_DIM], hi[HJ_MAX_DIM];
  int model;
  double params[8];
  int nparams;
  double d_lo[HJ_MAX_DIM], d_hi[HJ_MAX_DIM];
  int nd;
  int con_ball;                 /* 0: box con_a = lo, con_b = hi; 1: ball, centre con_a, radius con_b[0] */
  double con_a[HJ_MAX_DIM], con_b[HJ_MAX_DIM];
  int mode;                     /* HJ_COLD, or HJ_WARM = use the key's resident prior when exact */
  long long key;                /* subsystem identity for residency; 0 = none                  */
  hj_solve_opts opts;
  int coarse_n;                 /* >= 3: coarse initialisation (Sec. III-C).  The request first */
                                /* solves on a grid of coarse_n nodes per axis over the same    */
                                /* box, then migrates that value to its own grid (hj_prolong)   */
                                /* and finishes with a warm solve there.  Exact or conservative */
                                /* (Sec. III-B), usually far fewer fine steps.  0: off.         */
  int coarse_n2;                /* > coarse_n: an intermediate level (coarse -> coarse_n2 ->   */
                                /* n, each migrated and warm-solved; more levels "refined over */
                                /* time", Sec. III-C).  0: none.  Needs coarse_n.              */
  int coarse_scheme;            /* scheme of the coarse levels (cheap gradients on the coarse  */
                                /* grid, e.g. HJ_ENO2: faster, more conservative); 0: opts'    */
} hj_request;

typedef struct {
  long long submitted, admitted, completed, failed, rejected;
  long long warm_starts, cold_starts, evictions, rounds;
  long long bytes_in_use, peak_bytes;
  long long active;             /* requests stepping right now                                 */
  long long queued;
  double p50_ms, p99_ms;        /* submit-to-completion latency of completed requests          */
  double updates;               /* grid-point updates (nodes x steps) of all finished requests */
  double busy_ms;               /* wall time from first submit to last completion              */
  long long translated_starts;  /* warm starts from a translated prior (hj_translate): the key's */
                                /* prior dominates once its constraint is moved along the       */
                                /* position axis                                               */
} hj_server_stats;

/* Start a server on the current device.  hbm_budget_bytes bounds the device
 * memory of all its grids (four FP32 fields per node).  max_active bounds
 * the concurrent solves (<= 1024).  cuda_stream is the stream all work runs
 * on (NULL = a private stream). */
hj_status hj_server_create(hj_server* out, long long hbm_budget_bytes, int max_active,
                           void* cuda_stream);
/* Stop admitting, finish running requests, free everything. */
void hj_server_destroy(hj_server s);
/* Queue a request; *ticket identifies it.  The request is copied.
 * HJ_ERR_ARG: bad request.  HJ_ERR_OOM: it can never fit the budget. */
hj_status hj_server_submit(hj_server s, const hj_request* r, long long* ticket);
/* *done = 1 once the request finished; then *result is its hj_solve status and
 * *st its statistics (wall_ms = submit-to-completion latency). */
hj_status hj_server_poll(hj_server s, long long ticket, int* done, hj_status* result,
                         hj_solve_stats* st);
/* Block until the request finished or timeout_ms passed (<= 0: no limit).
 * HJ_ERR_NOT_CONVERGED is returned on timeout, HJ_OK when finished. */
hj_status hj_server_wait(hj_server s, long long ticket, double timeout_ms, hj_status* result,
                         hj_solve_stats* st);
/* Copy a finished request's value function (dense row-major FP32) out. */
hj_status hj_server_get_value(hj_server s, long long ticket, float* dst, int on_device);
/* Drop the caller's interest in a ticket; its memory may then be reused. */
hj_status hj_server_release(hj_server s, long long ticket);
/* Cancel a queued or running request (it finishes with HJ_ERR_ABORTED). */
hj_status hj_server_cancel(hj_server s, long long ticket);
hj_status hj_server_get_stats(hj_server s, hj_server_stats* out);

/* Admission policy.
 *   order: HJ_ORDER_FIFO admits in arrival order (the default).
 *     HJ_ORDER_SHORTEST admits the request with the least estimated work
 *     first.  The estimate is nodes x the largest axis length, since the
 *     steps to converge grow like 1 / dt ~ 1 / h.
 *   max_active_nodes: if > 0, a request is admitted only while the nodes of
 *     all stepping requests stay within it.  Exceptions: a request is always
 *     admitted when nothing is stepping, and requests below 1/64 of the cap
 *     are always admitted.  Large grids fill the GPU on their own; the cap
 *     stops them from time-slicing each other, while small grids still run
 *     beside them.
 * Applies from the next admission on. */
enum { HJ_ORDER_FIFO = 0, HJ_ORDER_SHORTEST = 1 };
hj_status hj_server_set_policy(hj_server s, int order, long long max_active_nodes);

/* Warm starts from translated priors (Sec. III-B reuse of a prior whose
 * constraint box moved along the position axis; see hj_translate).
 *   enable = 1: a HJ_WARM request whose key's prior dominates only once its
 *     box is moved warm-starts from the moved prior (counted in
 *     translated_starts).
 *   enable = 0 (the default): such a request solves cold.
 * The schemes here are not monotone, so a solve's limit can depend on its
 * start: on the 2-D ENO2 requests of the seeded serving trace a translated
 * start landed 1e-5 to 1e-4 (relative) above the cold fixed point at every
 * stop tolerance tried, and saved no steps in four of five cases.
 * HJ_ERR_ARG: enable not 0 or 1.  Applies from the next admission on. */
hj_status hj_server_set_translated_starts(hj_server s, int enable);

/* Safety filter of the safe-learning loop (Sec. II-B, II-C) for a system
 * decomposed into independent subsystem grids (Sec. III-A, e.g. the 10-D
 * quadcopter as x, y and z).  For each of nq full states:
 *   - Grid k sees the subsystem state x_k[d] = states[q * state_dim +
 *     axes[k * HJ_MAX_DIM + d]] for d < its ndim; W_k(x_k) and grad W_k are
 *     multilinear interpolations of the node values and of the node
 *     gradients (central differences, one-sided at the ends), in double.
 *   - The decomposed value is w_out[q] = min_k W_k (valid for separable
 *     constraint boxes).
 *   - Where W_k <= level, the control ctrl_index[k] is replaced by the
 *     optimal safety control u* = argmax_u min_d <grad W_k, f_k> (Sec. II-A;
 *     W = -V): the input's upper bound where grad W_k . df/du > 0, the lower
 *     where it is < 0; on a tie the performance control stays, clipped to
 *     the input box.  level = 0 switches on the boundary; level > 0 keeps a
 *     margin, e.g. the contracted sublevel set of the previous value
 *     function while an update runs (Sec. II-C).
 *   - active_out[q] has bit k set where grid k's safety control was applied.
 *   - Other controls copy u_perf.  ctrl_index[k] = -1: the grid drives no
 *     control (HJ_DRIFT has none).  No control may be driven by two grids.
 * Layout: states nq x state_dim, u_perf and u_out nq x ctrl_dim (doubles,
 * row-major); w_out nq doubles; active_out nq ints.  on_device = 1: all
 * buffers are device memory; 0: host memory, staged through a device block
 * and a pinned host block that grids[0] keeps for later calls (one copy in,
 * one copy out).  Runs on grids[0]'s stream; every grid must hold a value
 * and live on the same device; calls sharing grids[0] must not overlap.
 * HJ_ERR_ARG on bad indices or dimensions, or a state outside a grid's box
 * (the outputs are then undefined); HJ_ERR_STATE for a grid without value. */
hj_status hj_safety_filter(const hj_grid* grids, int ngrids, const int* axes,
                           const int* ctrl_index, int state_dim, int ctrl_dim, long long nq,
                           const double* states, const double* u_perf, double level,
                           double* u_out, double* w_out, int* active_out, int on_device);

/* Allocation-free fixed-horizon solve.  The paper has no counterpart: this
 * entry point exists for callers that must not allocate device memory after
 * start-up.  One example is a real-time safety filter running beside a
 * controller, as in the paper's ROS set-up: cudaMalloc and cudaFree can
 * synchronise the whole device and take unbounded time.  Another example is
 * a process whose device memory is owned entirely by another framework's
 * pool.
 *
 * What it does: the same computation as hj_grid_create + hj_set_dynamics +
 * hj_set_disturbance_bound + hj_set_constraint (box) + hj_solve with
 * opts.fixed_steps = steps, but with no handle:
 *   - W is caller-owned device memory with npts = n[0]*..*n[ndim-1] floats.
 *     With HJ_WARM it holds the prior on entry (HJ_COLD ignores it).  On
 *     return it holds the value after `steps` TVD-RK3 steps.
 *   - dt == 0 selects the CFL step with cfl = 0.5; dt < 0 (or NaN) is
 *     rejected with HJ_ERR_ARG.
 *   - W must be device (or managed) memory of the current device; a host
 *     pointer or memory of another device is rejected with HJ_ERR_ARG
 *     before any device work.
 *   - clamp is HJ_CLAMP_VI or HJ_CLAMP_MONOTONE.
 *   - The call returns after the work on cuda_stream has finished.
 *
 * Where the scratch lives: the working memory is one file-scope device
 * array, shared by every call in the process.  It holds the Lax-Friedrichs
 * coefficient accumulator, the g tan(th) table, a guarded working copy of W
 * and the two Runge-Kutta stage fields.  Every GPU that loads the library
 * holds the array (about 48 MiB) until the process exits.
 *
 * Limits: at most HJ_STATIC_MAX_POINTS nodes and at most HJ_STATIC_MAX_AXIS
 * nodes on the theta axis of HJ_QUAD_X4.  Larger problems fail with
 * HJ_ERR_ARG before any device work.
 *
 * The call never calls cudaMalloc, cudaFree or any allocating library
 * routine.
 *
 * First call on a device: it looks up the array's device address with that
 * device current.  Under lazy module loading (the CUDA default) that lookup
 * is also when the driver loads the module on the device and reserves the
 * 48 MiB array, so the first call can be slow or fail with HJ_ERR_CUDA when
 * the device is full.  Make one call (any small grid, steps = 0) on each
 * device at start-up, before any stream capture and before the device's
 * memory is handed to another pool.
 *
 * Concurrency: the array keeps the contents of the last call.  The call
 * clears what must start at zero itself.  Calls whose GPU work overlaps
 * (other streams, other host threads) race on the shared array and corrupt
 * each other's results; serialise them. */
#define HJ_STATIC_MAX_POINTS 4194304
#define HJ_STATIC_MAX_AXIS 4096
hj_status hj_solve_fixed_static(int ndim, const int* n, const double* lo, const double* hi,
                                int model, const double* params, int nparams,
                                const double* d_lo, const double* d_hi, int nd,
                                const double* box_lo, const double* box_hi, int mode,
                                int scheme, double dt, long long steps, int clamp, float* W,
                                void* cuda_stream);

/* Launch-shape autotuner.  It picks how the stage kernels map onto the
 * GPU for this grid and scheme, among:
 *   - the flat mapping: one thread per node over the flattened grid, in
 *     blocks of 128, 256 or 512 threads;
 *   - row tiles: each block stages tile_rows consecutive lines of the
 *     fastest axis in shared memory (16-byte loads, ghost values in place)
 *     and computes their nodes; the candidates are the line counts whose
 *     blocks (128 to 1024 threads) fill their warps best.  The halo width
 *     of a tile is the scheme's stencil radius (3 for WENO5, 2 for ENO2).
 * Every shape computes the same values bit for bit.  It times a few
 * TVD-RK3 steps of each candidate on the grid's current value, or on l if
 * the grid holds none (with the shape-specialised kernels where the grid
 * uses them), and keeps the fastest.  W is left unchanged.  The choice is
 * cached per (model, ndim, scheme, grid shape) for the whole process, and
 * later solves of this grid use it.  *threads_out (may be NULL) receives
 * the flat block size; hj_get_launch_shape gives the whole choice. */
hj_status hj_autotune(hj_grid g, int scheme, int* threads_out);

/* Sets the stage kernels' launch shape by hand: threads per block of the
 * flat mapping (128, 256 or 512) and tile_rows (0: the flat mapping; > 0:
 * row tiles of that many fastest-axis lines, at most 1024 nodes per tile).
 * HJ_ERR_ARG when the tile does not fit the grid.  Results do not depend on
 * the shape. */
hj_status hj_set_launch_shape(hj_grid g, int threads, int tile_rows);
/* The current launch shape (either pointer may be NULL). */
hj_status hj_get_launch_shape(hj_grid g, int* threads, int* tile_rows);

/* Shape-specialised stage kernels.  For grids of at least 2^19 nodes the
 * library compiles at run time (NVRTC, from the first use per grid shape,
 * scheme and block size) the stage kernels with the grid's axis lengths and
 * strides as constants, and keeps them for the process: the same arithmetic
 * per node with fewer index instructions.  Where NVRTC is not available or
 * a compilation fails, the precompiled kernels run.
 * The compile runs on a background thread: solves never wait for it, and
 * use the specialised kernels from the first launch after it finished.
 * hj_set_jit(0) turns this off (also HJ_JIT=0 in the environment), 1 on.
 * hj_jit_kernels() counts the kernel sets loaded so far; hj_jit_pending()
 * the compiles still running. */
void hj_set_jit(int enable);
long long hj_jit_kernels(void);
long long hj_jit_pending(void);
/* Diagnostic: builds the shape-specialised stage source for an ndim grid of
 * n[i] nodes per axis, the model and the scheme, and compiles it with NVRTC
 * for sm_103a.  Needs no device.  HJ_ERR_ARG on bad arguments; HJ_ERR_CUDA
 * when NVRTC is missing or the compile fails (hj_last_error holds the start
 * of NVRTC's log). */
hj_status hj_jit_check(int ndim, const int* n, int model, int scheme, int threads);
/* The same compile with ptxas reporting resources, for a box constraint on
 * the axes whose bits are set in con_axes (bit d: axis d; the others
 * unconstrained, as with +-INFINITY in hj_set_constraint): *max_registers
 * gets the largest register count per thread and *max_spill_bytes the
 * largest spill-store size (bytes per thread) over the three stage
 * kernels.  Grids of 2^23 nodes or more are compiled for 2048 resident
 * threads per SM (at most 32 registers), smaller ones for 1536.  Needs no
 * device.  HJ_ERR_ARG on bad arguments, NULL outputs or a con_axes that
 * names no axis of the grid (or one beyond it); HJ_ERR_CUDA when NVRTC is
 * missing, the compile fails or the log holds no resource report. */
hj_status hj_jit_check_resources(int ndim, const int* n, int model, int scheme, int threads,
                                 unsigned con_axes, int* max_registers, int* max_spill_bytes);
/* The same for the row-tile stage kernels of tile_rows lines per block. */
hj_status hj_jit_check_tiles(int ndim, const int* n, int model, int scheme, int tile_rows);
/* The same for the group kernels of a batch of ngrids grids (grid k:
 * ndims[k] axes of shapes[4k..4k+ndims[k]) nodes, models[k], schemes[k]),
 * the kernels a batch runs once they are compiled for its composition. */
hj_status hj_jit_check_group(int ngrids, const int* ndims, const int* shapes, const int* models,
                             const int* schemes);

/* Device memory allocator hook (no counterpart in the paper: an interop
 * convention of the boundary).  By default the library allocates its
 * device memory with cudaMalloc and returns it with cudaFree.  A caller
 * whose device memory belongs to a pool (PyTorch's caching allocator, for
 * one) can route those allocations through it instead:
 *   - alloc(bytes, device, user) returns `bytes` of device memory on
 *     `device` (the current device at the call), aligned to at least 256
 *     bytes, or NULL when it has none; free(ptr, device, user) takes it back.
 *   - The hook in force when a grid, a server or a batch is created serves
 *     all of that object's device allocations, including the ones made
 *     later (stage fields, disturbance and constraint fields, query and
 *     filter staging) and their release at destroy.  Pinned host buffers
 *     are not affected.
 *   - hj_set_allocator(NULL, NULL, NULL) restores cudaMalloc / cudaFree for
 *     objects created afterwards.  Giving only one of the two functions is
 *     HJ_ERR_ARG.
 *   - The hook may be called from the server's worker thread.  The library
 *     synchronises the object's stream before it frees memory, so a pool
 *     that reuses freed blocks on another stream sees no pending work.
 * A NULL from alloc makes the call that needed the memory fail with
 * HJ_ERR_OOM. */
typedef void* (*hj_alloc_fn)(size_t bytes, int device, void* user);
typedef void (*hj_free_fn)(void* ptr, int device, void* user);
hj_status hj_set_allocator(hj_alloc_fn alloc, hj_free_fn free_fn, void* user);

/* Number of nodes of the grid. */
long long hj_grid_points(hj_grid g);

/* Thread-local message describing the last failure of this thread. */
const char* hj_last_error(void);

/* Number of kernels this library has launched in the process so far.
 * Graph replays count each kernel node. */
unsigned long long hj_kernel_launches(void);

#ifdef __cplusplus
}
#endif
#endif /* HJ_H */
