/*
 * hjb.h -- C ABI of the GB300 semi-Lagrangian HJB library.
 *
 * The library solves the discrete Hamilton-Jacobi-Bellman fixed point
 * V = T(V) of Festa, "Reconstruction of independent sub-domains for a class
 * of Hamilton Jacobi equations and its application to parallel computing"
 * (arXiv:1405.3521), Sec. 3, eq. (SL)/(Tdef), for discounted optimal control
 * (the Kruzhkov-transformed minimum-time problem when lambda = 1, l = 1):
 *
 *   [T(V)]_i = beta * min_{a in A} I[V](x_i + h f(x_i, a)) + gamma * l_i   (x_i free)
 *   [T(V)]_i = 0                                                           (x_i target)
 *   beta = exp(-lambda h),  gamma = (1 - beta) / lambda,
 *
 * with I the multilinear (Q1) interpolation on a structured grid, a foot
 * strictly outside the closed box taking the value `value_out` (the image of
 * the paper's +infinity on ghost nodes), and the reconstruction (RA, Sec. 3)
 * and decomposed solve (ISA, Sec. 4) of independent sub-domains.  Options
 * select the printed step weights 1/(1 + lambda h), h/(1 + lambda h) and P1
 * interpolation on triangles (hjb_discount), and differential games with
 * the max over a second player's control b outside the min over a
 * (hjb_controls).
 *
 * Conventions for every entry point:
 *  - Return value: HJB_OK (0) or a negative HJB_ERR_* code.  The message of
 *    the last failure on the calling thread is returned by hjb_last_error().
 *  - Arrays are node fields in row-major order with x fastest:
 *    2D [ny][nx], 3D [nz][ny][nx].
 *  - Array arguments may be device memory or host memory; the library
 *    classifies each pointer (cudaPointerGetAttributes).  Host inputs are
 *    copied to device workspaces and host outputs are copied back, on the
 *    given stream, inside the call.  Device inputs are read in place.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream).  Every
 *    call enqueues its work on that stream and returns after the stream has
 *    completed it, so outputs and statistics are valid on return.
 *  - The caller owns every array it passes.  A problem keeps the field
 *    pointers given to hjb_create and reads them at every call: they must
 *    stay valid and unchanged in meaning until hjb_destroy.  The library owns
 *    only its workspaces (iteration buffers, work lists, graphs).
 *  - Calls on one problem are not thread-safe; distinct problems are
 *    independent.
 */
#ifndef HJB_H
#define HJB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HJB_OK 0
#define HJB_ERR_INVALID_ARG (-1)   /* bad descriptor, size or pointer */
#define HJB_ERR_CUDA (-2)          /* a CUDA call failed (message says which) */
#define HJB_ERR_OOM (-3)           /* device allocation failed */
#define HJB_ERR_NOT_CONVERGED (-4) /* max_iters reached; outputs and stats are valid */
#define HJB_ERR_UNSUPPORTED (-5)   /* valid but not supported combination */
#define HJB_ERR_TIMEOUT (-6)       /* a bounded device wait gave up; outputs invalid */

#define HJB_MAX_CONTROLS 128
#define HJB_MAX_TARGETS 32
/* Problems per hjb_solve_batch call, and tiles per grid: the sweep's work
 * queue addresses a tile of a problem in one 31-bit word (9 bits of problem,
 * 22 bits of tile).  A tile is 32 x 2 nodes at the smallest 2D shape and
 * 32 x 8 x 2 in 3D, so a 2D grid holds up to about 2.7e8 nodes. */
#define HJB_MAX_BATCH 512
#define HJB_MAX_TILES (1 << 22)

/* Structured grid of Sec. 3 (a uniform lattice in each dimension).  Non-periodic
 * dimension d has n[d] >= 2 nodes x = lo + i (hi-lo)/(n-1); a periodic
 * dimension has n[d] nodes on the period [lo, hi): x = lo + i (hi-lo)/n. */
typedef struct {
    int ndim;          /* 2 or 3 */
    int n[3];          /* nodes per dimension, x first */
    double lo[3];
    double hi[3];
    int periodic[3];   /* 0/1 per dimension */
} hjb_grid;

/* Dynamics f(x, a) of Sec. 2: trajectories solve y' = f(y, a).
 *  HJB_DYN_SPEED_CURRENT (2D): f = s(x) a + c(x), a in R^2 a control.
 *     speed: node field s [N] (device or host), NULL means s = 1;
 *     log_speed: node field theta [N] with s = exp(theta) (use one of the two);
 *     scale: node field D [N][2] of per-axis factors, f = diag(D(x)) a + c(x)
 *            (instead of speed / log_speed; Sec. 5, Example ex4);
 *     current: node field c [N][2], NULL means c = 0.
 *     With a second player (hjb_controls.count_b > 0) the control enters
 *     as a - b: f = D(x) (a - b) + c(x).
 *  HJB_DYN_DUBINS (3D, dimension 2 is the heading theta, periodic):
 *     f = (v cos theta, v sin theta, u), u a scalar control; v = dubins_v. */
#define HJB_DYN_SPEED_CURRENT 0
#define HJB_DYN_DUBINS 1
typedef struct {
    int kind;
    const float *speed;
    const float *current;
    const float *log_speed;
    double dubins_v;
    const float *scale;
} hjb_dynamics;

/* Running cost l > 0 (hypothesis H0): a node field [N], or the constant
 * l_const when l == NULL.  A constant cost lets the solver iterate on
 * W = l/lambda - V (a pure max-plus-scaling form, see hjb_solve_opts). */
typedef struct {
    const float *l;
    double l_const;
} hjb_cost;

/* Scheme parameters (Sec. 3): fictitious time step h, discount rate
 * lambda > 0, step weights and interpolation.
 *  weights: HJB_WEIGHTS_EXP (0): beta = exp(-lambda h), gamma = (1 - beta) /
 *           lambda, the exact discount over one step;
 *           HJB_WEIGHTS_IMPLICIT (1): beta = 1 / (1 + lambda h), gamma =
 *           h / (1 + lambda h), the weights printed in the scheme of Sec. 3.
 *           Both give the value l / lambda for a constant cost l.
 *  interp:  HJB_INTERP_Q1 (0): multilinear on the cell;
 *           HJB_INTERP_P1 (1, 2D only): linear on the triangle of the cell's
 *           split along its (0,0)-(1,1) diagonal that holds the foot (the
 *           linear interpolation in n dimensions the scheme of Sec. 3
 *           names).  P1 problems run the generic-count kernel;
 *           hjb_backward and hjb_solve_static take Q1 only. */
#define HJB_WEIGHTS_EXP 0
#define HJB_WEIGHTS_IMPLICIT 1
#define HJB_INTERP_Q1 0
#define HJB_INTERP_P1 1
typedef struct {
    double h;
    double lambda;
    int weights;
    int interp;
} hjb_discount;

/* Discrete control set A (Sec. 3 replaces the control space by a finite
 * set), host memory [count][dim], copied at hjb_create.  dim = 2 for
 * HJB_DYN_SPEED_CURRENT, 1 for HJB_DYN_DUBINS.  count <= HJB_MAX_CONTROLS.
 * Differential games (Sec. 2, the max over b of the min over a; Example
 * ex4): count_b > 0 gives the second player's set B, host [count_b][dim],
 * and T(V)_i = beta max_b min_a I[V](x_i + h f(x_i, a, b)) + gamma l_i.
 * 2D speed/current dynamics only; count * count_b <= HJB_MAX_CONTROLS; not
 * supported by hjb_backward and hjb_solve_static.  count_b = 0: no second
 * player. */
typedef struct {
    int count;
    int dim;
    const float *a;
    int count_b;
    const float *b;
} hjb_controls;

/* Target (the boundary set Gamma / dG of Sec. 3, with exit cost g = 0),
 * split into components Gamma_1..Gamma_m (Sec. 2, eq. HJD): labels [N],
 * 0 = free node, k in 1..n_targets = node of component k.
 * value_out: value of a foot outside the box and of ghost nodes; the
 * natural choice is l/lambda (the cost of never arriving), 1 for the
 * Kruzhkov transform. */
typedef struct {
    const uint8_t *labels;
    int n_targets; /* m <= HJB_MAX_TARGETS */
    double value_out;
} hjb_target;

typedef struct hjb_problem hjb_problem;

/* Create a problem.  Validates every descriptor, classifies the field
 * pointers, copies the control set, and sizes (but does not yet allocate)
 * the workspaces.  On success *out receives the handle.
 * Errors: HJB_ERR_INVALID_ARG (bad sizes, NULL required pointers, non-finite
 * controls or scalars), HJB_ERR_UNSUPPORTED (among others: a grid of more
 * than HJB_MAX_TILES tiles).  The foot displacement is checked by the solve
 * calls, which need the fields: HJB_ERR_UNSUPPORTED when a foot moves 4 or
 * more cells per step (2D), or 2 or more in (x, y) or 1 or more in theta
 * (Dubins). */
int hjb_create(const hjb_grid *grid, const hjb_dynamics *dyn, const hjb_cost *cost,
               const hjb_discount *disc, const hjb_controls *controls,
               const hjb_target *target, hjb_problem **out);

/* Free the problem and all its workspaces.  NULL is accepted. */
int hjb_destroy(hjb_problem *p);

/* Options of an iterative solve.
 *  tol: stop when ||V^{n+1} - V^n||_inf <= tol (the stopping remark of
 *       Sec. 3); by the contraction bound the distance to the fixed point is
 *       then at most beta/(1-beta) tol.  tol <= 0 selects 0.5e-4 (1 - beta),
 *       which guarantees 1e-4 in exact arithmetic.
 *  max_iters: cap on sweeps (<= 0: 100,000).
 *  use_w_form: 1 = iterate on W = l/lambda - V (constant cost only),
 *       0 = iterate on V, -1 = automatic (W form when the cost is constant).
 *  v_init: optional warm start [N] (a previous solution), NULL = start from
 *       value_out on free nodes and 0 on targets (a supersolution).  In
 *       hjb_solve_decomposed every sub-domain starts from it on its own nodes
 *       (for example a coarse solution interpolated onto the fine grid, the
 *       coarse-to-fine warm start between ISA steps 2 and 3); from a start
 *       that is not a supersolution the iteration still converges (T is a
 *       contraction) but not monotonically.
 *  sweeps_per_check: sweeps between two convergence tests in the device loop
 *       (<= 0: library default).
 *  local_iters: applications of T to each staged tile per sweep (<= 0:
 *       default 6, 4 for a game, 16 at most).  The first reads the previous
 *       sweep's values; each further one reads the tile's own latest values
 *       with the halo held (block Gauss-Seidel inside the tile), and a tile stops early
 *       once an application changes none of its nodes.  Every ordering of the
 *       updates has the same fixed point, and a sweep is still a
 *       beta-contraction, so tol keeps its meaning.  1 is plain value
 *       iteration (Jacobi).
 *  subdomain_targets (hjb_solve_decomposed only): the targets of sub-problem
 *       k.  HJB_SUBDOMAIN_TARGETS_ALL (0, default): every target node inside
 *       the sub-domain (the operator of Sec. 4 step 3 as written); equal
 *       sub-domains are then solved once.  HJB_SUBDOMAIN_TARGETS_OWN (1):
 *       only component k, the target choice of the auxiliary problems of RA
 *       step 1 (Sec. 3); nodes of other components inside it are free.
 *  n_subdomains (hjb_solve_decomposed only): the sub-domains of fine_mask,
 *       bits 0 .. n_subdomains - 1 (<= 0: n_targets); more than n_targets
 *       come from re-split components (hjb_ra_opts.max_splits) and need
 *       HJB_SUBDOMAIN_TARGETS_ALL.
 *  warm_start (hjb_solve_decomposed only, 2D): 1 = start sub-domain k from
 *       the Q1 interpolation onto the fine grid of the coarse auxiliary
 *       solution V_k of the problem's last hjb_subdomains call (a
 *       coarse-to-fine warm start between ISA steps 2 and 3; that call must
 *       have kept the division, and the iterated form must match); 0 = the
 *       usual start.  The fixed point does not depend on the start. */
#define HJB_SUBDOMAIN_TARGETS_ALL 0
#define HJB_SUBDOMAIN_TARGETS_OWN 1
typedef struct {
    double tol;
    int max_iters;
    int use_w_form;
    const float *v_init;
    int sweeps_per_check;
    int local_iters;
    int subdomain_targets;
    int n_subdomains;
    int warm_start;
} hjb_solve_opts;

/* Statistics of one solve (per problem or per sub-domain). */
typedef struct {
    int iterations;        /* sweeps (with local_iters 1: applications of T) */
    int converged;         /* 1: the residual reached tol; 2: it stopped decreasing at the
                              FP32 rounding floor (accepted); 0: not converged */
    long long node_updates;/* evaluations of T at free nodes (all controls), every
                              application inside a tile counted */
    double final_residual; /* last ||V^{n+1} - V^n||_inf */
    double ms;             /* device time of the call, milliseconds */
    long long ties;        /* label decisions within 1e-6 of the threshold */
    long long labelled;    /* sum over sub-domains of their node counts */
    long long launches;    /* CUDA kernels the call launched */
    int tile_rows;         /* rows of the 2D tiles the sweeps ran on (32 x 8, 4 or 2 nodes:
                              the autotuner's choice or HJB_TILE_ROWS); 0 for 3D */
    int tile_lanes;        /* lanes per node of those tiles (1, or 2: a_j and -a_j) */
    double delta;          /* hjb_subdomains: the threshold of RA step 3 it applied */
    double lipschitz;      /* hjb_subdomains: the M of that threshold (estimated when
                              hjb_ra_opts.M < 0 and delta < 0; 0 when delta was given) */
    int local_iters;       /* applications of T per staged tile and sweep that ran */
    int subdomains;        /* hjb_subdomains: components of the returned division */
    long long largest;     /* hjb_subdomains: nodes of its largest projected sub-domain */
    long long tile_visits; /* tiles staged and processed by the sweeps (each visit applies T
                              1 to local_iters times to the tile's nodes) */
    int tile_layers;       /* 3D: heading layers of the 32 x 8 tiles (4 or 2); 0 in 2D */
} hjb_stats;

/* Full-domain solve of V = T(V) by value iteration V^{n+1} = T(V^n)
 * (Sec. 3, eq. SL and the iteration following it).  v_out [N] receives V.
 * Returns HJB_ERR_NOT_CONVERGED (outputs valid) when max_iters is hit. */
int hjb_solve(hjb_problem *p, const hjb_solve_opts *opts, float *v_out, hjb_stats *stats,
              void *stream);

/* Options of the reconstruction (RA, Sec. 3, and ISA steps 1-2, Sec. 4).
 *  coarse_stride[d]: the coarse grid K is every stride-th fine node (the
 *       superimposed grids of the projection remark); (n-1) % stride == 0
 *       for non-periodic dimensions, n % stride == 0 for periodic ones.
 *  h_coarse: time step on K (<= 0: h * coarse_stride[0]).
 *  delta: threshold of eq. (rep), |V_k - V| <= delta (Prop. 3.1);
 *       delta < 0 selects 2 (C dx_K^q + M dx_K) with the C, M, q below.
 *  tol / max_iters: stopping rule of the auxiliary solves (RA step 1).
 *  max_splits, split_gain, split_labels: recursive re-splitting of the
 *       target components (the Conclusions: the unbalanced sub-domains of
 *       Example ex3 can be balanced by refining the division of Gamma
 *       recursively).  Each step splits the component whose projected
 *       sub-domain is largest (lowest index on ties) in two, along the x or y
 *       grid axis of larger index extent of its target nodes (x on ties):
 *       nodes with index at most s keep it, the others become component m + 1,
 *       s the smallest index holding at least half of its nodes (the next
 *       lower occupied index when that would leave the second part empty).
 *       RA and the projection are re-run with the first division's threshold
 *       (V = min_k V_k, hence the estimated M, does not change); the step is
 *       kept when both parts' sub-domains are smaller than (1 - split_gain)
 *       times the split one's, and the refinement stops at the first step
 *       that is not, after max_splits steps, at HJB_MAX_TARGETS components,
 *       or at a component that cannot be split.  The fine mask then has
 *       stats.subdomains bits; solve it with hjb_solve_decomposed and
 *       hjb_solve_opts.n_subdomains = stats.subdomains (the sub-problems'
 *       targets are the target nodes inside them, so the original labels
 *       serve), or pass split_labels to hjb_create.  v_aux_out must then be
 *       NULL. */
typedef struct {
    int coarse_stride[3];
    double h_coarse;
    double delta;
    double C, M, q;
    double tol;
    int max_iters;
    int max_splits;         /* recursive re-splitting steps (0: none; at most 32) */
    double split_gain;      /* a split is kept when both parts' sub-domains are below
                               (1 - split_gain) times the split one's (0: 0.05) */
    uint8_t *split_labels;  /* optional output [N]: the target labels of the final
                               division (device or host memory) */
} hjb_ra_opts;

/* RA (Sec. 3, steps 1-3) on the coarse grid followed by ISA step 2
 * (projection through the concave hull Con, Sec. 4).
 *  fine_mask_out [N]: bit k-1 set iff the fine node lies in the projected
 *       sub-domain of target component k.
 *  coarse_labels_out [N_K] (optional): the coarse labels (same bit layout).
 *  v_aux_out [m][N_K] (optional): the auxiliary solutions V_k of step 1.
 *  stats (optional): iterations = max over the auxiliary solves,
 *       node_updates = their sum, ties = label decisions within 1e-6 of
 *       delta, labelled = sum over k of |Sigma_k| on the fine grid. */
int hjb_subdomains(hjb_problem *p, const hjb_ra_opts *ra, uint32_t *fine_mask_out,
                   uint32_t *coarse_labels_out, float *v_aux_out, hjb_stats *stats,
                   void *stream);

/* ISA steps 3-4 (Sec. 4): for every k, iterate V_k = T(V_k) restricted to
 * the nodes with bit k-1 of fine_mask (every target node inside is kept as
 * a target, or only those of component k with opts->subdomain_targets =
 * HJB_SUBDOMAIN_TARGETS_OWN; nodes outside are ghosts with value
 * value_out), all sub-domains
 * in one persistent launch with per-sub-domain convergence; then
 * Vbar(j) = min{ V_k(j) : bit k-1 of fine_mask[j] }.  Nodes in no
 * sub-domain receive value_out.
 *  per_subdomain (optional): [n_targets] statistics; total (optional). */
int hjb_solve_decomposed(hjb_problem *p, const uint32_t *fine_mask, const hjb_solve_opts *opts,
                         float *v_out, hjb_stats *per_subdomain, hjb_stats *total,
                         void *stream);

/* Many independent problems (uneven grids allowed) in one persistent,
 * graph-captured launch with per-problem convergence.  All problems must use
 * the same dynamics kind, control set size and cost form; count <=
 * HJB_MAX_BATCH (HJB_ERR_INVALID_ARG otherwise).
 *  v_out[i] [N_i] receives problem i's V; per_problem (optional) [count]. */
int hjb_solve_batch(hjb_problem *const *problems, int count, const hjb_solve_opts *opts,
                    float *const *v_out, hjb_stats *per_problem, void *stream);

/* Adjoint of the converged fixed point with respect to a node field theta
 * (not in the paper: the transposed linear system of V = beta P_pi V + b
 * with the optimal policy pi frozen and recomputed from v):
 *     (I - beta P_pi)^T lambda = grad_v,
 *  pi_i = argmin_j I[v](foot_j), lowest index on ties, is decided in FP64
 *  arithmetic (the argmin of an FP32 evaluation picks other controls
 *  wherever neighbouring directions differ by less than their rounding,
 *  which moves adjoint mass), and on refined values: the FP32 v differs from
 *  the FP64 fixed point by the rounding carried along the characteristics,
 *  so the policy taken on v is frozen, the FP64 residual r of its linear
 *  system is formed, the correction dv = r + beta P_pi dv is iterated in FP32
 *  to its rounding floor (block Gauss-Seidel sweeps over staged tiles), and
 *  pi is decided again on v + dv (one round; the environment variable
 *  HJB_ADJ_REFINE sets 0-4 rounds).  stats->ties counts the free nodes whose
 *  two best control values differ by at most 1e-6, stats->local_iters the
 *  sweeps of the refinement.
 *  wrt = 0: grad_out = dL/dtheta for the log-speed field (s = exp(theta),
 *           HJB_DYN_SPEED_CURRENT):  lambda_i beta h s_i grad I[V](y_i) . a_pi(i)
 *  wrt = 1: grad_out = dL/dl for the cost field: lambda_i gamma.
 *  v [N]: the converged solution; grad_v [N]: dL/dV.  lambda is iterated by
 *  block Gauss-Seidel sweeps over 32 x 8 tiles (16 applications per staged
 *  tile and sweep, the halo held; HJB_ADJ_APPS sets 8, 16 or 32);
 *  stats->iterations counts the sweeps.
 *  opts->tol (optional, > 0) stops the iteration once a sweep changes lambda
 *  by at most tol (stats->converged = 1).  It always stops
 *  (stats->converged = 2) at the summation-order floor of the FP32
 *  accumulation: a change within 32 ulp of max|lambda|, or no new minimum of
 *  the change for 64 sweeps once it is below 1024 ulp of max|lambda|.
 *  Otherwise HJB_ERR_NOT_CONVERGED after opts->max_iters sweeps.  Feet of
 *  more than 6 cells (h |f| / dx) are HJB_ERR_UNSUPPORTED.  stats
 *  (optional). */
int hjb_backward(hjb_problem *p, const float *v, const float *grad_v, int wrt,
                 const hjb_solve_opts *opts, float *grad_out, hjb_stats *stats, void *stream);

/* Values of I[V] at P points [P][ndim] (physical coordinates, clamped into
 * the box) and, if grad_v != NULL, the gradient of the loss
 * L = (1/P) sum_p I[V](points_p) with respect to V, written to grad_v [N]. */
int hjb_point_values(hjb_problem *p, const float *v, const float *points, int P, float *values,
                     float *grad_v, void *stream);

/* Allocation-free full-domain solve.  The paper has no counterpart: this is
 * a deployment variant of hjb_solve for callers that cannot allocate device
 * memory while they run: real-time control loops, where cudaMalloc and
 * cudaFree may synchronise the device and take unbounded time, so they are
 * forbidden after start-up; and plug-ins or embedded solvers whose host
 * application owns every device allocation (its own pool and memory
 * budget), so the library may not add allocations of its own.  It takes
 * the descriptors of hjb_create directly (no problem object) and runs the
 * same sweep kernel as hjb_solve in one cooperative launch.
 *
 * Its working memory (iteration buffers, work queue, control block) lives in
 * a single 4 MiB file-scope device array that every GPU loading the library
 * holds until the process exits.  Limits: 2D speed/current dynamics,
 * n[0] * n[1] <= 262144 nodes and the layout must fit the 4 MiB (a grid
 * whose rows are padded to 32 floats, two buffers); larger grids are
 * rejected with HJB_ERR_INVALID_ARG and a message saying so.
 * Every array argument must be device memory (host arrays would need
 * staging buffers): host pointers are rejected with HJB_ERR_INVALID_ARG.
 * No cudaMalloc, cudaFree or allocating library call is made.  The call
 * reads the largest field magnitudes back to the host (to pick the
 * interpolation halo) and synchronises the stream before it returns.
 *
 * The array's device address is looked up (cudaGetSymbolAddress) by the
 * first call on each device, with that device current; that first call
 * should come before any stream capture.  All calls share the array, which
 * keeps the last call's contents, so calls that may overlap on the GPU
 * (other streams, other host threads) race: serialise them.  Each call
 * re-initialises every part of the array it reads.  Outputs and statistics
 * as for hjb_solve. */
int hjb_solve_static(const hjb_grid *grid, const hjb_dynamics *dyn, const hjb_cost *cost,
                     const hjb_discount *disc, const hjb_controls *controls,
                     const hjb_target *target, const hjb_solve_opts *opts, float *v_out,
                     hjb_stats *stats, void *stream);

/* Autotuner table (not in the paper: a property of this implementation).
 * hjb_solve, hjb_solve_decomposed and hjb_solve_batch run the sweep with a
 * tile shape (tile_rows: 2D tiles of 32 x 8, 32 x 4 or 32 x 2 nodes, with
 * 1, 2 or 4 warp groups splitting the controls of a node, or for 32 x 4
 * tiles lanes = 2 lanes per node; fixed at 8 for Dubins, games and P1; for
 * Dubins 32 x 8 tiles of 4 or 2 heading layers) and a number of
 * applications of T per staged tile and sweep (local_iters).  The first call for a problem class on a device runs the
 * whole call once per candidate on the caller's data and keeps the fastest
 * (ms: its device time) in a table keyed by
 *     "<device name>/<SM count>|<full|decomposed|batch>|<class fields>".
 * The table is also filled, at the first call that needs it, from the file
 * tune_cache.json of the package directory (one level above the directory
 * holding libhjb.so; read only) and then from the file named by the
 * environment variable HJB_TUNE_CACHE (read, and rewritten after every
 * tuning).  HJB_TUNE=off never times a call: it takes the table's choice or
 * the default (tile_rows 8, local_iters 6, 4 for a game), so that repeated
 * runs are bit for bit reproducible; HJB_TUNE=force times even when the
 * table holds a choice.  HJB_TILE_ROWS and HJB_LOCAL_ITERS (or
 * hjb_solve_opts.local_iters) pin their axis.  The file is a JSON array of
 * {"key": ..., "rows": ..., "lanes": ..., "layers": ..., "local_iters": ...,
 * "ms": ...} objects, one per line.  HJB_TILE_LANES=1|2 pins the lanes.  The
 * reconstruction (hjb_subdomains, key op "ra") tunes its auxiliary solves
 * the same way; there tile_rows = 1 selects the on-chip solve of a 2D
 * coarse grid (one thread-block cluster per auxiliary problem, iterating in
 * shared memory), and HJB_RA=tiles|chip pins the path.  HJB_TUNE_VERBOSE
 * prints every timed candidate to stderr.  Errors: HJB_ERR_INVALID_ARG (NULL argument, unknown key, a choice
 * out of range, a file that cannot be opened). */
typedef struct {
    int tile_rows;
    int lanes;         /* 1, or 2 (32 x 4 tiles): two lanes per node taking a_j and -a_j, for
                          control sets whose second half is the negated first half */
    int local_iters;
    double ms;
    int layers;        /* 3D (Dubins): heading layers per 32 x 8 tile, 4 or 2 */
} hjb_tune_choice;
int hjb_tune_get(const char *key, hjb_tune_choice *out);
int hjb_tune_set(const char *key, const hjb_tune_choice *choice);
int hjb_tune_load(const char *path, int *entries); /* merges the file's entries (they win) */
int hjb_tune_save(const char *path);               /* writes every entry of the table */
int hjb_tune_clear(void);                           /* empties the table (files not re-read) */

/* Message of the last failure on this thread ("" if none). */
const char *hjb_last_error(void);

/* Library version string. */
const char *hjb_version(void);

#ifdef __cplusplus
}
#endif

#endif /* HJB_H */
