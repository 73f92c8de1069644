/*
 * rkhsba.h -- C ABI of the GB300 (sm_103a) RKHS-BA hot path.
 *
 * The library evaluates the correspondence-free multi-frame objective of
 * RKHS-BA (Zhang et al., arXiv 2403.01254):
 *
 *   F(T) = sum_{(a,b) in C} sum_{i,j} c_ij * sigma^2 exp(-|T_a x_i - T_b y_j|^2 / (2 ell^2))
 *
 * (Eq. inner_product_actual_ba with the squared-exponential kernel of
 * Eq. kernel), restricted to point pairs closer than r_c = cutoff_mult * ell
 * (the sparse double sum of Sec. III-B), together with its gradient under the
 * right perturbation T exp(eps^), eps = [rho; phi] (Eq. inner_product_reformat)
 * and the Gauss-Newton matrix of the IRLS cost (Eq. irls_final), and runs the
 * damped Gauss-Newton (Levenberg-Marquardt) pose solve with the first frame
 * fixed (Sec. V-A).  All work runs in CUDA kernels on one GPU.
 *
 * Conventions shared by every call
 *  - Frames are numbered 0..K-1.  Points are given frame after frame in one
 *    flat array; n_points[m] says how many belong to frame m (0 allowed).
 *  - Poses are frame-to-world SE(3) matrices, 4x4 row-major float64, K of
 *    them back to back (16*K doubles).  Their rotation blocks must satisfy
 *    |R^T R - I|_max <= 1e-9 (else RKHSBA_EINVAL).
 *  - Edges are unordered frame pairs (a, b), a != b, each pair at most once;
 *    the library orders each as (min, max).
 *  - Gradient and Hessian coordinates are per frame [rho(3), phi(3)] in the
 *    frame's own (body) axes, frame after frame (6*K entries).
 *  - loss = -F (lower is better).  grad = d loss / d eps = (sigma^2/ell^2) * b
 *    with b = sum w J^T d; H = sum w J^T J, the IRLS Gauss-Newton matrix,
 *    where w_ij = c_ij exp(-|d_ij|^2 / (2 ell^2)) (Eq. irls_weight),
 *    d_ij = T_a x_i - T_b y_j, J = d d_ij / d eps.
 *  - c_ij = <l_i, l_j> (label vectors, sem_dim floats per point) times
 *    exp(-|col_i - col_j|^2 / (2 ell_color^2)) when colours are given and
 *    ell_color > 0 (the tensor-product label of Sec. III-A); with neither,
 *    c_ij = 1 (plain kernel correlation).
 *  - Host pointers are read during the call only; the library copies what it
 *    keeps.  Output buffers are caller-allocated.  Every call returns a
 *    status and never throws; rkhsba_last_error() gives a message.
 *  - A context is not thread-safe: one host thread at a time.
 *  - Limits: sum of points < 2^31, sem_dim <= 32, 1 <= K <= 4096 frames,
 *    |coordinate| / (1.001 * r_c) < 2^29.
 */
#ifndef RKHSBA_H
#define RKHSBA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rkhsba_ctx rkhsba_ctx;

typedef enum {
    RKHSBA_OK = 0,
    RKHSBA_EINVAL = 1,    /* invalid argument or input data (NaN/Inf, bad pose, bad edge) */
    RKHSBA_ENOMEM = 2,    /* device allocation failed */
    RKHSBA_ECUDA = 3,     /* CUDA runtime error */
    RKHSBA_ENOTCONV = 4,  /* solve stopped at max_iters before converging */
    RKHSBA_ETIMEOUT = 5,  /* a bounded device wait gave up */
    RKHSBA_EBUSY = 6      /* resource exhausted (server slots / memory) */
} rkhsba_status;

/* Kernel and solver parameters.  Zero means "default" for every field. */
typedef struct {
    double ell;          /* lengthscale ell of Eq. kernel, metres, > 0 (required) */
    double cutoff_mult;  /* r_c = cutoff_mult * ell (default 3) */
    double sigma;        /* sigma of Eq. kernel (default 1) */
    double ell_color;    /* colour lengthscale; <= 0 disables the colour factor */
    int32_t sem_dim;     /* floats per label vector, 0..32; 0 = no labels */
    int32_t sem_bf16;    /* 1: keep labels on the device as bfloat16 (rounded) */
    int32_t max_iters;   /* LM evaluations after the first (default 100) */
    int32_t top_k;       /* 0: every pair inside r_c (default).  1..8: for every point
                            of an edge's second frame only the top_k pairs of largest
                            w count (the 8-neighbour variant of Sec. VI, time
                            analysis; ties: the candidate met first in the
                            grid's cell order) */
    double lambda0;      /* initial LM damping (default 1e-4) */
    double tol_step;     /* stop when an accepted step has |delta|_inf below (1e-10) */
    double tol_rel_f;    /* stop when an accepted step gains less than this relative F (1e-12) */
    double sem_min;      /* > 0: drop pairs whose semantic kernel <l_i, l_j> is below
                            sem_min (the semantic pruning of Sec. VII); 0: off */
    double cell_scale;   /* grid cell edge h = cell_scale * r_c * (1 + 2^-10), 1..4
                            (default 1).  Larger cells put more queries in a unit
                            and more candidates in the 27-cell stencil; results
                            do not depend on it beyond FP32 rounding (the
                            autotuner picks it per workload) */
} rkhsba_params;

typedef struct {
    int32_t iters;       /* evaluations after the first */
    int32_t status;      /* RKHSBA_OK converged, RKHSBA_ENOTCONV hit max_iters */
    double final_loss;   /* -F at the returned poses */
    double lambda;       /* damping at exit */
    int64_t pair_terms;  /* pair-terms summed over every evaluation of the solve */
} rkhsba_solve_info;

/*
 * rkhsba_create -- upload a problem and build its per-frame uniform grids.
 *
 * Problem statement of Sec. III: frames X_m of 3-D points, pose graph C,
 * pose-invariant labels l(x) (Sec. III-A), kernel parameters of Eq. kernel.
 *
 *   out        receives the new context (NULL on failure)
 *   n_frames   K >= 1
 *   n_points   [K] points per frame (>= 0)
 *   xyz        [sum n_points * 3] float64, frame-local coordinates, HOST memory
 *   sem        [sum n_points * sem_dim] float32 labels, or NULL (requires sem_dim == 0)
 *   rgb        [sum n_points * 3] float32 colours, or NULL
 *   n_edges    >= 1
 *   edges      [n_edges * 2] int32 frame indices
 *   params     see rkhsba_params; params->ell > 0
 *   cuda_stream  cudaStream_t to run on (NULL: the library's own stream)
 *
 * Errors: EINVAL for NaN/Inf coordinates, labels or colours, empty pose
 * graph, self/duplicate/out-of-range edges, unsupported sem_dim or limits;
 * ENOMEM / ECUDA from the device.  The context owns all device memory.
 */
rkhsba_status rkhsba_create(rkhsba_ctx** out, int32_t n_frames, const int64_t* n_points,
                            const double* xyz, const float* sem, const float* rgb,
                            int32_t n_edges, const int32_t* edges,
                            const rkhsba_params* params, void* cuda_stream);

/* Same as rkhsba_create with xyz / sem / rgb in DEVICE memory (copied). */
rkhsba_status rkhsba_create_device(rkhsba_ctx** out, int32_t n_frames, const int64_t* n_points,
                                   const double* d_xyz, const float* d_sem, const float* d_rgb,
                                   int32_t n_edges, const int32_t* edges,
                                   const rkhsba_params* params, void* cuda_stream);

void rkhsba_destroy(rkhsba_ctx* ctx);

/*
 * rkhsba_eval -- loss, gradient and Gauss-Newton matrix at the given poses
 * (Eq. inner_product_actual_ba, Eq. inner_product_reformat, Eq. irls_final).
 *
 *   poses      [K*16] HOST float64 poses
 *   loss       [1] -F, or NULL
 *   grad       [6K] d loss / d eps, or NULL
 *   H_full     [6K*6K] row-major sum w J^T J, or NULL
 *   H_blocks   [n_edges*144] per-edge 12x12 blocks, rows/cols ordered
 *              [rho_a, phi_a, rho_b, phi_b] with (a, b) = (min, max), or NULL
 *   edge_pairs [n_edges] int64 pair-terms per edge, or NULL
 *
 * Synchronous: returns after the outputs are written.
 */
rkhsba_status rkhsba_eval(rkhsba_ctx* ctx, const double* poses, double* loss, double* grad,
                          double* H_full, double* H_blocks, int64_t* edge_pairs);

/*
 * rkhsba_solve -- damped Gauss-Newton on the IRLS cost with the weights
 * recomputed after every step (Eq. irls_final), frame 0 held fixed, steps
 * accepted while the original cost F increases (Sec. V-C).
 *
 *   poses  [K*16] HOST float64: initial guess in, solution out
 *   info   [1] summary, or NULL
 *
 * Returns RKHSBA_OK when converged, RKHSBA_ENOTCONV at max_iters (poses
 * still hold the best iterate), other codes on error.
 */
rkhsba_status rkhsba_solve(rkhsba_ctx* ctx, double* poses, rkhsba_solve_info* info);

/*
 * Device-resident stepping, for callers that keep everything in HBM.
 * All three are asynchronous on the context stream and do not synchronise.
 *   rkhsba_set_poses_device  copy K*16 float64 poses from DEVICE memory and
 *                            reset the LM state (lambda0, iteration 0)
 *   rkhsba_rebuild           rebuild the per-frame grids from the resident
 *                            points (the grid step; poses untouched)
 *   rkhsba_iterate           run n LM iterations (each one solve, one
 *                            evaluation and one accept/reject); the first
 *                            call after set_poses also evaluates the start
 * rkhsba_get_state synchronises and copies poses [K*16] / info to the host.
 */
rkhsba_status rkhsba_set_poses_device(rkhsba_ctx* ctx, const double* d_poses);
rkhsba_status rkhsba_rebuild(rkhsba_ctx* ctx);
rkhsba_status rkhsba_iterate(rkhsba_ctx* ctx, int32_t n_iters);
rkhsba_status rkhsba_get_state(rkhsba_ctx* ctx, double* poses, rkhsba_solve_info* info);

/*
 * rkhsba_edge_pairs -- the pair set of one edge at the given poses, as found
 * by the device radius search (for verification).
 *
 *   poses     [K*16] HOST float64
 *   edge      index into the create() edge list
 *   capacity  length of i_out / j_out
 *   i_out     [capacity] int32 point index within frame a = min(edge)
 *   j_out     [capacity] int32 point index within frame b = max(edge)
 *   n_out     total pairs (may exceed capacity; then only capacity written)
 * Pairs are returned in no particular order.
 */
rkhsba_status rkhsba_edge_pairs(rkhsba_ctx* ctx, const double* poses, int32_t edge,
                                int64_t capacity, int32_t* i_out, int32_t* j_out,
                                int64_t* n_out);

/*
 * rkhsba_profile -- CUDA-event timing of the phases of the hot path on the
 * context stream: [0] grid build, [1] transforms + query binning, [2] pair
 * kernel, [3] FP64 assembly, [4] LM solve + accept.
 *   enable    1: clear and start recording; 0: stop recording
 *   ms        [5] summed milliseconds of the recorded launches, or NULL
 *   launches  [5] number of recorded launches per phase, or NULL
 * Reading (ms or launches non-NULL) synchronises the stream.
 */
rkhsba_status rkhsba_profile(rkhsba_ctx* ctx, int32_t enable, double* ms, int64_t* launches);

/*
 * rkhsba_eval_static -- the evaluation of rkhsba_eval for a small problem,
 * without allocating any device memory.  The paper has no counterpart; this
 * entry point exists for callers that cannot call cudaMalloc: code living
 * inside another runtime that owns the device memory through its own pool,
 * and real-time loops that must not take allocator locks or face an
 * allocation failure mid-run.
 *
 * Every temporary buffer comes from one fixed 32 MiB device array inside the
 * library (each GPU that loads the library holds it until the process
 * exits).  Limits: n_frames <= 16, n_edges <= 64, total points <= 32768,
 * queries (sum over edges of the points of the larger-index frame) <= 131072,
 * grid cells <= 2^20 over all frames and over all edges' home cells;
 * larger problems return RKHSBA_EINVAL with a message and touch no memory
 * beyond the array.  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture on that device.  All calls share the array and reuse its contents
 * (what must start at zero is cleared in every call); calls whose GPU work
 * overlaps (other streams or other host threads) race on it, so the caller
 * serialises them.
 *
 * The call waits on its stream twice (the host lays out the grids from the
 * frames' bounding boxes, then reads the results back), so it cannot run on
 * a stream that is being captured: it returns RKHSBA_EINVAL there without
 * touching the stream.
 *
 *   n_frames, n_points, edges, params  as for rkhsba_create
 *   d_xyz, d_sem, d_rgb   DEVICE inputs laid out as for rkhsba_create
 *                         (d_sem/d_rgb may be NULL)
 *   poses      [K*16] HOST float64 poses
 *   loss, grad, H_full    HOST outputs as for rkhsba_eval (each may be NULL)
 *   cuda_stream  stream to run on (NULL: the default stream)
 * Synchronous: returns after the outputs are written.
 */
rkhsba_status rkhsba_eval_static(int32_t n_frames, const int64_t* n_points, const double* d_xyz,
                                 const float* d_sem, const float* d_rgb, int32_t n_edges,
                                 const int32_t* edges, const rkhsba_params* params,
                                 const double* poses, double* loss, double* grad, double* H_full,
                                 void* cuda_stream);

/*
 * rkhsba_selftest_lookback_timeout -- failure-detection self-test of the
 * bounded device waits (the paper has no counterpart).  The radix sort of
 * the grid build and of the query binning passes tile counts between blocks
 * by decoupled look-back; every wait on another block's record polls at most
 * a fixed number of times, then raises an error word that the calling entry
 * point reports as RKHSBA_ETIMEOUT (the kernel returns, the context stays
 * usable).  This call makes such a wait run out on purpose: one pass over two
 * tiles of keys whose only block takes the second tile while the first
 * tile's record is never published.
 *
 *   spin_limit        polls before the wait gives up, 1 .. 2^20 (else EINVAL)
 *   writes_in_bounds  HOST out (may be NULL): 1 when the guard words on both
 *                     sides of the output arrays are untouched
 * Returns RKHSBA_ETIMEOUT when the wait gave up (the expected outcome),
 * RKHSBA_OK if it did not, ECUDA on a runtime error.  Allocates and frees its
 * own small buffers; synchronises the device.
 */
rkhsba_status rkhsba_selftest_lookback_timeout(int32_t spin_limit, int32_t* writes_in_bounds);

/* ------------------------------------------------------------------------
 * Function-space distance and cosine (Sec. III-A, Eq. dist_rkhs).
 *
 * A frame X_m is the function f_{T X}(.) = sum_i l(x_i) k(., T x_i) in the
 * RKHS of the kernel; two frames compare through
 *   <f_a, f_b>     = sigma^2 sum_{i,j} c_ij exp(-|T_a x_i - T_b y_j|^2 / 2 ell^2)
 *   |f_a - f_b|^2  = <f_a, f_a> + <f_b, f_b> - 2 <f_a, f_b>
 *   cos(f_a, f_b)  = <f_a, f_b> / (|f_a| |f_b|)
 * with the same sparse sums (pairs closer than r_c) and labels as the
 * objective.  At host poses [K*16] this writes, each output HOST and
 * caller-allocated and each may be NULL:
 *   self_ip [K]  <f_m, f_m> (pose invariant; i = j terms included)
 *   cross_ip[E]  <f_a, f_b> for edge e = (a, b), the objective's per-edge F
 *   dist    [E]  |f_a - f_b|^2
 *   cosine  [E]  cos(f_a, f_b); 0 when a frame has a zero self term
 *   dD_dell [1]  d (sum_e dist[e]) / d ell = sigma^2 / ell^3 * sum c k |d|^2
 *                over the same terms (the cutoff held fixed)
 * The self terms are evaluated on the first call (a second, self-edge
 * context kept with ctx) and reused.  Synchronous.
 * ------------------------------------------------------------------------ */
rkhsba_status rkhsba_inner_products(rkhsba_ctx* ctx, const double* poses, double* self_ip,
                                    double* cross_ip, double* dist, double* cosine, double* dD_dell);

/* Rotation search of Sec. IV-A: frame b is tried against frame a under the
 * 60 rotations R_k of the icosahedral group (the identity; half turns about
 * the 15 axes through opposite edge midpoints; 2pi/3, 4pi/3 about the 10
 * axes through opposite face centres; 2k pi/5, k = 1..4, about the 6 axes
 * through opposite vertices; icosahedron with vertices at the cyclic
 * permutations of (0, +-1, +-phi)).  Candidate k places b at
 *   T_a [R_k | mu_a - R_k mu_b]      (mu = frame-local centroid)
 * and is scored by cos(f_a, f_b); the best candidate has the largest cosine
 * (lowest k on ties).  All 60 candidates are one batched evaluation.
 *   a, b         frames (a != b, both non-empty)
 *   poses        [K*16] HOST; only T_a is read
 *   cosine       [60] HOST out (may be NULL)
 *   rotations    [60*9] HOST out, row-major R_k (may be NULL)
 *   best_pose    [16] HOST out: the pose of b of the best candidate (may be NULL)
 *   best         HOST out: its index k (may be NULL)
 * Device memory: a temporary context with 1 + 60 copies of frame b. */
rkhsba_status rkhsba_rotation_search(rkhsba_ctx* ctx, int32_t a, int32_t b, const double* poses,
                                     double* cosine, double* rotations, double* best_pose,
                                     int32_t* best);

/* Lengthscale decay (Sec. V-C): an outer loop over ell around the LM solve.
 * Level t solves the poses at ell_t (rkhsba_solve's loop, from the previous
 * level's poses), then sets
 *   ell_{t+1} = max(ell_min, ell_t (1 - decay * sign(dD/dell)))
 * with dD/dell as in rkhsba_inner_products at the solved poses.  The loop ends
 * when a level accepts no LM step (the objective at that ell stopped
 * increasing), when ell stops changing, or after max_outer levels.  ctx keeps
 * its own ell; each level runs in a temporary context of the same problem. */
typedef struct {
    double decay;        /* fraction per outer step, in (0, 1) */
    double ell_min;      /* floor of ell (>= 0) */
    int32_t max_outer;   /* levels, >= 1 */
    int32_t reserved;    /* must be 0 */
} rkhsba_ell_schedule;

typedef struct {
    int32_t levels;      /* levels run */
    int32_t status;      /* status of the last level's solve (OK or ENOTCONV) */
    double ell_final;    /* ell of the last level */
    double final_loss;   /* -F at the last level's ell and the returned poses */
    int64_t iters;       /* LM iterations over all levels */
    int64_t pair_terms;  /* pair-terms over all evaluations */
} rkhsba_ell_info;

/*   poses       [K*16] HOST in: initial poses; out: final poses
 *   ell_levels  [max_outer] HOST out: ell of each level run (may be NULL)
 *   dD_levels   [max_outer] HOST out: dD/dell after each level (may be NULL) */
rkhsba_status rkhsba_solve_ell_decay(rkhsba_ctx* ctx, const rkhsba_ell_schedule* sched, double* poses,
                                     double* ell_levels, double* dD_levels, rkhsba_ell_info* info);

/* ------------------------------------------------------------------------
 * Pair-kernel tuning and the autotuner (the paper has no counterpart; these
 * pick launch shapes of the sparse double sum of Sec. III-B per workload).
 *
 * Three knobs change the speed of the pair stage but not its results beyond
 * FP32 rounding (pair sets and the exact fixed-point sums do not change):
 *   cell_scale    grid cell edge in units of r_c (params.cell_scale, fixed
 *                 at rkhsba_create: the grids are built for it)
 *   unit_queries  queries of one home cell handed to a warp at a time (1..32;
 *                 1..64 for BF16 labels without colour, pruning or top_k,
 *                 whose dense pair kernel takes units of up to 64 queries)
 *   ctas_per_sm   resident CTAs per SM of the persistent pair launch
 *                 (0: as many as fit)
 * ------------------------------------------------------------------------ */
typedef struct {
    double cell_scale;
    int32_t unit_queries;
    int32_t ctas_per_sm;
    double ms;             /* autotuner: mean time of one evaluation with these settings */
} rkhsba_tuning;

/* Set the runtime knobs of a context (captured LM graphs are rebuilt). */
rkhsba_status rkhsba_set_tuning(rkhsba_ctx* ctx, int32_t unit_queries, int32_t ctas_per_sm);
rkhsba_status rkhsba_get_tuning(const rkhsba_ctx* ctx, rkhsba_tuning* out);

/*
 * rkhsba_autotune -- time the evaluation of one problem under every
 * candidate setting (cell_scale 1, 1.25, 1.5 x unit_queries 32, 16 and,
 * where the pair kernel takes it, 64 x ctas_per_sm all, 1; the default
 * setting first) and report the fastest.
 * For each cell size a temporary context is built from the inputs
 * (arguments as for rkhsba_create, or as for rkhsba_create_device when
 * inputs_on_device is 1); each setting is run once untimed, then at least
 * `reps` (1..100) evaluations at `poses` ([K*16] HOST), and at least 20 ms of
 * them, are timed with CUDA events on cuda_stream.  The default setting is
 * kept unless another is faster by more than 3%.
 *   best      HOST out: the chosen setting and its mean time (ms)
 *   table     HOST out [table_cap] (may be NULL when table_cap is 0): every
 *             setting tried, in order; *n_table receives the count (12, or
 *             18 with 64-query units)
 * Creating a context with params.cell_scale = best.cell_scale and calling
 * rkhsba_set_tuning(ctx, best.unit_queries, best.ctas_per_sm) applies it.
 * Synchronous; holds one temporary context at a time.
 */
rkhsba_status rkhsba_autotune(int32_t n_frames, const int64_t* n_points, const double* xyz, const float* sem,
                              const float* rgb, int32_t n_edges, const int32_t* edges,
                              const rkhsba_params* params, int32_t inputs_on_device, const double* poses,
                              void* cuda_stream, int32_t reps, rkhsba_tuning* best, rkhsba_tuning* table,
                              int32_t table_cap, int32_t* n_table);

/* ------------------------------------------------------------------------
 * Request server: continuous batching of BA solves on one GPU.
 *
 * Requests (each a problem as for rkhsba_create plus initial poses) are
 * queued by rkhsba_submit and admitted while an in-flight slot is free and
 * the device-memory budget allows (the problem's buffers are estimated from
 * its sizes before admission and charged at their real size after).  Every
 * admitted problem keeps its points and grids resident and runs the
 * rkhsba_solve loop (Sec. V-A, V-C).  In batched mode (the default) the
 * server advances all admitted problems together, one LM iteration per
 * round: each problem's damped solve and query binning on its own stream,
 * then one persistent pair launch over the units of every problem (each
 * adding into its own accumulators), then each problem's assembly and
 * accept/reject on its own stream; in per-request mode every problem runs
 * whole iterations on its own stream, a few per issue.  Either way the GPU
 * work of different requests overlaps; a finished request frees its slot and
 * memory and the next one is admitted at once.
 * Results do not depend on what else is running: a request solved alone and
 * in a mix, in either mode, gives the same poses bit for bit.
 *
 * Threads: rkhsba_submit / rkhsba_poll / rkhsba_cancel / rkhsba_server_stats
 * may be called from any host threads; the server's own threads make all
 * CUDA calls for its requests.  Failures of one request (invalid input,
 * allocation failure, watchdog timeout) end that request only.
 * ------------------------------------------------------------------------ */
typedef struct rkhsba_server rkhsba_server;

typedef struct {
    int32_t max_inflight;      /* concurrently admitted requests (default 8) */
    int32_t iters_per_issue;   /* LM iterations issued per round (default 4) */
    int64_t memory_budget;     /* bytes of device memory for admitted requests
                                  (0: half of the free memory at creation) */
    double request_timeout_ms; /* watchdog per request from admission (0: none) */
    int32_t mode;              /* 0 (default): batched rounds -- every round runs one LM
                                  iteration of every admitted request, with ONE
                                  persistent pair launch over the units of all of
                                  them that share a label layout; 1: per-request
                                  streams, iters_per_issue whole iterations per issue */
    int32_t autotune;          /* 1: the first request of each workload class (label
                                  layout; mean points per frame < 16k, < 64k, more) is
                                  timed under the autotuner's settings (rkhsba_autotune)
                                  and the chosen one is used for it and later ones of
                                  that class; 0: off */
} rkhsba_server_config;

typedef struct {
    int32_t state;             /* 0 queued, 1 running, 2 finished, 3 failed, 4 cancelled */
    int32_t status;            /* RKHSBA_OK / ENOTCONV when finished, error code otherwise */
    rkhsba_solve_info solve;   /* as for rkhsba_solve */
    double queue_ms;           /* submit -> admission */
    double latency_ms;         /* submit -> result ready */
    int64_t device_bytes;      /* device memory the request held */
} rkhsba_request_info;

rkhsba_status rkhsba_server_create(rkhsba_server** out, const rkhsba_server_config* cfg);

/* Stop the server: running and queued requests are cancelled; returns once
 * all GPU work of the server has finished and its memory is freed. */
void rkhsba_server_destroy(rkhsba_server* srv);

/* Queue one problem (arguments as for rkhsba_create, HOST memory, copied
 * before the call returns) with initial poses [K*16]; *ticket names it. */
rkhsba_status rkhsba_submit(rkhsba_server* srv, int32_t n_frames, const int64_t* n_points,
                            const double* xyz, const float* sem, const float* rgb,
                            int32_t n_edges, const int32_t* edges, const rkhsba_params* params,
                            const double* poses0, int64_t* ticket);

/* Wait up to timeout_ms (0: do not wait, < 0: wait forever) for a request.
 * Returns RKHSBA_OK once it has ended (finished, failed or cancelled; see
 * info->state / info->status) and writes poses [K*16] when finished; the
 * ticket is then released.  Returns RKHSBA_EBUSY while it is still queued or
 * running, RKHSBA_EINVAL for an unknown ticket. */
rkhsba_status rkhsba_poll(rkhsba_server* srv, int64_t ticket, int32_t timeout_ms, double* poses,
                          rkhsba_request_info* info);

/* Ask a queued or running request to stop; its poll then reports state 4. */
rkhsba_status rkhsba_cancel(rkhsba_server* srv, int64_t ticket);

/* Counters: requests queued, running, finished so far; device bytes held. */
rkhsba_status rkhsba_server_stats(rkhsba_server* srv, int64_t* queued, int64_t* running,
                                  int64_t* finished, int64_t* device_bytes);

/* Problem shape and device memory of a context. */
rkhsba_status rkhsba_info(const rkhsba_ctx* ctx, int32_t* n_frames, int32_t* n_edges,
                          int64_t* n_points_total, int64_t* device_bytes);

/* Message of the last failure on ctx (or of the calling thread when ctx is NULL). */
const char* rkhsba_last_error(const rkhsba_ctx* ctx);

/* Number of CUDA kernels this library has launched in the process. */
int64_t rkhsba_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* RKHSBA_H */
