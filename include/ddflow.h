/*
 * ddflow.h - C ABI of the GB300 library for domain decomposition of entropic
 * optimal transport with flow updates (Medina & Schmitzer, "Flow updates for
 * domain decomposition of entropic optimal transport").
 *
 * The problem (Eq. entropic-transport): two probability measures mu, nu on the
 * same N1 x N2 pixel grid with spacing h, squared-Euclidean cost
 * c(x, y) = |x - y|^2, regularisation eps:
 *     min_{pi in Pi(mu, nu)} <c, pi> + eps KL(pi | mu (x) nu).
 * X is split into basic cells of cell_size x cell_size pixels (Def. 2.2); the
 * composite partitions A and B group 2 x 2 basic cells, B shifted by one basic
 * cell and truncated at the image border (Fig. 3). The state is the set of
 * basic-cell Y-marginals nu_i (Eq. basic-cell-Y-marginal), each on its
 * bounding box (Section A.1, "Bounding box representation").
 *
 * Conventions shared by every entry point:
 *  - Return value: DD_OK (0) or a negative DD_ERR_* code; dd_strerror() names it.
 *  - Pointers are HOST pointers; the library copies inputs in and outputs out.
 *    With DD_FLAG_DEVICE_PTRS in dd_options.flags, the array arguments of
 *    dd_init (mu, nu), dd_set_plan (hdr, data), dd_get_plan (hdr, data) and
 *    dd_get_duals (alpha, hdr, beta) are instead CUDA device pointers on the
 *    context's device (copies ordered on the context's stream); every other
 *    entry point keeps host pointers unless its comment says otherwise.
 *    Outputs are caller-allocated. Where an entry point takes a `size_t* count`,
 *    passing NULL for the data pointer only stores the required element count.
 *  - Arrays are row-major. Pixel (p, q) has flat index p * N2 + q; basic cell
 *    (bi, bj) has index i = bi * (N2 / cell_size) + bj.
 *  - A box header is 4 int32: (o1, o2, h, w) = top-left pixel and extent; a box
 *    with h = w = 0 is empty. Box data follow each other in cell order, each box
 *    h x w row-major, without padding.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream);
 *    every device operation of a context is ordered on it.
 *  - One context belongs to one host thread at a time; calls on the same
 *    context are not re-entrant.
 */
#ifndef DDFLOW_H
#define DDFLOW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DD_OK 0
#define DD_ERR_ARG (-1)     /* invalid argument                                   */
#define DD_ERR_OOM (-2)     /* device or host allocation failed                   */
#define DD_ERR_CUDA (-3)    /* a CUDA call failed                                 */
#define DD_ERR_MAXITER (-4) /* a cell hit the Sinkhorn iteration cap (result is
                               still exactly Y-feasible, its X error above tol)   */
#define DD_ERR_STALL (-5)   /* reserved: FP32 stall detected                      */
#define DD_ERR_FLOW (-6)    /* min-cost flow failed; the stationary flow was kept */
#define DD_ERR_POOL (-7)    /* a bounding box exceeds what one cell kernel holds   */
#define DD_ERR_STATE (-8)   /* call order violated (e.g. flow update first)       */

#define DD_INIT_PRODUCT 0 /* initial plan mu (x) nu                              */
#define DD_INIT_USER 1    /* initial plan given by dd_set_plan                    */

#define DD_WARM_PREV 0 /* alpha_init = alpha of the previous solve on the same
                          partition (Alg. 4 input), zero on the first solve        */
#define DD_WARM_COLD 1 /* alpha_init = 0 for every solve                          */
#define DD_WARM_AFFINE 2 /* alpha_init = the cell's affine dual: the exact dual
                            when nu_J is mu_J translated and stretched per axis
                            (barycentres and variances of the two marginals);
                            not in the paper                                     */
#define DD_WARM_MLP 3  /* learned (dd_set_warmstart_weights; cells with a full
                          8 x 8 block, the others as DD_WARM_PREV): a solve
                          without a previous dual of its cell (the first of each
                          partition) starts from the affine dual + the network's
                          correction, later ones from the previous dual
                          (DD_FLAG_MLP_EVERY_SOLVE: from the previous dual + the
                          network's predicted change of the dual between the two
                          solves); not in the paper, requires cell_size 4       */

#define DD_FLAG_KEEP_PREBALANCE 1 /* keep the pre-balance basic marginals of the
                                     last half-iteration for dd_get_prebalance     */
#define DD_FLAG_COLLECT 2 /* compute the warm-start network's inputs before, and
                             its training targets after, every cell solve, for
                             dd_collect_cells (requires cell_size 4)              */
#define DD_FLAG_NO_GRAPH 4 /* dd_step runs its steps one by one instead of
                              replaying a captured CUDA graph                     */
#define DD_FLAG_TRACE 8 /* record per-cell solve timelines for dd_get_trace       */
#define DD_FLAG_MLP_EVERY_SOLVE 16 /* DD_WARM_MLP: evaluate the network before
                                      every solve (predicted change of the dual),
                                      not only before solves without a previous
                                      dual                                        */
#define DD_FLAG_DEVICE_PTRS 32 /* the arrays of dd_init, dd_set_plan, dd_get_plan
                                  and dd_get_duals are device pointers (see the
                                  conventions above)                              */
#define DD_FLAG_FUSED_C2B 64 /* CompositeToBasic, balancing and truncation
                                (Alg. 1, Def. 3.4) of a cell by the CTA that
                                solved it, right after the solve (one-CTA
                                solves whose arrays fit the solve's freed
                                shared memory; the others after all solves, as
                                by default, in a kernel of their own). The same
                                arithmetic, its partial sums over another CTA
                                size. Off by default: on the 256 x 256 bench
                                the persistent large-box grid then holds the
                                SMs longer and the small boxes finish later,
                                so a half-iteration took as long as without  */

typedef struct dd_grid {
    int32_t N1, N2; /* pixels per axis                                          */
    double h;       /* pixel spacing (cost uses h^2 (dp^2 + dq^2))               */
} dd_grid;

typedef struct dd_options {
    double tol;          /* cell stop: L1 X-marginal error <= tol * mu(X_J); 1e-5 */
    int32_t max_iter;    /* Sinkhorn iteration cap per cell solve; 100000         */
    int32_t fixed_iters; /* > 0: exactly this many iterations per cell, no tol    */
    double trunc;        /* entries below this are dropped after balancing; 1e-15 */
    int32_t init_kind;   /* DD_INIT_PRODUCT or DD_INIT_USER                        */
    int32_t warm;        /* DD_WARM_PREV or DD_WARM_COLD                           */
    int32_t threads;     /* threads per cell solve (64..512); 0 = autotuned        */
    int32_t flags;       /* DD_FLAG_*                                              */
    double plan_tol;     /* dd_set_plan feasibility tolerance (L1, both marginals); 1e-12 */
    double omega;        /* X-update over-relaxation a <- a + omega (X(b) - a): 1 = plain
                            Sinkhorn (default, the paper's solver), (1, 2) fixed, < 0
                            adaptive; same fixed point and the same stopping pair      */
    double graph_margin; /* dd_step graphs: buffer capacities = sizes seen x (1 + margin)
                            (plus slack when > 0); 0.5. 0 exercises the overflow path  */
    int32_t eps_levels;  /* eps-scaling inside every cell solve (tolerance mode): first
                            at eps f^L, ..., eps f, then at eps with the usual stop; the
                            solution is that of eps. 0 (default) = plain solve         */
    double eps_factor;   /* f > 1; 4                                                    */
    double eps_tol;      /* a coarse level ends at L1 X error <= eps_tol mu(X_J); 1e-3 */
    double tol_share;    /* s in [0, 1]: cell J stops at L1 X error
                              <= tol ((1 - s) mu(X_J) + s mu(X) / #cells),
                            budgets that sum to tol mu(X) over the partition, the
                            bound of the paper's batch stopping criterion (Section 5,
                            "Stopping criterion"); 0 (default) = tol mu(X_J) per cell */
    double tol_gamma;    /* >= 0: with previous iteration counts it_J, the budgets above
                            are weighted by (it_J / mean it)^tol_gamma and rescaled to
                            sum to tol mu(X) (the same batch bound), so that slowly
                            converging cells stop earlier and fast ones later; 0 = off */
    int32_t anderson;    /* 0 (default): plain Sinkhorn updates of the X dual. 1..4:
                            Anderson acceleration of the X-dual fixed-point iteration
                            (tolerance mode): the next X dual combines the last
                            anderson + 1 iterates and their plain updates by
                            mu-weighted least squares on the residuals, restarted
                            when the L1 X error more than doubles; same fixed point,
                            same stopping pair (alpha_old, beta); omega is ignored */
    double eps_gamma;    /* edge candidates of the flow update (Def. 3.7, Remark 3.8):
                            0 (default) = product gluing candidates (eps_gamma =
                            infinity); > 0 = gluing candidates from the entropic
                            optimal plans gamma_ij between mu_i / m_i and mu_j / m_j
                            at this regularisation (cost units, like eps), computed
                            once by dd_init in FP64 (L1 marginal error <= 1e-13);
                            cell_size <= 8                                         */
} dd_options;

/* Statistics of one half-iteration (Alg. 4). */
typedef struct dd_stats {
    int32_t part;          /* 0 = A, 1 = B                                        */
    int32_t ncell;         /* composite cells solved                              */
    int32_t iters_max;     /* largest Sinkhorn iteration count                    */
    int32_t n_maxiter;     /* cells that hit max_iter                             */
    int32_t n_stalled;     /* cells stopped at their FP32 floor above tol (their
                              error stays within 50 tol; result Y-feasible)       */
    double iters_mean;     /* mean Sinkhorn iterations per cell                   */
    double objective;      /* E = sum_J <alpha_J, r_J> + <beta_J, nu_J>, Prop. 2.1 */
    double l1_x;           /* sum_J sum_x |r_J(x) - mu(x)| of the Gibbs cell plans */
    double lse_terms;      /* log-sum-exp terms evaluated by the cell kernel      */
    double ms_total;       /* device time of the half-iteration (ms)              */
    double ms_cells;       /* device time of the fused cell kernel (ms)           */
    int64_t stored_entries;/* entries of the output basic boxes                   */
    double ms_c2b;         /* device time of CompositeToBasic + balancing +
                              truncation (part of ms_cells, ms)                   */
    double bytes_c2b;      /* its algorithmic bytes: read nu_J (4 B per composite
                              box entry), write the output basic boxes (4 B per
                              stored entry)                                       */
} dd_stats;

/* Statistics of one flow update (Section 3.2, steps of Section 5.1). */
typedef struct dd_flow_stats {
    double value;        /* optimal value sum w_ij c_bar_ij (<= 0)                */
    int32_t nonzero;     /* off-diagonal arcs with w_ij > 0                       */
    int32_t pivots;      /* network-simplex pivots                                */
    double moved;        /* sum_{i != j} w_ij                                     */
    double ms_costs;     /* device time, edge costs (ms)                          */
    double ms_solve;     /* host time, min-cost flow (ms)                         */
    double ms_exchange;  /* device time, exchange + re-box (ms)                   */
    double bytes_exchange; /* algorithmic bytes of the exchange: read every source
                              box with w_ij > 0, write the new boxes (4 B each)  */
    double ms_host_step;   /* device time from the edge costs to the flow back on
                              the device: the copies, the host solve and the
                              handover to and from the host (ms)               */
} dd_flow_stats;

typedef struct dd_ctx dd_ctx;

/* Fill `opt` with the defaults listed in dd_options. */
void dd_default_options(dd_options* opt);

/* Human-readable name of a status code (static string). */
const char* dd_strerror(int status);

/* The CUDA call and error message behind the last DD_ERR_CUDA (static string,
 * shared by all contexts; empty if none). */
const char* dd_last_error(void);

/*
 * Create a context. mu, nu: N1*N2 float64, >= 0, each summing to 1 within
 * 1e-12. eps > 0. cell_size must divide N1 and N2, give an even number of basic
 * cells per axis, and every basic cell needs mu(X_i) > 0 (Def. 2.2). The
 * initial plan is mu (x) nu (DD_INIT_PRODUCT) or the one passed next to
 * dd_set_plan (DD_INIT_USER). opt may be NULL (defaults). On success *out owns
 * device memory until dd_destroy. Errors: DD_ERR_ARG, DD_ERR_OOM, DD_ERR_CUDA.
 */
int dd_init(const double* mu, const double* nu, const dd_grid* grid, double eps, int cell_size,
            const dd_options* opt, void* stream, dd_ctx** out);

/*
 * Replace the state by a user plan given as basic-cell Y-marginals: hdr is
 * nbasic x 4 int32 box headers, data the packed float64 box contents, n their
 * total count. The plan must be feasible: |nu_i| = mu(X_i) and sum_i nu_i = nu,
 * each within opt.plan_tol (L1); otherwise DD_ERR_ARG. The warm-start duals are
 * kept (they only initialise the next solves).
 */
int dd_set_plan(dd_ctx* ctx, const int32_t* hdr, const double* data, size_t n);

/*
 * Change the entropic regularisation eps of the next half-iterations (eps > 0),
 * for an eps schedule across hybrid iterations (the eps-scaling of the paper's
 * solvers, Section 5, "Multi-scale and eps-scaling"). The plan is kept. The
 * stored X duals of both partitions are rescaled so that the dual potentials
 * alpha (cost units) stay the same: in every cell's gauge a - log2 mu scales as
 * 1/eps, a <- log2 mu + (eps_old / eps) (a - log2 mu); they warm-start the next
 * solves. The learned start's stored predictions are dropped (the next solve of
 * each partition starts from the network's prediction). Captured graphs are
 * re-captured. Errors: DD_ERR_ARG (eps <= 0 or not finite), DD_ERR_CUDA.
 */
int dd_set_eps(dd_ctx* ctx, double eps);

/*
 * One domain-decomposition half-iteration (Alg. 1 in the form of Alg. 4):
 * BasicToComposite, the batched log-domain cell Sinkhorn solves, CompositeToBasic
 * with <c, pi_i>, balancing, truncation. part = 0 (A), 1 (B) or -1 (the other
 * partition than the last one; A first). st may be NULL. Returns DD_ERR_MAXITER
 * if a cell hit max_iter (the state is still updated).
 */
int dd_iterate(dd_ctx* ctx, int part, dd_stats* st);

/*
 * One flow update (Def. 3.4 with product gluing candidates, Remark 3.8): edge
 * costs Eq. (edge-cost), min-cost flow Eq. (MinCostFlow) solved on the host,
 * exchange Eq. (flow-update-cell-marginals). Valid only directly after
 * dd_iterate (DD_ERR_STATE otherwise). st may be NULL.
 */
int dd_flow_update(dd_ctx* ctx, dd_flow_stats* st);

/*
 * n hybrid iterations of Alg. 3 (A half-iteration, B half-iteration, flow
 * update). After one iteration run step by step (which fixes buffer sizes and
 * the flow solver), every iteration is replayed from a captured CUDA graph:
 * cell classification and ordering run on the device, the min-cost flow is a
 * host node of the graph. Buffers get capacity margins; if a box or pool would
 * exceed them, the graph's remaining kernels do nothing and the iteration is
 * finished step by step (same results), after which the graph is captured
 * again. DD_FLAG_NO_GRAPH disables the graph. Any of the stats pointers may be
 * NULL; when given they receive the values of the LAST iteration (in graph
 * mode stored_entries is that of the state after the flow update). All n
 * iterations run; the status is DD_ERR_FLOW if a flow solve failed (the
 * stationary flow was kept), else DD_ERR_MAXITER if some cell reached max_iter
 * (the state is still updated), else DD_OK; other errors stop at once.
 */
int dd_step(dd_ctx* ctx, int n, dd_stats* sa, dd_stats* sb, dd_flow_stats* sf);

/* Statistics of the last dd_step iteration (HOST structures, any may be NULL).
 * A replayed iteration called with all three dd_step statistics pointers NULL
 * reads nothing back from the device; this call reads them afterwards (the
 * per-cell counts, errors and event times stay valid until the next
 * half-iteration, flow update or plan change), so a caller can time iterations
 * without the read-back and still inspect each one. DD_ERR_STATE if no
 * dd_step iteration has run since the last such change. */
int dd_step_stats(dd_ctx* ctx, dd_stats* sa, dd_stats* sb, dd_flow_stats* sf);

/* Basic-cell boxes of the current state: hdr (nbasic x 4), data (float64). */
int dd_get_plan(dd_ctx* ctx, int32_t* hdr, double* data, size_t* count);

/*
 * Duals of the last solve on `part`: alpha on X (N1*N2 float64; every pixel
 * belongs to exactly one composite cell) and beta per composite cell on its
 * box (hdr ncell x 4, beta packed float64), both in the mu (x) nu convention of
 * Prop. 2.1: pi_J = exp((alpha + beta - c) / eps) mu (x) nu. beta is -inf where
 * nu_J = 0. Duals are defined up to (alpha + C_J, beta - C_J) per cell.
 */
int dd_get_duals(dd_ctx* ctx, int part, double* alpha, int32_t* hdr, double* beta, size_t* count);

/* Composite Y-marginals nu_J (Eq. get-composite-cell-marginal) of the last solve on `part`. */
int dd_get_composite(dd_ctx* ctx, int part, int32_t* hdr, double* data, size_t* count);

/* Per-cell Sinkhorn iterations and L1 X errors of the last solve on `part` (ncell each). */
int dd_get_cell_stats(dd_ctx* ctx, int part, int32_t* iters, double* err);

/*
 * Objective E and L1 X error of the last half-iteration (Prop. 2.1 / Section A.2),
 * and the L1 Y error sum_y |sum_i nu_i(y) - nu(y)| of the current state. Any
 * pointer may be NULL.
 */
int dd_get_objective(dd_ctx* ctx, double* E, double* l1_x, double* l1_y);

/* Composite cells of `part`: members (ncell x 4 int32, -1 padded), *ncell. */
int dd_get_partition(dd_ctx* ctx, int part, int32_t* members, int32_t* ncell);

/* Neighbourhood set (Def. 3.1): nbasic x 5 int32 (self, -axis1, +axis1, -axis2, +axis2), -1 if none. */
int dd_get_neighbours(dd_ctx* ctx, int32_t* nbr);

/* Basic-cell quantities of the last half-iteration: D_i = <c, pi_i> (before
 * balancing), mass |nu_i|, barycentre ybar_i (2) and variance V_i of nu_i / |nu_i|
 * (after balancing); each nbasic float64 (ybar: nbasic x 2). NULL skips. */
int dd_get_basic_moments(dd_ctx* ctx, double* D, double* mass, double* ybar, double* var);

/* Edge costs c_bar (nbasic x 5) and flows w (nbasic x 5) of the last flow update. */
int dd_get_flow(dd_ctx* ctx, double* cbar, double* w);

/* With DD_FLAG_KEEP_PREBALANCE: the basic marginals of the last half-iteration
 * right after CompositeToBasic (before balancing/truncation), each on its
 * composite cell's box: hdr nbasic x 4, data packed float64. */
int dd_get_prebalance(dd_ctx* ctx, int32_t* hdr, double* data, size_t* count);

/*
 * Host min-cost flow of Eq. (MinCostFlow) on the neighbourhood graph, exposed
 * for testing; no GPU involved. n basic cells, nbr (n x 5, -1 = no arc), cbar
 * (n x 5 costs), m (n masses > 0). Writes the flow w (n x 5) with
 * sum_k w[i,k] = m_i and inflow m_j, and *value = sum w c_bar; *pivots may be
 * NULL. Exact network simplex on masses scaled to integers (2^60 in total) and
 * costs scaled to integers (2^40 at the largest |c_bar|).
 */
int dd_min_cost_flow(int32_t n, const int32_t* nbr, const double* cbar, const double* m, double* w,
                     double* value, int32_t* pivots);

/* Diagnostics: the raw FP32 values the cell kernel kept for composite cell J of
 * `part`: its X dual a (hx * wx, base 2, the kernel's gauge), its Y dual b~ on the
 * composite box (h * w), the 8 gauge parameters (d1, d2, l1, l2, uc1, uc2, vc1,
 * vc2) and the X block / box (r0, c0, hx, wx, o1, o2, h, w). Buffers hold at
 * least (2 cell_size)^2, h * w, 8 and 8 entries; pass NULL for b to get h, w. */
int dd_debug_cell(dd_ctx* ctx, int part, int J, float* a, float* b, float* gauge, int32_t* geom);

/* Counters since dd_init: kernels launched by the library, bytes copied host to
 * device and device to host. Any pointer may be NULL. */
int dd_get_counters(dd_ctx* ctx, int64_t* launches, int64_t* h2d_bytes, int64_t* d2h_bytes);

/*
 * Launch configuration of the cell kernels (the persistent Sinkhorn kernel runs
 * one CTA per composite cell at a time, in three size classes):
 *   class 1: padded box area <= small_area and box height, width <= small_side
 *            (shared memory, many CTAs per SM),
 *   class 0: other boxes that fit shared memory,
 *   class 2: boxes beyond shared memory (their arrays in global scratch).
 * threads[k] is the CTA size of class k (64, 128, 256 or 512).
 */
typedef struct dd_tuning {
    int32_t threads[3];
    int32_t small_area;
    int32_t small_side;
    double ms_default; /* dd_autotune: time of the trial run with the defaults   */
    double ms_best;    /* and with the chosen configuration (ms)                 */
    int32_t trials;    /* configurations timed (0: taken from the cache file)    */
    int32_t cl_size;   /* 2 or 4: the largest-work cells of the large class are
                          solved by thread-block clusters of this many CTAs (of
                          threads[0] threads, 256 or 512), one cluster per cell;
                          1 = off                                                 */
    int32_t cl_cells;  /* at most this many cells per half-iteration on clusters
                          (and at most #SMs / cl_size): whole quarter-octave
                          buckets of the work key h w (previous iterations), from
                          the top, boxes of at least 1024 entries                */
    int32_t sm_reserve; /* the persistent grid of the large-box class has at most
                           (#SMs - sm_reserve) x (CTAs per SM) CTAs, so that the
                           small-box class starts on the reserved SMs at once (a
                           512-thread large-box CTA holds a whole SM's registers);
                           0 = off, < #SMs                                        */
} dd_tuning;

/* Defaults: threads {256, 128, 256}, small_area 1536, small_side 64, clusters
   off, sm_reserve 0. */
int dd_get_tuning(dd_ctx* ctx, dd_tuning* t);
int dd_set_tuning(dd_ctx* ctx, const dd_tuning* t);

/*
 * Autotuner: times every candidate configuration (threads of the small class
 * 64 / 128 / 256 and of the large class 256 / 512, the small-class limit, then
 * clusters of 2 or 4 CTAs for 4, 8, 16, 32 or 48 cells on the two fastest, and
 * 8, 16 or 32 SMs reserved for the small-box class on the fastest) on the
 * context's current state, both partitions, every cell solved to the
 * context's tolerance from the current warm start (restored before each trial
 * and after the last, so every configuration does the same solves and the
 * state and next solve are unchanged), best of two runs each; the three
 * fastest are timed again (best of four fresh runs) and the fastest of those is
 * kept (ms_best is that fresh time). With cache_path not NULL the
 * result is looked up in / appended to that text file, keyed by GPU name, SM
 * count, grid, cell size, eps / h^2 and the median / largest box area of the
 * state. The chosen configuration is in *out (may be NULL).
 */
int dd_autotune(dd_ctx* ctx, const char* cache_path, dd_tuning* out);

/* With DD_FLAG_TRACE: the timeline of the last solve of every cell of `part`,
 * ncell x 8 int64 (HOST): start and end of the solve (ns, the GPU's global
 * timer), the SM it ran on, its CTA size (x cluster size), the end of the
 * gather of nu_J, the start and the end of the Sinkhorn iterations, and the end
 * of the cell's CompositeToBasic when its solving CTA did it (else 0). */
int dd_get_trace(dd_ctx* ctx, int part, int64_t* trace);

/*
 * Measured throughput of the base-2 exponential (ex2.approx, the MUFU unit) on
 * the current device, in ex2 per second (best of five timed launches of a
 * persistent grid of independent ex2 chains, 4 CTAs of 512 threads per SM).
 * Every log-sum-exp term of the cell Sinkhorn kernel is one ex2, so this rate
 * calibrates the kernel's roofline (Section A.1 "Custom CUDA Sinkhorn" is the
 * step it bounds). Allocates a small device buffer; synchronises `stream`.
 * *ms (may be NULL) receives the best launch time. Errors: DD_ERR_ARG,
 * DD_ERR_OOM, DD_ERR_CUDA.
 */
int dd_probe_ex2_rate(void* stream, double* ex2_per_s, double* ms);

/* dd_step graph counters since dd_init: graphs captured, iterations replayed
 * from a graph, replays finished step by step after a capacity overflow. */
int dd_get_graph_counters(dd_ctx* ctx, int64_t* captures, int64_t* replays, int64_t* fallbacks);

/*
 * Allocation-free variant of the L1 Y-marginal error of dd_get_objective (the
 * paper has no counterpart; this is a library facility). For callers that
 * cannot allocate device memory: real-time pipelines that reserve all device
 * memory up front and forbid allocation afterwards, and host frameworks whose
 * own caching allocator owns the GPU's memory. It computes
 *     *l1_out = sum_y | sum_i nu_i(y) - nu(y) |
 * with scratch memory taken from a fixed __device__ array inside the library,
 * never from cudaMalloc.
 *  - All pointers are DEVICE pointers on the current device: hdr (nbasic x 4
 *    int32 box headers o1, o2, h, w), data (float32 box contents packed in cell
 *    order, each h x w row-major, no padding), nu (N1 * N2 float64), l1_out (one
 *    float64, overwritten). Entries of a box outside the grid are ignored; a
 *    box with h <= 0 or w <= 0 is empty. data must hold sum_i h_i w_i entries.
 *  - Limits: N1 * N2 <= DD_STATIC_MAX_PIXELS and nbasic <= DD_STATIC_MAX_CELLS;
 *    larger problems return DD_ERR_ARG without touching the GPU. The array
 *    (about 8.5 MB) is held by every GPU that loads the library until exit.
 *  - The first call on a device looks up the array's device address
 *    (cudaGetSymbolAddress) with that device current; make that first call
 *    before any stream capture. Host threads may make it concurrently.
 *  - Every call shares the array: calls that overlap on the GPU (other streams,
 *    other host threads on the same device) race. Calls ordered on one stream are
 *    safe; each call clears the accumulator it uses.
 *  - Work is enqueued on `stream` (cudaStream_t as void*); the call returns
 *    before it completes.
 */
#define DD_STATIC_MAX_PIXELS (1024 * 1024)
#define DD_STATIC_MAX_CELLS 65536
int dd_l1_y_error_static(int32_t N1, int32_t N2, int32_t nbasic, const int32_t* hdr, const float* data,
                         const double* nu, double* l1_out, void* stream);

/* ------------------------------------------------------------------------
 * Learned warm start (not in the paper). A multilayer perceptron maps features
 * of a composite-cell problem to a correction r of the cell's affine dual; the
 * solver starts from alpha_init = affine dual + r (DD_WARM_MLP). The
 * converged Sinkhorn error judges it: a poor prediction costs iterations, never
 * accuracy (every solve still runs to tol).
 *
 * Network: DD_MLP_NIN -> DD_MLP_NHID -> DD_MLP_NHID -> DD_MLP_NHID ->
 * DD_MLP_NOUT, SiLU on the hidden layers, linear output; BF16 weights and
 * activations, FP32 accumulation (tensor cores). Parameters are one flat float
 * vector of DD_MLP_NPARAMS: W_1 (NHID x NIN, row-major, row n = the weights into
 * output n), b_1, W_2, b_2, W_3, b_3, W_4 (NOUT x NHID), b_4.
 *
 * Inputs (per cell, BF16): mu on the 8 x 8 block / its mean - 1 (64), nu_J
 * resampled to 16 x 16 by exact area overlap / its mean - 1 (256), and 16
 * scalars of the cell's change of gauge. Outputs: r on the block (64, base-2
 * units, mu-weighted mean zero) and an auxiliary Y-side log dual on 16 x 16
 * sample pixels of the box (256, trained, not used by the solver).
 * ---------------------------------------------------------------------- */
#define DD_MLP_NIN 336
#define DD_MLP_NHID 256
#define DD_MLP_NOUT 320
#define DD_MLP_NPARAMS 300096

typedef struct dd_mlp dd_mlp;

/* A network (parameters zero) with buffers for batches of up to max_batch
 * rows; its work is ordered on `stream`. Errors: DD_ERR_ARG, DD_ERR_OOM. */
int dd_mlp_create(int32_t max_batch, void* stream, dd_mlp** out);

/* Parameters from / to HOST memory (n = DD_MLP_NPARAMS floats). Setting them
 * resets the optimiser state. Both synchronise the network's stream. */
int dd_mlp_set_params(dd_mlp* m, const float* params, int64_t n);
int dd_mlp_get_params(dd_mlp* m, float* params, int64_t n);

/* Forward pass of M <= max_batch rows: x_dev (M x NIN BF16, DEVICE) -> y_dev
 * (M x NOUT float, DEVICE). Asynchronous. With the default DD_MLP_GEMM_UMMA the
 * layer products run on the fifth-generation tensor cores (TMA loads,
 * tcgen05.mma into tensor memory), which needs x_dev and y_dev 16-byte aligned
 * (DD_ERR_ARG otherwise); a timed-out wait inside them is reported as
 * DD_ERR_CUDA by the next call that synchronises (dd_mlp_get_params,
 * dd_mlp_loss_grad, dd_mlp_train_step with a loss). */
int dd_mlp_forward(dd_mlp* m, const uint16_t* x_dev, int32_t M, float* y_dev);

/* Kernel of the forward layer products: DD_MLP_GEMM_UMMA (default; tcgen05.mma
 * with TMEM accumulators, operands staged by TMA) or DD_MLP_GEMM_MMA (warp-level
 * mma.sync, the kernel the backward pass uses; kept as the reference the first
 * is tested against). Same arithmetic up to the FP32 summation order.
 * Errors: DD_ERR_ARG (unknown kind). */
#define DD_MLP_GEMM_UMMA 0
#define DD_MLP_GEMM_MMA 1
int dd_mlp_set_gemm(dd_mlp* m, int32_t kind);

/* Loss L = (1/M) sum_rows sum_j w_j (y_j - t_j)^2 of M rows and its gradient:
 * x_dev (M x NIN BF16), t_dev (M x NOUT float), w_dev (NOUT float), all DEVICE;
 * *loss (may be NULL) and grad_host (DD_MLP_NPARAMS floats, HOST, may be NULL).
 * Synchronises. */
int dd_mlp_loss_grad(dd_mlp* m, const uint16_t* x_dev, const float* t_dev, const float* w_dev, int32_t M,
                     double* loss, float* grad_host);

/* One Adam step (beta 0.9, 0.999, eps 1e-8, learning rate lr) on the batch of
 * rows idx_dev[0..B) (DEVICE int32) of the data set x_all (rows x NIN BF16) /
 * t_all (rows x NOUT float), loss weights w_dev; all DEVICE. If loss is not NULL
 * it receives the batch loss before the step (and the call synchronises);
 * otherwise the step is only enqueued. */
int dd_mlp_train_step(dd_mlp* m, const uint16_t* x_all, const float* t_all, const int32_t* idx_dev, int32_t B,
                      const float* w_dev, float lr, double* loss);

void dd_mlp_destroy(dd_mlp* m);

/* Give the context the warm-start network's parameters (HOST, DD_MLP_NPARAMS
 * floats; weights are used in BF16, biases in FP32). Needed before dd_iterate
 * with DD_WARM_MLP (DD_ERR_STATE otherwise). Requires cell_size 4. */
int dd_set_warmstart_weights(dd_ctx* ctx, const float* params, int64_t n);

/* With DD_FLAG_COLLECT: the network inputs (rows x NIN BF16) and targets (rows x
 * NOUT float) of the last half-iteration on `part`, one row per composite cell
 * with a full 8 x 8 block, in cell order, into DEVICE buffers of max_rows rows.
 * *rows receives the row count; with feat_dev NULL only the count is stored.
 * DD_ERR_STATE if the last half-iteration was not on `part`. */
int dd_collect_cells(dd_ctx* ctx, int part, uint16_t* feat_dev, float* targ_dev, int32_t max_rows, int32_t* rows);

/* Release every resource of the context (NULL is ignored). */
void dd_destroy(dd_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* DDFLOW_H */
