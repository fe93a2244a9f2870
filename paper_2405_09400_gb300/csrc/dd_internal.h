// Internal declarations of the ddflow library: the context, device buffers and
// kernel launchers. Not part of the C ABI (see include/ddflow.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/ddflow.h"

#define DD_NEG (-1.0e30f)  // log2 of zero mass

// Cells solved by thread-block clusters: box area at least this, and the work key
// (h w max(1, previous iterations)) in the top quarter-octave buckets.
constexpr long long kClusterMinArea = 1024;
// octave (bk) and quarter-octave (fb) bucket of a work key; fb / 4 == bk
__host__ __device__ inline void cluster_key_bucket(long long key, int& bk, int& fb) {
    int L = 0;
    while (L < 62 && (key >> (L + 1)) > 0) ++L;  // floor(log2 key), 0 for key < 2
    const int frac = L >= 2 ? (int)((key >> (L - 2)) & 3) : 0;
    bk = L < 47 ? L : 47;
    const int f = 4 * L + frac;
    fb = f < 191 ? f : 191;
}

// Box header layout in device memory (int32 x 8 per box).
enum { BH_O1 = 0, BH_O2, BH_H, BH_W, BH_STRIDE, BH_START, BH_STRIDE_HI, BH_START_HI, BH_N };
// Composite header (int32 x 8 per cell): box + pool offsets.
enum { CH_O1 = 0, CH_O2, CH_H, CH_W, CH_STRIDE, CH_COMP_LO, CH_COMP_HI, CH_OUT_SLOT, CH_N };
// Composite X block (int32 x 8 per cell).
enum { XB_R0 = 0, XB_C0, XB_HX, XB_WX, XB_NMEM, XB_PAD0, XB_PAD1, XB_PAD2, XB_N };

// Per-basic-cell moments written by the half-iteration (double x 8 per cell).
enum { BM_D = 0, BM_MASS, BM_Y1, BM_Y2, BM_VAR, BM_PREMASS, BM_PAD0, BM_PAD1, BM_N };

// Totals computed by the planning kernels (long long x 8).
enum { PT_COMP = 0, PT_OUT, PT_MAXAREA, PT_MAXH, PT_MAXW, PT_ENTRIES, PT_PAD0, PT_PAD1, PT_N };

struct McfSolver;
int mcf_create(int32_t n, const int32_t* nbr, const double* m, McfSolver** out);
int mcf_solve(McfSolver* S, const double* cbar, double* w, double* value, int32_t* pivots);
void mcf_destroy(McfSolver* S);

struct DevPart {
    int ncell = 0;
    int32_t* members = nullptr;  // ncell x 4, -1 padded
    int32_t* xblk = nullptr;     // ncell x XB_N
    double* mJ = nullptr;        // ncell, mu(X_J)
    double mbar = 0.0;           // mean of mu(X_J) over the partition
    double* budget = nullptr;    // ncell: stop budget of each cell's next solve (absolute L1 X error)
    int32_t* chdr = nullptr;     // ncell x CH_N (last solve)
    float* alpha = nullptr;      // ncell x amax, centred base-2 gauge
    float* gauge = nullptr;      // ncell x 2, displacement (cell centre - box centre) in pixels
    int32_t* iters = nullptr;    // ncell
    double* err = nullptr;       // ncell
    double* Ecell = nullptr;     // ncell
    int32_t* order = nullptr;    // ncell, processing order
    int32_t* c2b_order = nullptr;  // ncell, k_c2b order of the step-by-step path (largest work first)
    float* comp_b = nullptr;     // composite pool: b' (centred base-2 dual, absorbs log2 nu_J)
    float* comp_nu = nullptr;    // composite pool: nu_J
    size_t comp_cap = 0;
    bool warm_valid = false;
    bool solved = false;
    bool pred_old_valid = false;  // d_pred_old holds the network outputs of this partition's last solve
    std::vector<int32_t> h_members;  // host copy
    std::vector<int32_t> h_xblk;     // host copy
};

constexpr int kStatusMlp = 24, kStatusInts = 25;  // d_status: flag index, length

struct dd_ctx {
    int N1 = 0, N2 = 0, s = 0, n1 = 0, n2 = 0, nb = 0, amax = 0;
    double h = 0, eps = 0;
    float k2 = 0;    // h^2 / eps * log2(e): cost exponent per squared pixel, base 2 (FP32 copy)
    double k2d = 0;  // the same in FP64 (kernel tables, gauge conversions)
    dd_options opt{};
    cudaStream_t stream = nullptr;
    int dev = 0, nsm = 0;

    std::vector<double> h_mu, h_nu, h_m;
    double* d_mu = nullptr;
    double* d_nu = nullptr;
    float* d_lgmu = nullptr;   // log2 mu (DD_NEG where 0)
    double* d_lnmu = nullptr;  // ln mu, ln nu (FP64; -inf where 0)
    double* d_lnnu = nullptr;
    float* d_lnnuf = nullptr;  // ln nu in FP32 (DD_NEG where 0)
    double* d_m = nullptr;     // basic masses
    double* d_xmom = nullptr;  // per basic cell: x1bar, x2bar, var (pixels)
    int32_t* d_nbr = nullptr;  // nb x 5
    int32_t* d_rev = nullptr;  // nb x 5: position of j in the list of nbr[j][k]
    std::vector<int32_t> h_nbr;

    DevPart part[2];
    int last_part = -1;
    dd_tuning tune{};  // launch configuration of the cell kernels
    bool flow_ready = false;

    // basic state, double buffered
    float* pool[2] = {nullptr, nullptr};
    size_t pool_cap[2] = {0, 0};
    int32_t* bhdr[2] = {nullptr, nullptr};
    int cur = 0;

    double* d_bmom = nullptr;  // nb x BM_N
    long long* d_tot = nullptr;  // PT_N
    long long* h_tot = nullptr;  // pinned
    int* d_queue = nullptr;
    int* d_status = nullptr;   // 3 slices of 8 (eager, graph A, graph B): [0] maxiter, [1] empty cell,
                               // [2] shared memory too small, [3] stalled; then [kStatusMlp]: a
                               // wait of the network's tensor-core GEMM timed out

    // prebalance copy
    float* d_pre = nullptr;
    size_t pre_cap = 0;
    // global scratch for cells whose boxes exceed shared memory
    float* d_gscr = nullptr;
    size_t gscr_cap = 0;
    long long* d_goff = nullptr;
    int32_t* d_prehdr = nullptr;

    // flow
    double* d_cbar = nullptr;
    double* d_w = nullptr;
    double* h_cbar = nullptr;  // pinned
    double* h_w = nullptr;     // pinned
    int32_t* d_xhdr = nullptr; // exchange output headers (nb x CH_N)
    dd_flow_stats last_flow{};
    McfSolver* mcf = nullptr;  // persistent basis across flow updates

    // gluing edge candidates (opt.eps_gamma > 0): per directed edge (i, k = 1..4) and
    // pixel x' of X_i the moments A, B (3) of gamma_ij's disintegration at x';
    // per basic cell and pixel the mass and mean displacement (3) of the cell plan
    double* d_gAB = nullptr;   // nb x 4 x s^2 x 3
    double* d_pmom = nullptr;  // nb x s^2 x 3

    // l1_y scratch
    double* d_yacc = nullptr;
    double* d_red = nullptr;
    // plan transfer (dd_set_plan / dd_get_plan): packed FP64 boxes, their offsets,
    // per-cell masses of a plan being checked
    double* d_plan64 = nullptr;
    size_t plan64_cap = 0;
    long long* d_soff = nullptr;
    double* d_cellmass = nullptr;

    cudaEvent_t ev[8] = {};  // eager timing: half-iteration 0-2 (ev[7]: CompositeToBasic), flow 3-6
    cudaStream_t side = nullptr;  // second stream: the large-box class of cells
    cudaStream_t side2 = nullptr;  // third stream: the cells solved by clusters
    cudaStream_t side3 = nullptr;  // step by step: the small-box class (normal priority)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join2 = nullptr, ev_join3 = nullptr;
    long long n_launch = 0, n_h2d = 0, n_d2h = 0;
    double last_E = 0, last_l1x = 0;
    // statistics of the last dd_step iteration: filled at once, or (a graph replay
    // called without statistics) read back later by dd_step_stats / dd_get_objective
    dd_stats last_sa{}, last_sb{};
    dd_flow_stats last_sf{};
    bool last_stats_valid = false;
    bool stats_pending = false;

    // CUDA-graph execution of dd_step: one graph per parity of `cur` at the start
    // of a hybrid iteration (the state buffers alternate), recaptured whenever a
    // buffer it captured was reallocated (gen changes).
    struct GraphExec {
        cudaGraphExec_t exec = nullptr;
        long long gen = -1;
        long long launches = 0;
    } graph[2];
    long long gen = 0;
    long long n_capture = 0, n_replay = 0, n_fallback = 0;
    bool capturing = false;          // launches go to the capture stream, kernels gated by d_guard
    int status_slot = 0;             // d_status slice of the running stage (0 eager, 1 A, 2 B)
    cudaStream_t gstream = nullptr;  // capture stream (the legacy stream cannot be captured)
    int* d_guard = nullptr;          // [0]: 0, or the stage (1 A, 2 B, 3 flow) that would overflow a buffer
    int* d_fused = nullptr;          // per cell: CompositeToBasic done by its solving CTA (cleared by k_c2b)
    bool fuse_c2b = false;           // the cell launches being issued are followed by k_c2b
    int* h_guard = nullptr;          // pinned copy (read by the flow host node and after a replay)
    int32_t* d_corder[2] = {nullptr, nullptr};  // per partition: class-grouped order, 3 x ncell
    int* d_ccount[2] = {nullptr, nullptr};      // per partition: cells per class
    // capacities a graph is captured with, and the sizes eager steps have seen
    struct Caps {
        long long pool = 0, comp[2] = {0, 0}, gscr = 0;
        long long a0 = 0, h0 = 0, w0 = 0;  // class 0 (shared-memory boxes, 256 threads)
        long long h2 = 0, w2 = 0;          // class 2 (global-scratch boxes) and k_c2b
        int grid[3] = {0, 0, 0};
        size_t smem[3] = {0, 0, 0};
        size_t smem_c2b = 0;
        int cl_cap = 0;  // cluster class: most cells (0: off)
    } gcap;
    struct Seen {
        long long out = 0, comp[2] = {0, 0}, gscr = 0, a0 = 0, h0 = 0, w0 = 0, hmax = 0, wmax = 0, n0 = 0, n2 = 0;
    } seen;
    // flow host node results
    double g_value = 0, g_ms_solve = 0;
    int32_t g_piv = 0;
    int g_frc = DD_OK;
    bool g_skipped = false;
    cudaEvent_t gev[12] = {};  // graph timing: A 0-2, B 3-5, flow 6-9, CompositeToBasic of A 10, of B 11

    // learned warm start: network, per-cell features / outputs / targets
    dd_mlp* mlp = nullptr;
    bool mlp_ready = false;
    uint16_t* d_feat = nullptr;  // maxcell x DD_MLP_NIN (BF16)
    float* d_pred = nullptr;     // maxcell x DD_MLP_NOUT
    float* d_pred_old[2] = {nullptr, nullptr};  // per partition: the outputs used by its last solve
    float* d_targ = nullptr;     // maxcell x DD_MLP_NOUT
    int32_t* d_full[2] = {nullptr, nullptr};  // per partition: cells with a full 8 x 8 block
    long long* d_trace[2] = {nullptr, nullptr};  // DD_FLAG_TRACE: ncell x 4 per partition
    int n_full[2] = {0, 0};
};

// last CUDA error, kept for dd_last_error()
int dd_record_cuda_error(cudaError_t e, const char* where);
inline int launch_status(const char* where) {
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? DD_OK : dd_record_cuda_error(e, where);
}

// kernels / launchers (dd_half.cu)
int launch_plan_half(dd_ctx* c, int part);
int half_padw(int w);
int launch_half(dd_ctx* c, int part, const int32_t* order, int ncell, int* queue, const long long dims[3],
                int threads, size_t smem, int grid, cudaStream_t stream, bool global_boxes = false,
                const int* count_dev = nullptr);
// graph mode: size classes and processing order on the device (see k_classify)
int launch_classify(dd_ctx* c, int part, int stage);
// one eager half-iteration up to the cell kernels (with_c2b: and CompositeToBasic);
// records ev[0] (start), ev[1] (cells), ev[2] (end); does not flip the state
int half_iteration_eager(dd_ctx* c, int part, bool with_c2b);
size_t half_smem_bytes(dd_ctx* c, long long maxarea, long long maxh, long long maxw);
int half_kernel_max_smem();
size_t c2b_smem_bytes(dd_ctx* c, long long maxh, long long maxw);
int launch_c2b(dd_ctx* c, int part, const long long dims[3], size_t smem, const int32_t* order, const int* count);
// the cell kernel on thread-block clusters of `cl` (2 or 4) CTAs, one cluster per
// cell, nclusters clusters; box arrays of cells with goff >= 0 in global scratch
int launch_half_cluster(dd_ctx* c, int part, const int32_t* order, int ncell, int* queue, const long long dims[3],
                        int threads, int cl, size_t smem, int nclusters, cudaStream_t stream,
                        const int* count_dev = nullptr);
int half_cluster_size(int requested);
// the warm-start network runs before this half-iteration's solves of `part`
inline bool mlp_active(const dd_ctx* c, int part) {
    return c->opt.warm == DD_WARM_MLP && (!c->part[part].warm_valid || (c->opt.flags & DD_FLAG_MLP_EVERY_SOLVE));
}
// the previous solve's network outputs are kept for the predicted change of the dual
inline bool mlp_keeps_old(const dd_ctx* c) {
    return c->opt.warm == DD_WARM_MLP && (c->opt.flags & DD_FLAG_MLP_EVERY_SOLVE);
}
// plan transfer: pack c->d_plan64 (packed FP64 boxes at offsets c->d_soff) into
// pool[dst] with the headers in bhdr[dst] (validate: cell masses and the Y
// marginal against m and nu into d_red[0..1], bad-value flag in d_red[2]);
// unpack the current pool into c->d_plan64
int launch_pack_plan(dd_ctx* c, int dst, bool validate);
int launch_unpack_plan(dd_ctx* c);
// per-cell stop budgets of the next solves of `part` into P.budget (dd_options tol_share, tol_gamma)
int launch_budget(dd_ctx* c, int part, cudaStream_t st = nullptr);
// stored X duals of a partition: a <- log2 mu + f (a - log2 mu) (eps change by 1 / f)
int launch_rescale_alpha(dd_ctx* c, int part, double f);
int half_occupancy(int threads, size_t smem);
int launch_feat(dd_ctx* c, int part);
int launch_collect(dd_ctx* c, int n, const int32_t* idx, uint16_t* feat, float* targ);
// dd_mlp.cu
int mlp_forward_dev(dd_mlp* m, const uint16_t* x, int M, float* y, cudaStream_t st, int* err);
// dd_flow.cu
int launch_cbar(dd_ctx* c);
int launch_plan_exchange(dd_ctx* c, int stage = 0);
int launch_exchange(dd_ctx* c);
int launch_l1y(dd_ctx* c, double* out_dev);
// dd_glue.cu
int launch_gamma(dd_ctx* c, int* status_dev);
int launch_cbar_glued(dd_ctx* c);
