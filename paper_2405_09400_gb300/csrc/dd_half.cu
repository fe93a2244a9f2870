// One domain-decomposition half-iteration on the GPU (Alg. 1 as restated in
// Alg. 4), as two kernels:
//
//  k_plan_half  one CTA: for every composite cell the union box of its member
//               boxes (BasicToComposite's output box, Eq. get-composite-cell-
//               marginal), and prefix sums that place the composite marginal and
//               the member outputs in their pools;
//  k_sink       a persistent kernel with a work queue; one CTA solves one
//               composite cell at a time, entirely in shared memory:
//                 1. gather nu_J from the member boxes (BasicToComposite),
//                 2. log-domain Sinkhorn (Section A.1, "Custom CUDA Sinkhorn")
//                    with the separable per-axis log-sum-exp for the squared
//                    cost, until the L1 X error <= tol * mu(X_J),
//               and writes the duals, the objective and the error;
//  k_c2b        one CTA per cell, from those duals:
//                 3. CompositeToBasic by the partial log-sum-exp over each
//                    basic cell (Section A.1, "Online reduction"), with
//                    D_i = <c, pi_i> from the same partial sums,
//                 4. balancing and 5. truncation at `trunc` (Alg. 4), and the
//                    minimal box of each member, compacted in place.
//
// Number format: the LSE runs in FP32 in base 2 (ex2/lg2); masses, errors, D_i,
// moments and the objective accumulate in FP64.
//
// Dual representation. With x = (r0 + u1, c0 + u2) in the cell block and
// y = (o1 + v1, o2 + v2) in the box, the kernel keeps
//   pi(x, y) = 2^( a(u) + b(v) - k2 |ubar - vbar|^2 ),
// where ubar = u - (block centre), vbar = v - (box centre), k2 = h^2/eps*log2(e),
// a absorbs log2 mu(x) and b absorbs log2 nu_J(y). The true duals follow from
//   alpha/eps = ln2 (a + 2 k2 d.ubar + k2|d|^2/2) - ln mu,
//   beta_t/eps = ln2 (b - 2 k2 d.vbar + k2|d|^2/2) - ln nu_J,
// with d = (block centre) - (box centre) in pixels (the linear part of the cost
// is absorbed so that the FP32 duals stay small).
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>

#include "dd_internal.h"

#define RET_IF(x)                   \
    do {                            \
        int r_ = (x);               \
        if (r_ != DD_OK) return r_; \
    } while (0)

namespace cg = cooperative_groups;

namespace {

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2f(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr float kLn2 = 0.69314718055994530942f;

__device__ __forceinline__ unsigned dyn_smem_bytes() {
    unsigned r;
    asm volatile("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
    return r;
}
constexpr double kLn2d = 0.69314718055994530942;

// ---------------------------------------------------------------------------
// block reductions
//
// Sums over a CTA in fixed order. Across the lanes of a warp a value travels as
// an unevaluated sum of two floats (hi + lo, combined by Knuth's error-free
// two-sum: about 48 significant bits), and only the per-warp results are added
// in FP64, by one lane per value: GB300 runs FP64 at 1/64 of the FP32 rate
// shared by the SM, so an FP64 shuffle tree in every warp of every resident CTA
// cost tens of microseconds per cell.
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
    const float s = h + bh;
    const float bb = s - h;
    const float e = ((h - (s - bb)) + (bh - bb)) + (l + bl);  // two-sum error + the low parts
    h = s + e;
    l = e - (h - s);
}

template <int N>
__device__ void block_sum_ff(float (&hi)[N], float (&lo)[N], double (&out)[N], double* sh /* >= 33*N */) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    float* shf = reinterpret_cast<float*>(sh);  // [warp][value][hi, lo] in sh[0, 32 N)
#pragma unroll
    for (int k = 0; k < N; ++k) {
        float h = hi[k], l = lo[k];
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_down_sync(0xffffffffu, h, o);
            const float ol = __shfl_down_sync(0xffffffffu, l, o);
            ff_add(h, l, oh, ol);
        }
        if (lane == 0) {
            shf[2 * (wid * N + k)] = h;
            shf[2 * (wid * N + k) + 1] = l;
        }
    }
    __syncthreads();
    if (threadIdx.x < N) {
        double x = 0.0;
        for (int w = 0; w < nw; ++w)
            x += (double)shf[2 * (w * N + threadIdx.x)] + (double)shf[2 * (w * N + threadIdx.x) + 1];
        sh[32 * N + threadIdx.x] = x;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < N; ++k) out[k] = sh[32 * N + k];
    __syncthreads();
}

// block sum of per-thread FP32 partials, totals in FP64 (valid in every thread)
template <int N>
__device__ void block_sum_f(const float (&v)[N], double (&out)[N], double* sh) {
    float h[N], l[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        h[k] = v[k];
        l[k] = 0.f;
    }
    block_sum_ff<N>(h, l, out, sh);
}

// block sum of per-thread FP64 values (each split into hi + lo floats first)
template <int N>
__device__ void block_sum_d(double (&v)[N], double* sh) {
    float h[N], l[N];
#pragma unroll
    for (int k = 0; k < N; ++k) {
        h[k] = (float)v[k];
        l[k] = (float)(v[k] - (double)h[k]);
    }
    block_sum_ff<N>(h, l, v, sh);
}

// exclusive scan over a block of long long (blockDim.x <= 1024)
__device__ long long block_exscan(long long x, long long* sh, long long* total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    long long inc = x;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) sh[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        long long s = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < nw) sh[lane] = s;  // inclusive warp totals
    }
    __syncthreads();
    long long base = wid > 0 ? sh[wid - 1] : 0;
    *total = sh[nw - 1];
    __syncthreads();
    return base + inc - x;
}

// Row stride of the box arrays in shared memory: a multiple of 4 floats (float4
// access) whose quarter is odd, so that the rows touched by one warp fall in
// different 16-byte bank groups.
__host__ __device__ __forceinline__ int padw(int w) {
    int s = (w + 3) & ~3;
    if (((s >> 2) & 1) == 0) s += 4;
    return s;
}

// ---------------------------------------------------------------------------
// planning: union boxes and pool offsets (one CTA)
__global__ void k_plan_half(int ncell, const int32_t* __restrict__ members, const int32_t* __restrict__ bhdr,
                            int32_t* __restrict__ chdr, const int32_t* __restrict__ xblk, long long* __restrict__ tot) {
    __shared__ long long sh[64];
    __shared__ long long smax[3];
    const int T = blockDim.x;
    const int per = (ncell + T - 1) / T;
    const int c0 = min(ncell, threadIdx.x * per), c1 = min(ncell, c0 + per);
    if (threadIdx.x < 3) smax[threadIdx.x] = 0;
    __syncthreads();
    long long sa = 0, so = 0, ma = 0, mh = 0, mw = 0;
    for (int J = c0; J < c1; ++J) {
        // the four members' header loads are independent: issue them together
        int mi[4], bo1[4], bo2[4], bh[4], bw[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) mi[k] = members[4 * J + k];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int32_t* b = bhdr + (size_t)BH_N * (mi[k] < 0 ? 0 : mi[k]);
            bo1[k] = mi[k] < 0 ? 0 : b[BH_O1];
            bo2[k] = mi[k] < 0 ? 0 : b[BH_O2];
            bh[k] = mi[k] < 0 ? 0 : b[BH_H];
            bw[k] = mi[k] < 0 ? 0 : b[BH_W];
        }
        int lo1 = INT32_MAX, lo2 = INT32_MAX, hi1 = INT32_MIN, hi2 = INT32_MIN;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (bh[k] <= 0 || bw[k] <= 0) continue;
            lo1 = min(lo1, bo1[k]);
            lo2 = min(lo2, bo2[k]);
            hi1 = max(hi1, bo1[k] + bh[k]);
            hi2 = max(hi2, bo2[k] + bw[k]);
        }
        int h = 0, w = 0;
        if (hi1 > lo1) { h = hi1 - lo1; w = hi2 - lo2; } else { lo1 = lo2 = 0; }
        int stride = (w + 3) & ~3;
        int32_t* ch = chdr + (size_t)CH_N * J;
        ch[CH_O1] = lo1; ch[CH_O2] = lo2; ch[CH_H] = h; ch[CH_W] = w; ch[CH_STRIDE] = stride;
        long long area = (long long)h * stride;
        sa += area;
        so += area * xblk[XB_N * J + XB_NMEM];
        ma = max(ma, (long long)h * padw(w));
        mh = max(mh, (long long)h);
        mw = max(mw, (long long)w);
    }
    long long ta, to;
    long long ea = block_exscan(sa, sh, &ta);
    long long eo = block_exscan(so, sh, &to);
    for (int J = c0; J < c1; ++J) {
        int32_t* ch = chdr + (size_t)CH_N * J;
        long long area = (long long)ch[CH_H] * ch[CH_STRIDE];
        ch[CH_COMP_LO] = (int32_t)(ea & 0xffffffffLL);
        ch[CH_COMP_HI] = (int32_t)(ea >> 32);
        ch[CH_OUT_SLOT] = (int32_t)eo;
        ea += area;
        eo += area * xblk[XB_N * J + XB_NMEM];
    }
    atomicMax((unsigned long long*)&smax[0], (unsigned long long)ma);
    atomicMax((unsigned long long*)&smax[1], (unsigned long long)mh);
    atomicMax((unsigned long long*)&smax[2], (unsigned long long)mw);
    __syncthreads();
    if (threadIdx.x == 0) {
        tot[PT_COMP] = ta;
        tot[PT_OUT] = to;
        tot[PT_MAXAREA] = smax[0];
        tot[PT_MAXH] = smax[1];
        tot[PT_MAXW] = smax[2];
    }
}

// ---------------------------------------------------------------------------
struct HalfArgs {
    int N1, N2, s, ncell, amax;
    float k2;
    double k2d;
    double eps, h2;
    const int32_t* members;
    const int32_t* xblk;
    const double* mJ;
    const int32_t* order;
    const int32_t* bhdr_in;
    const float* pool_in;
    int32_t* bhdr_out;
    float* pool_out;
    int32_t* chdr;
    float* comp_b;
    float* comp_nu;
    float* alpha;
    float* gauge;
    int warm;
    const float* lgmu;
    const double* mu;
    const double* nu;
    const double* lnmu;  // ln mu, ln nu (FP64, for the objective)
    const double* lnnu;
    const float* lnnuf;  // ln nu in FP32
    const double* m;
    double tol;
    double tol_share, mbar;  // stop budget tol ((1 - share) mu(X_J) + share mbar)
    const double* budget;    // per-cell stop budgets (absolute), or null for the formula above
    float omega;  // 1: plain Sinkhorn; (1, 2): fixed over-relaxation; < 0: adaptive
    int max_iter, fixed_iters;
    float trunc;
    int32_t* iters;
    double* err;
    double* Ecell;
    double* bmom;
    float* pre;  // optional prebalance copy (same layout as pool_out)
    int* queue;
    int* status;
    float* gscratch;        // box arrays of cells too large for shared memory
    const long long* goff;  // per cell: offset in gscratch, or -1 (shared memory)
    int smaxA, smaxH, smaxW;  // shared-memory capacities
    // learned / analytic warm start (cells with a full 2s x 2s block only)
    int affine;         // start from the cell's affine dual (a = log2 mu in the gauge)
    const float* pred;  // ncell x DD_MLP_NOUT network outputs (first 64: predicted r), or null
    const float* pred_old;  // the outputs of the previous solve of this partition, or null
    float* targ;        // ncell x DD_MLP_NOUT training targets written after the solve, or null
    // Anderson acceleration of the X-dual iteration (tolerance mode): memory, 0 = off
    int aa_m;
    // per cell: 1 once its solving CTA has also done CompositeToBasic (k_sink sets,
    // k_c2b skips such a cell and clears the mark), or null: k_sink leaves it to k_c2b
    int* fused;
    // k_c2b's cell of CTA b: c2b_order[b] (c2b_count null), or from the class lists
    // of k_classify (c2b_count its three counts: the cluster list at 2 ncell first,
    // then the large list at 0 and the small list at ncell); null: cell b
    const int32_t* c2b_order;
    const int* c2b_count;
    // gluing edge candidates: per basic cell and pixel, mass r and mean displacement
    // d (2) of the Gibbs cell plan (nb x s^2 x 3, FP64), or null (product candidates)
    double* pmom;
    // eps-scaling inside each solve (tolerance mode only): levels eps f^L .. eps
    int eps_levels;
    float eps_factor;
    double eps_tol;     // a coarse level ends at L1 X error <= eps_tol * mu(X_J)
    // graph mode
    const int* guard;   // non-zero: a buffer of this iteration would overflow, skip all work
    const int* count;   // cells in `order` (device), instead of ncell
    long long* trace;   // DD_FLAG_TRACE: per cell start / end (ns, globaltimer), SM, CTA size
    // capacities (floats) of the pools the kernels write: a cell whose slots would
    // reach beyond them is skipped and counted in status[4] (never expected)
    long long comp_cap, out_cap, gscr_cap, pre_cap;
};

// shared-memory layout (floats unless noted); BS = padw(max box width)
struct Smem {
    float* lgnu;  // maxH * BS: log2 nu_J (DD_NEG where nu_J = 0 and in the padding)
    float* b;     // maxH * BS: Y dual b~ (DD_NEG where nu_J = 0 and in the padding)
    float* T;     // (2s) * BS: Y-update stage 1
    float* R;     // maxH * (2s): X stage 1
    float* tab1;  // (2s) * maxH: axis-1 kernel (gauge-reduced)
    float* tab2;  // (2s) * BS: axis-2 kernel (gauge-reduced, 0 in the padding)
    float* a;     // 2 * amax: X dual, ping-pong
    float* lgm;   // amax
    float* muxf;  // amax: mu on the block (FP32 copy)
    double* mux;  // amax
    double* red;  // 32 * 16 + 16
    double* B1;   // maxH: min over u1 of the axis-1 kernel at v1 (FP64)
    double* B2;   // BS: min over u2 of the axis-2 kernel at v2
    double* clx;  // 16: per-CTA sums exchanged within a cluster
    float* pm;    // 8 * amax: partial X-update log-sums of every rank of a cluster
                  // ([buffer][rank][u], two buffers, up to 4 ranks), written by the ranks
    float* aa;    // Anderson history (aa_m > 0): residual differences dG[aa_m][amax],
                  // iterate differences dX[aa_m][amax], last residual g[amax], last
                  // iterate x[amax], Gram matrix of dG (kAAMax x kAAMax)
    float* coef;  // 16
    int* ctl;     // 32
    long long end;  // bytes used
};

constexpr int kAAMax = 4;  // largest Anderson memory
// floats of the Anderson history for memory m and X blocks of amax pixels
__host__ __device__ __forceinline__ int aa_floats(int m, int amax) {
    return m > 0 ? (2 * m + 2) * amax + kAAMax * kAAMax : 0;
}

__device__ Smem carve(char* base, const HalfArgs& A) {
    Smem S;
    const int s2 = 2 * A.s;
    const int BS = padw(A.smaxW);
    double* d = reinterpret_cast<double*>(base);
    S.mux = d;
    d += A.amax;
    S.red = d;
    d += 32 * 16 + 16;
    S.B1 = d;
    d += A.smaxH;
    S.B2 = d;
    d += BS;
    S.clx = d;
    d += 16;
    float* f = reinterpret_cast<float*>(((uintptr_t)d + 15) & ~(uintptr_t)15);  // float4 rows
    // every array after this point is read as float4 rows: keep 16-byte offsets
    const int A4 = (A.smaxA + 3) & ~3;
    S.lgnu = f; f += A4;
    S.b = f; f += A4;
    S.T = f; f += s2 * BS;
    S.R = f; f += A.smaxH * s2;
    S.tab1 = f; f += A.smaxH * s2;
    S.tab2 = f; f += BS * s2;
    S.a = f; f += 2 * A.amax;
    S.lgm = f; f += A.amax;
    S.muxf = f; f += A.amax;
    S.pm = f; f += 8 * A.amax;
    S.aa = f; f += aa_floats(A.aa_m, A.amax);
    S.coef = f; f += 16;
    S.ctl = reinterpret_cast<int*>(f);
    S.end = reinterpret_cast<char*>(f + 32) - base;
    return S;
}

// log2 sum_k 2^t_k for a line read through a functor, two passes (exact shift)
template <typename F>
__device__ __forceinline__ float lse2(int n, F term) {
    float m = DD_NEG;
    for (int k = 0; k < n; ++k) m = fmaxf(m, term(k));
    float s = 0.f;
    for (int k = 0; k < n; ++k) s += ex2f(term(k) - m);
    return m + lg2f(s);
}

// a sum s = sum_k 2^(t_k - m) taken with a guessed shift m is trusted when it
// neither over- nor underflows: then no significant term was flushed to zero
__device__ __forceinline__ bool shift_ok(float s) { return s >= 8.67e-19f && s <= 1.15e18f; }  // 2^-60 .. 2^60

constexpr int kMlpBlock = 64;  // X block of a full composite cell (8 x 8 pixels)

// Square root of a symmetric positive semidefinite 2 x 2 matrix [[a, b], [b, c]]:
// (M + sqrt(det M) I) / sqrt(tr M + 2 sqrt(det M)).
__device__ void sqrtm2(double a, double b, double c, double& ra, double& rb, double& rc) {
    const double s = sqrt(fmax(a * c - b * b, 0.0));
    const double t = sqrt(fmax(a + c + 2.0 * s, 0.0));
    if (!(t > 0.0)) { ra = rb = rc = 0.0; return; }
    ra = (a + s) / t; rb = b / t; rc = (c + s) / t;
}

// The cell's affine dual beyond the gauge. With S, T the covariances of mu_J and
// nu_J, A = S^(-1/2) (S^(1/2) T S^(1/2))^(1/2) S^(-1/2) is the transport map
// between Gaussians of those moments; its dual minus the gauge's per-axis part
// is q(u) = k2 ub' (diag(l) - A) ub, returned as (l1 - A11, -A12, l2 - A22).
// When det S <= 1e-6 the per-axis map stands in (q = 0).
__device__ void affine_excess(double s11, double s12, double s22, double t11, double t12, double t22, double l1,
                              double l2, float& q11, float& q12, float& q22) {
    q11 = q12 = q22 = 0.f;
    if (!(s11 * s22 - s12 * s12 > 1e-6)) return;
    double h11, h12, h22;
    sqrtm2(s11, s12, s22, h11, h12, h22);
    const double dh = h11 * h22 - h12 * h12;
    const double i11 = h22 / dh, i12 = -h12 / dh, i22 = h11 / dh;
    // M = Sh T Sh
    const double p11 = h11 * t11 + h12 * t12, p12 = h11 * t12 + h12 * t22;
    const double p21 = h12 * t11 + h22 * t12, p22 = h12 * t12 + h22 * t22;
    const double m11 = p11 * h11 + p12 * h12, m12 = p11 * h12 + p12 * h22, m22 = p21 * h12 + p22 * h22;
    double r11, r12, r22;
    sqrtm2(m11, m12, m22, r11, r12, r22);
    // A = Shi R Shi
    const double e11 = i11 * r11 + i12 * r12, e12 = i11 * r12 + i12 * r22;
    const double e21 = i12 * r11 + i22 * r12, e22 = i12 * r12 + i22 * r22;
    const double a11 = e11 * i11 + e12 * i12, a22 = e21 * i12 + e22 * i22;
    const double a12 = 0.5 * ((e11 * i12 + e12 * i22) + (e21 * i11 + e22 * i12));
    q11 = (float)(l1 - a11);
    q12 = (float)(-a12);
    q22 = (float)(l2 - a22);
}

// Kernel tables of one cell at cost scale k2d (base-2 units per squared pixel).
// With t = vbar / l_k, the axis kernel is
//   K_k(u, v) = k2 l_k (ubar - t)^2,
// its minimum over the block's grid points is B_k(v) = k2 l_k (ubar* - t)^2 at
// the grid point ubar* nearest to t, and the table holds
//   K_k - B_k = k2 l_k D (D + w0),  D = u - u* (integer), w0 = 2 (ubar* - t),
// w0 taken in FP64 per v and rounded once, so that the small values that matter
// keep full FP32 precision. The Y dual is stored as b~ = b - B_1(v1) - B_2(v2)
// (an exact change of gauge). No barrier: the caller synchronises.
__device__ void build_tables(const Smem& S, double k2d, int h, int w, int bs, int hx, int wx, float uc1, float uc2,
                             float vc1, float vc2, float l1, float l2) {
    const int tid = threadIdx.x, NT = blockDim.x;
    const double il1 = S.clx[12], il2 = S.clx[13];  // 1 / l1, 1 / l2
    for (int v1 = tid; v1 < h; v1 += NT) {
        const double tt = (v1 - (double)vc1) * il1;
        const int us = min(hx - 1, max(0, (int)rint(tt + (double)uc1)));
        const double w0 = 2.0 * ((us - (double)uc1) - tt);
        S.B1[v1] = 0.25 * k2d * l1 * w0 * w0;
        const float w0f = (float)w0, kl = (float)(k2d * l1);
        for (int u1 = 0; u1 < hx; ++u1) {
            const float D = (float)(u1 - us);
            S.tab1[u1 * h + v1] = kl * D * (D + w0f);
        }
    }
    for (int v2 = tid; v2 < bs; v2 += NT) {
        if (v2 >= w) {
            for (int u2 = 0; u2 < wx; ++u2) S.tab2[u2 * bs + v2] = 0.f;
            continue;
        }
        const double tt = (v2 - (double)vc2) * il2;
        const int us = min(wx - 1, max(0, (int)rint(tt + (double)uc2)));
        const double w0 = 2.0 * ((us - (double)uc2) - tt);
        S.B2[v2] = 0.25 * k2d * l2 * w0 * w0;
        const float w0f = (float)w0, kl = (float)(k2d * l2);
        for (int u2 = 0; u2 < wx; ++u2) {
            const float D = (float)(u2 - us);
            S.tab2[u2 * bs + v2] = kl * D * (D + w0f);
        }
    }
}

// Training targets of the warm-start network for one solved cell: the dual
// relative to the cell's affine dual, r(u) = a(u) - log2 mu(u) - q(u) in the
// gauge (q: see affine_excess), with a mu-weighted mean of zero, and the
// auxiliary Y-side log dual
//   G(v) = -LSE2_u [a(u) - K(u, v)]
// at the 16 x 16 sample pixels v = ((2i+1) h div 32, (2j+1) w div 32), with a
// plain mean of zero. K = table + B (the tables hold K - B).
__device__ __noinline__ void write_targets(const HalfArgs& A, const Smem& S, int J, const float* aC, int h, int w,
                                           int bs, int hx, int wx, double musum, float uc1, float uc2, float q11,
                                           float q12, float q22) {
    const int tid = threadIdx.x, NT = blockDim.x;
    float* tg = A.targ + (long long)DD_MLP_NOUT * J;
    auto rr = [&](int u) {
        const int u1 = u / wx, u2 = u - u1 * wx;
        const float ub1 = u1 - uc1, ub2 = u2 - uc2;
        return aC[u] - S.lgm[u] - A.k2 * (q11 * ub1 * ub1 + 2.f * q12 * ub1 * ub2 + q22 * ub2 * ub2);
    };
    double cm[1] = {0.0};
    for (int u = tid; u < hx * wx; u += NT)
        if (S.lgm[u] > 0.5f * DD_NEG) cm[0] += S.mux[u] * (double)rr(u);
    block_sum_d<1>(cm, S.red);
    const float sh = (float)(cm[0] / musum);
    for (int u = tid; u < hx * wx; u += NT) tg[u] = S.lgm[u] > 0.5f * DD_NEG ? rr(u) - sh : 0.f;
    double gs[1] = {0.0};
    for (int p = tid; p < 256; p += NT) {
        const int v1 = ((2 * (p >> 4) + 1) * h) / 32, v2 = ((2 * (p & 15) + 1) * w) / 32;
        auto term = [&](int u) {
            const int u1 = u / wx, u2 = u - u1 * wx;
            return aC[u] - S.tab1[u1 * h + v1] - S.tab2[u2 * bs + v2];
        };
        float m = DD_NEG;
        for (int u = 0; u < hx * wx; ++u)
            if (S.lgm[u] > 0.5f * DD_NEG) m = fmaxf(m, term(u));
        float sacc = 0.f;
        for (int u = 0; u < hx * wx; ++u)
            if (S.lgm[u] > 0.5f * DD_NEG) sacc += ex2f(term(u) - m);
        const float G = -(m + lg2f(sacc)) + (float)(S.B1[v1] + S.B2[v2]);
        tg[64 + p] = G;
        gs[0] += G;
    }
    block_sum_d<1>(gs, S.red);
    const float gm = (float)(gs[0] / 256.0);
    for (int p = tid; p < 256; p += NT) tg[64 + p] -= gm;
}

// Sum of per-CTA values (valid in every thread) over the CTAs of the cluster, in
// rank order, so that every CTA gets the same bits. Slots clx[slot, slot + N) of
// every CTA are read remotely after the cluster barrier; the caller passes a
// further cluster barrier before those slots are written again.
template <int N>
__device__ void cluster_sum_d(double (&v)[N], double* clx, int slot) {
    cg::cluster_group cl = cg::this_cluster();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k) clx[slot + k] = v[k];
    }
    cl.sync();
    const unsigned nr = cl.num_blocks();
#pragma unroll
    for (int k = 0; k < N; ++k) {
        double x = 0.0;
        for (unsigned r = 0; r < nr; ++r) x += cl.map_shared_rank(clx, r)[slot + k];
        v[k] = x;
    }
}

// One Anderson step on the X dual (type II, memory m <= kAAMax), run by one warp
// (every lane computes the same coefficients). x = aC is the current iterate and
// aN holds its plain Sinkhorn update F(x); g = F(x) - x. With the columns
// dG_j = g_j - g_(j-1) and dX_j = x_j - x_(j-1) of the last q <= m iterations,
//   gamma = argmin sum_u w(u) (g(u) - sum_j gamma_j dG_j(u))^2   (w = mu / mu(X_J)),
// solved from the normal equations with a Tikhonov term (1e-4 trace / q, at
// least the squared FP32 resolution of the duals) by a Cholesky factorisation,
// and the next iterate
//   x' = x + g - sum_j gamma_j (dX_j + dG_j)
// overwrites aN. q = 0 (first iteration, after a restart) leaves the plain update.
// The history ring holds the columns in slots [0, q); `head` is the slot the new
// column goes to. Coefficients that are not finite or very large keep the plain
// update and restart the history, as does an error more than twice the last one.
__device__ void anderson_step(const Smem& S, int nx, int amax, int m, float err, float err_last,
                              const float* __restrict__ aC, float* __restrict__ aN) {
    const int lane = threadIdx.x & 31;
    // history state in shared memory: ctl[8] = count | head << 4 | prev << 8, ctl[9] = 1 / mu(X_J)
    const int st = S.ctl[8];
    const float wnorm = __int_as_float(S.ctl[9]);
    int cnt = st & 15, head = (st >> 4) & 15;
    bool prev = (st >> 8) & 1;
    if (prev && err > 2.f * err_last) {  // restart when the error more than doubled
        cnt = head = 0;
        prev = false;
    }
    float* const dG = S.aa;
    float* const dX = dG + m * amax;
    float* const gp = dX + m * amax;
    float* const xp = gp + amax;
    float* const Mg = xp + amax;  // kAAMax x kAAMax
    const int q = prev ? min(cnt + 1, m) : cnt;
    const int head_next = prev ? (head + 1 == m ? 0 : head + 1) : head;
    // the new difference column, the stored iterate / residual, and this lane's
    // parts of the new Gram row <dG_head, dG_j> and of the right-hand side <dG_j, g>
    float v[2 * kAAMax];
#pragma unroll
    for (int j = 0; j < 2 * kAAMax; ++j) v[j] = 0.f;
    for (int u = lane; u < nx; u += 32) {
        const bool live = S.lgm[u] > 0.5f * DD_NEG;
        const float g = live ? aN[u] - aC[u] : 0.f;
        const float x = live ? aC[u] : 0.f;
        float gn = 0.f;
        if (prev) {
            gn = g - gp[u];
            dG[head * amax + u] = gn;
            dX[head * amax + u] = x - xp[u];
        }
        gp[u] = g;
        xp[u] = x;
        const float w = S.muxf[u] * wnorm;
#pragma unroll
        for (int j = 0; j < kAAMax; ++j) {
            if (j < q) {
                const float dj = w * dG[j * amax + u];  // own writes: visible to this lane
                v[j] += dj * gn;
                v[kAAMax + j] += dj * g;
            }
        }
    }
    if (q == 0) {  // the plain update stays in aN
        if (lane == 0) S.ctl[8] = (1 << 8);
        return;
    }
    // sum the 8 values over the warp: halve the values per lane at each of the
    // first three steps (lane bit 16, 8, 4), then two plain butterfly steps; lane
    // l ends with the total of value ((l >> 4) & 1) * 4 + ((l >> 3) & 1) * 2 + ((l >> 2) & 1)
    {
        const bool b = lane & 16;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const float send = b ? v[i] : v[i + 4];
            const float keep = b ? v[i + 4] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
    }
    {
        const bool b = lane & 8;
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float send = b ? v[i] : v[i + 2];
            const float keep = b ? v[i + 2] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
    }
    {
        const bool b = lane & 4;
        const float send = b ? v[0] : v[1];
        const float keep = b ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
    v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
    float pm[kAAMax], pr[kAAMax];
#pragma unroll
    for (int k = 0; k < 2 * kAAMax; ++k) {
        const float t = __shfl_sync(0xffffffffu, v[0], ((k >> 2) & 1) * 16 + ((k >> 1) & 1) * 8 + (k & 1) * 4);
        if (k < kAAMax) pm[k] = t;
        else pr[k - kAAMax] = t;
    }
    // Gram matrix: the stored entries, with the new row / column of `head`
    float L[kAAMax][kAAMax];
    float tr = 0.f;
#pragma unroll
    for (int i = 0; i < kAAMax; ++i) {
#pragma unroll
        for (int j = 0; j < kAAMax; ++j) {
            float e = 0.f;
            if (i < q && j < q) e = (prev && i == head) ? pm[j] : (prev && j == head) ? pm[i] : Mg[i * kAAMax + j];
            L[i][j] = e;
        }
        if (i < q) tr += L[i][i];
    }
    if (prev && lane == 0) {  // keep the new row for the next iterations (read after a block barrier)
#pragma unroll
        for (int j = 0; j < kAAMax; ++j)
            if (j < q) {
                Mg[head * kAAMax + j] = pm[j];
                Mg[j * kAAMax + head] = pm[j];
            }
    }
    // Tikhonov term: relative to the Gram trace, and at least the squared FP32
    // resolution of the dual differences (8e-6 in base-2 units), so that
    // columns made of rounding noise get no weight
    const float lam = fmaxf(1e-4f * tr / (float)q, 6.4e-11f);
    bool ok = tr > 0.f && isfinite(tr);
    // the factor's diagonal is kept as its reciprocal (rsqrt, then products only):
    // the coefficients are extrapolation weights, a few ulp do not matter, and the
    // chain of IEEE square roots and divisions is most of the step's latency
    float rd[kAAMax];
#pragma unroll
    for (int j = 0; j < kAAMax; ++j) {
        rd[j] = 0.f;
        if (j < q) {
            float d = L[j][j] + lam;
#pragma unroll
            for (int k = 0; k < kAAMax; ++k)
                if (k < j) d -= L[j][k] * L[j][k];
            ok = ok && d > 0.f;
            rd[j] = rsqrtf(fmaxf(d, 1e-30f));
#pragma unroll
            for (int i = 0; i < kAAMax; ++i) {
                if (i > j && i < q) {
                    float t = L[i][j];
#pragma unroll
                    for (int k = 0; k < kAAMax; ++k)
                        if (k < j) t -= L[i][k] * L[j][k];
                    L[i][j] = t * rd[j];
                }
            }
        }
    }
    float gam[kAAMax];
#pragma unroll
    for (int i = 0; i < kAAMax; ++i) {  // L y = r
        float t = pr[i];
#pragma unroll
        for (int k = 0; k < kAAMax; ++k)
            if (k < i) t -= L[i][k] * gam[k];
        gam[i] = i < q ? t * rd[i] : 0.f;
    }
#pragma unroll
    for (int i = kAAMax - 1; i >= 0; --i) {  // L^T gamma = y
        if (i < q) {
            float t = gam[i];
#pragma unroll
            for (int k = 0; k < kAAMax; ++k)
                if (k > i && k < q) t -= L[k][i] * gam[k];
            gam[i] = t * rd[i];
        }
    }
    float gs = 0.f;
#pragma unroll
    for (int j = 0; j < kAAMax; ++j) gs += fabsf(gam[j]);
    if (!ok || !(gs <= 1e3f)) {  // keep the plain update; restart the history
        if (lane == 0) S.ctl[8] = 0;
        return;
    }
    if (lane == 0) S.ctl[8] = q | (head_next << 4) | (1 << 8);
    for (int u = lane; u < nx; u += 32) {
        if (!(S.lgm[u] > 0.5f * DD_NEG)) continue;
        float xn = xp[u] + gp[u];
#pragma unroll
        for (int j = 0; j < kAAMax; ++j)
            if (j < q) xn -= gam[j] * (dX[j * amax + u] + dG[j * amax + u]);
        aN[u] = xn;
    }
}

// Shared-memory arrays of CompositeToBasic (floats unless noted).
struct C2bSmem {
    double* red;  // 33 x 16 doubles (block sums)
    float* T;     // T2 and M2: 2 x (wx / s) x hx x w
    float* tab1;  // hx x h: axis-1 kernel of the solve's gauge
    float* tab2;  // wx x padw(w): axis-2 kernel
    float* L;     // gluing candidates (pmom): h x wx log2 row sums over v2
    float* E;     // and the means of v2 under them (h x wx)
    float* coef;  // 16
    int* ctl;     // 32 (uses [4, 20))
};

// floats of C2bSmem::T, L and E that one cell needs
__host__ __device__ __forceinline__ long long c2b_cell_floats(int s, int hx, int wx, int h, int w, bool pmom) {
    return 2LL * (wx / s) * hx * w + (pmom ? 2LL * h * wx : 0);
}

__device__ void c2b_cell_fused(const HalfArgs& A, int J, const C2bSmem& S, const float* aC);

// The cell solver. CL = 1: one CTA per cell. CL > 1: the CL CTAs of a thread-block
// cluster solve one cell together (for the few largest cells, which would
// otherwise run alone on one SM for most of the half-iteration): rank r owns the
// box rows [h r / CL, h (r + 1) / CL) for the gather, the Y-update stage 2, the
// X-update stage 1 and the Y side of the outputs; the X-update stage 2 takes a
// partial log-sum-exp over the own rows, and the partials of all ranks are
// combined through distributed shared memory after one cluster barrier per
// iteration, in rank order, so that every CTA holds the same X dual and error and
// takes the same branches. The small X-side work (Y-update stage 1, tables) is
// repeated in every CTA.
template <int NTB, int CL>
__global__ void __launch_bounds__(NTB, 768 / NTB) k_sink(HalfArgs A) {
    extern __shared__ __align__(16) char smem_raw[];
    if (A.guard && *A.guard) return;
    Smem S = carve(smem_raw, A);
    if (S.end > (long long)dyn_smem_bytes() || blockDim.x != NTB) {  // host and kernel disagree on the layout
        if (threadIdx.x == 0) atomicAdd(&A.status[2], 1);
        return;
    }
    const int ncell = A.count ? *A.count : A.ncell;
    const int tid = threadIdx.x, NT = blockDim.x;
    const int lane = tid & 31, wid = tid >> 5;
    int crank = 0;
    if constexpr (CL > 1) crank = (int)cg::this_cluster().block_rank();
    const bool lead = crank == 0;  // writes the per-cell results

    while (true) {
        if constexpr (CL > 1) cg::this_cluster().sync();  // every CTA is done with the previous cell
        if (tid == 0 && lead) S.ctl[0] = atomicAdd(A.queue, 1);
        int t;
        if constexpr (CL > 1) {
            cg::this_cluster().sync();
            t = *cg::this_cluster().map_shared_rank(S.ctl, 0);
        } else {
            __syncthreads();
            t = S.ctl[0];
        }
        if (t >= ncell) break;
        const int J = A.order[t];
        unsigned long long t_start = 0, t_gather = 0, t_loop0 = 0, t_loop1 = 0;
        if (A.trace && tid == 0 && lead) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_start));
        const int32_t* xb = A.xblk + XB_N * J;
        const int r0 = xb[XB_R0], c0 = xb[XB_C0], hx = xb[XB_HX], wx = xb[XB_WX], nmem = xb[XB_NMEM];
        const int32_t* ch = A.chdr + CH_N * J;
        const int o1 = ch[CH_O1], o2 = ch[CH_O2], h = ch[CH_H], w = ch[CH_W], stride = ch[CH_STRIDE];
        const long long comp = ((long long)ch[CH_COMP_HI] << 32) | (unsigned int)ch[CH_COMP_LO];
        const long long slot0 = ch[CH_OUT_SLOT];
        const long long area = (long long)h * stride;
        const int nx = hx * wx, nA = h * w;
        const int bs = padw(w), bq = bs >> 2;
        // log2 nu_J and b~ live in shared memory, or for boxes too large for it
        // in a global scratch slot of the cell (L2-resident)
        const long long go = A.goff ? A.goff[J] : -1;
        if (comp + area > A.comp_cap || (go >= 0 && go + 2LL * h * bs > A.gscr_cap)) {
            if (tid == 0 && lead) atomicAdd(&A.status[4], 1);
            __syncthreads();
            continue;
        }
        // box rows of this CTA
        const int rlo = (h * crank) / CL, rhi = (h * (crank + 1)) / CL;
        float* const lgnu_p = go >= 0 ? A.gscratch + go : S.lgnu;
        float* const b_p = go >= 0 ? A.gscratch + go + (long long)h * bs : S.b;
        int32_t mem[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) mem[k] = A.members[4 * J + k];
        if (nA == 0) {  // no Y mass in the cell: only possible for an infeasible state
            if (tid == 0 && lead) {
                atomicAdd(&A.status[1], 1);
                A.iters[J] = 0;
                A.err[J] = A.mJ[J];
                A.Ecell[J] = 0.0;
                for (int k = 0; k < nmem; ++k) {
                    int32_t* bo = A.bhdr_out + BH_N * mem[k];
                    bo[BH_O1] = bo[BH_O2] = bo[BH_H] = bo[BH_W] = bo[BH_STRIDE] = 0;
                    bo[BH_START] = (int32_t)slot0;
                }
            }
            __syncthreads();
            continue;
        }

        // ---- 1. gather nu_J ---------------------------------------------------
        // per-thread partial sums in FP32 (a few entries each), block sum in FP64;
        // they only choose the change of gauge, which is exact for any value
        float gf[12] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        // member boxes relative to the composite box (registers, read once)
        int mo1[4], mo2[4], mh[4], mw[4], mst[4];
        long long mstart[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            mh[k] = 0; mw[k] = 0; mo1[k] = 0; mo2[k] = 0; mst[k] = 0; mstart[k] = 0;
            if (mem[k] < 0) continue;
            const int32_t* bh = A.bhdr_in + BH_N * mem[k];
            mo1[k] = bh[BH_O1] - o1; mo2[k] = bh[BH_O2] - o2; mh[k] = bh[BH_H]; mw[k] = bh[BH_W];
            mst[k] = bh[BH_STRIDE]; mstart[k] = bh[BH_START];
        }
        for (int v = rlo * bs + tid; v < rhi * bs; v += NT) {
            const int v1 = v / bs, v2 = v - v1 * bs;
            float lg = DD_NEG;
            if (v2 < w) {
                float acc = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int p1 = v1 - mo1[k], p2 = v2 - mo2[k];
                    if (p1 >= 0 && p1 < mh[k] && p2 >= 0 && p2 < mw[k])
                        acc += A.pool_in[mstart[k] + (long long)p1 * mst[k] + p2];
                }
                A.comp_nu[comp + (long long)v1 * stride + v2] = acc;
                if (acc > 0.f) lg = lg2f(acc);
                const float f1 = (float)v1, f2 = (float)v2;
                gf[0] += acc; gf[1] += acc * f1; gf[2] += acc * f2; gf[3] += acc * f1 * f1; gf[4] += acc * f2 * f2;
                gf[10] += acc * f1 * f2;
            }
            lgnu_p[v] = lg;
            b_p[v] = DD_NEG;
        }
        for (int q = tid; q < hx * bs; q += NT) S.T[q] = DD_NEG;
        for (int u = tid; u < nx; u += NT) {
            const int u1 = u / wx, u2 = u - u1 * wx;
            const float mux = (float)A.mu[(r0 + u1) * A.N2 + (c0 + u2)];
            const float f1 = (float)u1, f2 = (float)u2;
            gf[5] += mux; gf[6] += mux * f1; gf[7] += mux * f2; gf[8] += mux * f1 * f1; gf[9] += mux * f2 * f2;
            gf[11] += mux * f1 * f2;
        }
        double gm[12];
        block_sum_f<12>(gf, gm, S.red);
        if (A.trace && tid == 0 && lead) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_gather));
        if constexpr (CL > 1) {  // nu_J moments over all rows (the mu moments are complete in every CTA)
            double nv[6] = {gm[0], gm[1], gm[2], gm[3], gm[4], gm[10]};
            cluster_sum_d<6>(nv, S.clx, 0);
            gm[0] = nv[0]; gm[1] = nv[1]; gm[2] = nv[2]; gm[3] = nv[3]; gm[4] = nv[4]; gm[10] = nv[5];
        }
        // Reparametrisation (exact for any choice): origins at the barycentres of
        // mu_J and nu_J, the linear part of the cost absorbed through d, and a
        // per-axis stretch l_k absorbed so that the kernel
        //   k2 (sqrt(l_k) ubar_k - vbar_k / sqrt(l_k))^2
        // is small along the cell's local map; keeps the FP32 duals small.
        // The scalars are computed in FP64 by one warp and shared through shared
        // memory: at GB300's FP64 rate the same divisions and square roots in
        // every thread of a 512-thread CTA would cost microseconds per solve.
        // The affine start (and the learned one) use the full 2 x 2 map (q), needed
        // only where a solve starts from it or writes training targets.
        const bool need_q = (A.affine && !A.warm) || (A.pred && nx == kMlpBlock) || A.targ;
        if (wid == 0) {
            // two FP64 reciprocals and products (each FP64 division is a long
            // sequence at GB300's FP64 rate); the stretch ratio in FP32 (the gauge
            // is exact for any value)
            const double i5 = 1.0 / gm[5], i0 = 1.0 / gm[0];
            const double duc1 = gm[6] * i5, duc2 = gm[7] * i5;
            const double dvc1 = gm[1] * i0, dvc2 = gm[2] * i0;
            const float fuc1 = (float)duc1, fuc2 = (float)duc2, fvc1 = (float)dvc1, fvc2 = (float)dvc2;
            const double vu1 = fmax(gm[8] * i5 - (double)fuc1 * fuc1, 0.0), vu2 = fmax(gm[9] * i5 - (double)fuc2 * fuc2, 0.0);
            const double vv1 = fmax(gm[3] * i0 - (double)fvc1 * fvc1, 0.0), vv2 = fmax(gm[4] * i0 - (double)fvc2 * fvc2, 0.0);
            const float fl1 = (vu1 > 1e-3) ? fminf(8.f, fmaxf(0.125f, sqrtf((float)vv1 / (float)vu1))) : 1.f;
            const float fl2 = (vu2 > 1e-3) ? fminf(8.f, fmaxf(0.125f, sqrtf((float)vv2 / (float)vu2))) : 1.f;
            float fq11 = 0.f, fq12 = 0.f, fq22 = 0.f;
            if (need_q)
                affine_excess(vu1, gm[11] * i5 - (double)fuc1 * fuc2, vu2, vv1, gm[10] * i0 - (double)fvc1 * fvc2,
                              vv2, fl1, fl2, fq11, fq12, fq22);
            if (lane == 0) {
                S.coef[0] = fuc1; S.coef[1] = fuc2; S.coef[2] = fvc1; S.coef[3] = fvc2;
                S.coef[4] = fl1; S.coef[5] = fl2; S.coef[6] = fq11; S.coef[7] = fq12; S.coef[8] = fq22;
                S.clx[12] = 1.0 / (double)fl1;  // for the kernel tables
                S.clx[13] = 1.0 / (double)fl2;
                S.clx[14] = (double)(float)(1.0 / gm[5]);  // 1 / mu(X_J) (FP32 value)
                // exact displacement of the float origins (FP64) for the gauge
                // conversion of the outputs, and its constant term
                const double x1 = (double)(r0 - o1) + (double)fuc1 - (double)fvc1;
                const double x2 = (double)(c0 - o2) + (double)fuc2 - (double)fvc2;
                S.clx[9] = x1;
                S.clx[10] = x2;
                S.clx[11] = 0.5 * A.k2d * (x1 * x1 + x2 * x2);
            }
        }
        __syncthreads();
        const float uc1 = S.coef[0], uc2 = S.coef[1], vc1 = S.coef[2], vc2 = S.coef[3];
        const float l1 = S.coef[4], l2 = S.coef[5];
        const float q11 = S.coef[6], q12 = S.coef[7], q22 = S.coef[8];
        const float d1 = (float)(r0 - o1) + uc1 - vc1, d2 = (float)(c0 - o2) + uc2 - vc2;
        // Kernel tables (see build_tables), at the coarsest level of the optional
        // eps-scaling: eps_L = eps f^L, the cost in base-2 units k2 / f^L.
        const bool scaling = A.eps_levels > 0 && A.fixed_iters <= 0;
        int lev = scaling ? A.eps_levels : 0;
        float lev_scale = 1.f;  // eps / eps_level
        for (int k = 0; k < lev; ++k) lev_scale /= A.eps_factor;
        build_tables(S, A.k2d * (double)lev_scale, h, w, bs, hx, wx, uc1, uc2, vc1, vc2, l1, l2);
        // X side: log2 mu and the warm start
        float* aC = S.a;
        float* aN = S.a + A.amax;
        const float* ap = A.alpha + (long long)A.amax * J;
        const float* pg = A.gauge + 8 * J;
        const float pd1 = pg[0], pd2 = pg[1], pl1 = pg[2], pl2 = pg[3];
        // network prediction r of the dual relative to the cell's affine dual, and
        // the prediction for the previous solve of the cell (same X block)
        const float* pr = (A.pred && nx == kMlpBlock) ? A.pred + (long long)DD_MLP_NOUT * J : nullptr;
        const float* pro = (pr && A.pred_old && A.warm) ? A.pred_old + (long long)DD_MLP_NOUT * J : nullptr;
        for (int u = tid; u < nx; u += NT) {
            const int u1 = u / wx, u2 = u - u1 * wx;
            const int x = (r0 + u1) * A.N2 + (c0 + u2);
            S.mux[u] = A.mu[x];
            S.muxf[u] = (float)A.mu[x];
            const float lg = A.lgmu[x];
            S.lgm[u] = lg;
            const float ub1 = u1 - uc1, ub2 = u2 - uc2;
            float a0;
            const float qa = A.k2 * (q11 * ub1 * ub1 + 2.f * q12 * ub1 * ub2 + q22 * ub2 * ub2);
            // the previous dual of this cell in the new gauge (mu_J, hence uc, is
            // the same; only d and l change): exact change of gauge
            const float aprev = A.warm ? ap[u] + 2.f * A.k2 * ((pd1 - d1) * ub1 + (pd2 - d2) * ub2) +
                                             A.k2 * ((l1 - pl1) * ub1 * ub1 + (l2 - pl2) * ub2 * ub2)
                                       : 0.f;
            if (pro)  // previous dual + the network's predicted change of the dual
                a0 = aprev + (pr[u] - pro[u]);
            else if (pr)  // first solve: the network's prediction
                a0 = lg + qa + pr[u];
            else if (A.warm)
                a0 = aprev;
            else if (A.affine)
                a0 = lg + qa;
            else
                a0 = lg - 2.f * A.k2 * (d1 * ub1 + d2 * ub2) + A.k2 * ((l1 - 1.f) * ub1 * ub1 + (l2 - 1.f) * ub2 * ub2);
            // at a coarser level the dual relative to log2 mu scales as 1 / eps
            aC[u] = lg > 0.5f * DD_NEG ? lg + lev_scale * (a0 - lg) : DD_NEG;
        }
        {
            // the duals are defined up to (a + C, b - C): start every solve with
            // a mu-weighted mean of zero, so that no constant accumulates across
            // warm starts and the FP32 values keep their resolution
            // (FP32: the shift only picks the gauge)
            float cmf[1] = {0.f};
            for (int u = tid; u < nx; u += NT)
                if (aC[u] > 0.5f * DD_NEG) cmf[0] += S.muxf[u] * aC[u];
            double cm[1];
            block_sum_f<1>(cmf, cm, S.red);
            const float shift = (float)cm[0] * (float)S.clx[14];
            for (int u = tid; u < nx; u += NT)
                if (aC[u] > 0.5f * DD_NEG) aC[u] -= shift;
            if (tid == 0) {  // empty Anderson history; its weights mu / mu(X_J)
                S.ctl[8] = 0;
                S.ctl[9] = __float_as_int((float)S.clx[14]);
            }
        }
        __syncthreads();

        // ---- 2. Sinkhorn (4 barriers per iteration) ----------------------------
        // Every log-sum-exp is first taken with the previous iteration's value of
        // the same line as the shift (one pass); lines whose sum over- or
        // underflows, and all lines of the first iteration, use the exact max.
        // the error bookkeeping is FP32: it only decides when to stop, and GB300's
        // FP64 rate (1/64 of FP32) would make a per-iteration FP64 sum by every
        // thread a large share of an iteration of a big cell
        const float tolm = (float)(A.budget ? A.budget[J]
                                            : A.tol * ((1.0 - A.tol_share) * A.mJ[J] + A.tol_share * A.mbar));
        const float eps_tolm = (float)(A.eps_tol * A.mJ[J]);
        int it = 0;
        float err = 0.f, best = 3.0e38f;
        int since = 0;
        bool stalled = false, first = true;
        // over-relaxation of the X-update (same fixed point): a <- a + w (X(b) - a).
        // Adaptive: plain for the first iterations, then w from the observed
        // contraction r of the error, w = 2 / (1 + sqrt(1 - r)) (Young's rule).
        // Anderson acceleration replaces the over-relaxation when it is on
        const bool aa_on = A.aa_m > 0 && A.fixed_iters <= 0;
        float om = (A.omega > 1.f && !aa_on) ? A.omega : 1.f;
        float err_prev = 0.f, err_mark = 0.f;
        int om_start = 5;

        // threads per line of the X-update stage 2 (a power of two, lanes adjacent)
        int P2 = 1;
        while (P2 * 2 * nx <= NT && P2 < 16) P2 *= 2;
        const int nxl = (rhi - rlo) * wx;  // X-update stage 1 lines of this CTA
        // lines in full rounds of NT take one lane each; the rest, PX lanes each
        // (the last round is otherwise a few lines for a few warps while the other
        // warps wait at the barrier)
        const int xfull = nxl > NT ? (nxl / NT) * NT : 0;
        int PX = 1;
        while (PX * 2 * (nxl - xfull) <= NT && PX < 8) PX *= 2;
        const float4* b4 = reinterpret_cast<const float4*>(b_p);
        const float4* t24 = reinterpret_cast<const float4*>(S.tab2);
        const int nq = (w + 3) >> 2;  // float4 groups holding data per row
        // 2D cursors of the per-entry loops (no integer division per entry):
        // Y-update 1 over (u1, v2) with rows of w, Y-update 2 over (v1, g4) with rows of nq
        const int y1u0 = tid / w, y1v0 = tid - y1u0 * w, y1du = NT / w, y1dv = NT - y1du * w;
        const int y2u0 = rlo + tid / nq, y2v0 = tid - (tid / nq) * nq, y2du = NT / nq, y2dv = NT - y2du * nq;
        int lp2 = 0, lpx = 0;
        while ((1 << lp2) < P2) ++lp2;
        while ((1 << lpx) < PX) ++lpx;
        if (A.trace && tid == 0 && lead) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_loop0));
        while (true) {
            ++it;
            // Y-update stage 1: T(u1, v2) = LSE_u2 [a(u1, u2) - K2(u2, v2)]
            // (full 8 x 8 blocks: all operands loaded first, fixed trip counts)
            if (hx == 8 && wx == 8) {
                int u1 = y1u0, v2 = y1v0;
                for (int q = tid; q < 8 * w; q += NT, u1 += y1du, v2 += y1dv) {
                    if (v2 >= w) { v2 -= w; ++u1; }
                    const float4 a0 = reinterpret_cast<const float4*>(aC + u1 * 8)[0];
                    const float4 a1 = reinterpret_cast<const float4*>(aC + u1 * 8)[1];
                    const float* tb = S.tab2 + v2;
                    float d[8];
                    d[0] = a0.x - tb[0]; d[1] = a0.y - tb[bs]; d[2] = a0.z - tb[2 * bs]; d[3] = a0.w - tb[3 * bs];
                    d[4] = a1.x - tb[4 * bs]; d[5] = a1.y - tb[5 * bs]; d[6] = a1.z - tb[6 * bs];
                    d[7] = a1.w - tb[7 * bs];
                    float m = first ? 0.f : S.T[u1 * bs + v2];
                    float sacc = 0.f;
                    if (!first) {
                        float s0 = 0.f, s1 = 0.f;
#pragma unroll
                        for (int k = 0; k < 8; k += 2) {
                            s0 += ex2f(d[k] - m);
                            s1 += ex2f(d[k + 1] - m);
                        }
                        sacc = s0 + s1;
                    }
                    if (first || !shift_ok(sacc)) {
                        m = DD_NEG;
#pragma unroll
                        for (int k = 0; k < 8; ++k) m = fmaxf(m, d[k]);
                        sacc = 0.f;
#pragma unroll
                        for (int k = 0; k < 8; ++k) sacc += ex2f(d[k] - m);
                    }
                    S.T[u1 * bs + v2] = m + lg2f(sacc);
                }
            } else
            for (int q = tid, u1 = y1u0, v2 = y1v0; q < hx * w; q += NT, u1 += y1du, v2 += y1dv) {
                if (v2 >= w) { v2 -= w; ++u1; }
                const float* ar = aC + u1 * wx;
                const float* tb = S.tab2 + v2;
                float m = first ? 0.f : S.T[u1 * bs + v2];
                float sacc = 0.f;
                if (!first) {
                    float s0 = 0.f, s1 = 0.f;
#pragma unroll
                    for (int u2 = 0; u2 < 16; u2 += 2) {
                        if (u2 >= wx) break;
                        s0 += ex2f(ar[u2] - tb[u2 * bs] - m);
                        if (u2 + 1 < wx) s1 += ex2f(ar[u2 + 1] - tb[(u2 + 1) * bs] - m);
                    }
                    sacc = s0 + s1;
                }
                if (first || !shift_ok(sacc)) {
                    m = DD_NEG;
                    for (int u2 = 0; u2 < wx; ++u2) m = fmaxf(m, ar[u2] - tb[u2 * bs]);
                    sacc = 0.f;
                    for (int u2 = 0; u2 < wx; ++u2) sacc += ex2f(ar[u2] - tb[u2 * bs] - m);
                }
                S.T[u1 * bs + v2] = m + lg2f(sacc);
            }
            __syncthreads();
            // Y-update stage 2: b(v) = log2 nu_J(v) - LSE_u1 [T(u1, v2) - K1(u1, v1)],
            // four adjacent v2 per thread (float4 rows of T, b, log2 nu_J)
            if (NTB < 512 && hx == 8 && !first) {
                // full blocks after the first iteration: operands loaded first
                int v1 = y2u0, g4 = y2v0;
                for (int q = rlo * nq + tid; q < rhi * nq; q += NT, v1 += y2du, g4 += y2dv) {
                    if (g4 >= nq) { g4 -= nq; ++v1; }
                    const float4 ln4 = reinterpret_cast<const float4*>(lgnu_p)[v1 * bq + g4];
                    const float4 bp4 = b4[v1 * bq + g4];
                    const float* tb = S.tab1 + v1;
                    float4 T4[8];
                    float kk[8];
#pragma unroll
                    for (int u1 = 0; u1 < 8; ++u1) {
                        T4[u1] = reinterpret_cast<const float4*>(S.T + u1 * bs)[g4];
                        kk[u1] = tb[u1 * h];
                    }
                    const float ln[4] = {ln4.x, ln4.y, ln4.z, ln4.w};
                    const float bp[4] = {bp4.x, bp4.y, bp4.z, bp4.w};
                    // one shift for the four columns (as in the 512-thread path below)
                    float m0 = DD_NEG, sa[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (ln[k] > 0.5f * DD_NEG) m0 = fmaxf(m0, ln[k] - bp[k]);
                        sa[k] = 0.f;
                    }
                    if (!(m0 > 0.5f * DD_NEG)) m0 = 0.f;
#pragma unroll
                    for (int u1 = 0; u1 < 8; ++u1) {
                        const float km = kk[u1] + m0;
                        sa[0] += ex2f(T4[u1].x - km);
                        sa[1] += ex2f(T4[u1].y - km);
                        sa[2] += ex2f(T4[u1].z - km);
                        sa[3] += ex2f(T4[u1].w - km);
                    }
                    float out[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const int v2 = 4 * g4 + k;
                        if (v2 >= w || !(ln[k] > 0.5f * DD_NEG)) { out[k] = DD_NEG; continue; }
                        float mk = m0;
                        if (!shift_ok(sa[k])) {
                            float mm = DD_NEG;
                            for (int u1 = 0; u1 < 8; ++u1) mm = fmaxf(mm, S.T[u1 * bs + v2] - tb[u1 * h]);
                            float ss = 0.f;
                            for (int u1 = 0; u1 < 8; ++u1) ss += ex2f(S.T[u1 * bs + v2] - tb[u1 * h] - mm);
                            mk = mm;
                            sa[k] = ss;
                        }
                        out[k] = ln[k] - (mk + lg2f(sa[k]));
                    }
                    reinterpret_cast<float4*>(b_p)[v1 * bq + g4] = make_float4(out[0], out[1], out[2], out[3]);
                }
            } else if (hx == 8 && !first) {
                // full blocks after the first iteration (512-thread CTAs): a thread
                // keeps the 8 x 4 values of T of its column group in registers and
                // walks its rows (row blocks nrb rows apart), so T is read once
                const int nrows = rhi - rlo;
                const int nrb = max(1, min(nrows, NT / nq));
                for (int q = tid; q < nrb * nq; q += NT) {
                    const int rb = q / nq, g4 = q - rb * nq;
                    float4 T4[8];
#pragma unroll
                    for (int u1 = 0; u1 < 8; ++u1) T4[u1] = reinterpret_cast<const float4*>(S.T + u1 * bs)[g4];
                    for (int v1 = rlo + rb; v1 < rhi; v1 += nrb) {
                        const float4 ln4 = reinterpret_cast<const float4*>(lgnu_p)[v1 * bq + g4];
                        const float4 bp4 = b4[v1 * bq + g4];
                        const float* tb = S.tab1 + v1;
                        float kk[8];
#pragma unroll
                        for (int u1 = 0; u1 < 8; ++u1) kk[u1] = tb[u1 * h];
                        const float ln[4] = {ln4.x, ln4.y, ln4.z, ln4.w};
                        const float bp[4] = {bp4.x, bp4.y, bp4.z, bp4.w};
                        // one shift for the four columns: the largest of their previous
                        // values (adjacent columns' log-sums differ little; a column whose
                        // sum leaves 2^+-60 is taken again exactly), so that a term costs
                        // one subtraction from a per-row kk + shift
                        float m0 = DD_NEG, sa[4], sb[4];  // even / odd u1: shorter add chains
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            if (ln[k] > 0.5f * DD_NEG) m0 = fmaxf(m0, ln[k] - bp[k]);
                            sa[k] = 0.f;
                            sb[k] = 0.f;
                        }
                        if (!(m0 > 0.5f * DD_NEG)) m0 = 0.f;
                        float km[8];
#pragma unroll
                        for (int u1 = 0; u1 < 8; ++u1) km[u1] = kk[u1] + m0;
#pragma unroll
                        for (int u1 = 0; u1 < 8; u1 += 2) {
                            sa[0] += ex2f(T4[u1].x - km[u1]);
                            sa[1] += ex2f(T4[u1].y - km[u1]);
                            sa[2] += ex2f(T4[u1].z - km[u1]);
                            sa[3] += ex2f(T4[u1].w - km[u1]);
                            sb[0] += ex2f(T4[u1 + 1].x - km[u1 + 1]);
                            sb[1] += ex2f(T4[u1 + 1].y - km[u1 + 1]);
                            sb[2] += ex2f(T4[u1 + 1].z - km[u1 + 1]);
                            sb[3] += ex2f(T4[u1 + 1].w - km[u1 + 1]);
                        }
#pragma unroll
                        for (int k = 0; k < 4; ++k) sa[k] += sb[k];
                        float out[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const int v2 = 4 * g4 + k;
                            if (v2 >= w || !(ln[k] > 0.5f * DD_NEG)) { out[k] = DD_NEG; continue; }
                            float mk = m0;
                            if (!shift_ok(sa[k])) {
                                float mm = DD_NEG;
                                for (int u1 = 0; u1 < 8; ++u1) mm = fmaxf(mm, S.T[u1 * bs + v2] - tb[u1 * h]);
                                float ss = 0.f;
                                for (int u1 = 0; u1 < 8; ++u1) ss += ex2f(S.T[u1 * bs + v2] - tb[u1 * h] - mm);
                                mk = mm;
                                sa[k] = ss;
                            }
                            out[k] = ln[k] - (mk + lg2f(sa[k]));
                        }
                        reinterpret_cast<float4*>(b_p)[v1 * bq + g4] = make_float4(out[0], out[1], out[2], out[3]);
                    }
                }
            } else
            for (int q = rlo * nq + tid, v1 = y2u0, g4 = y2v0; q < rhi * nq; q += NT, v1 += y2du, g4 += y2dv) {
                if (g4 >= nq) { g4 -= nq; ++v1; }
                const float4 ln4 = reinterpret_cast<const float4*>(lgnu_p)[v1 * bq + g4];
                const float4 bp4 = b4[v1 * bq + g4];
                const float ln[4] = {ln4.x, ln4.y, ln4.z, ln4.w};
                const float bp[4] = {bp4.x, bp4.y, bp4.z, bp4.w};
                float m[4], sa[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    m[k] = first ? 0.f : (ln[k] > 0.5f * DD_NEG ? ln[k] - bp[k] : 0.f);
                    sa[k] = 0.f;
                }
                const float* tb = S.tab1 + v1;
                if (!first) {
#pragma unroll
                    for (int u1 = 0; u1 < 16; ++u1) {
                        if (u1 >= hx) break;
                        const float4 T4 = reinterpret_cast<const float4*>(S.T + u1 * bs)[g4];
                        const float kk = tb[u1 * h];
                        sa[0] += ex2f(T4.x - kk - m[0]);
                        sa[1] += ex2f(T4.y - kk - m[1]);
                        sa[2] += ex2f(T4.z - kk - m[2]);
                        sa[3] += ex2f(T4.w - kk - m[3]);
                    }
                }
                float out[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int v2 = 4 * g4 + k;
                    if (v2 >= w || !(ln[k] > 0.5f * DD_NEG)) { out[k] = DD_NEG; continue; }
                    if (first || !shift_ok(sa[k])) {
                        float mm = DD_NEG;
                        for (int u1 = 0; u1 < hx; ++u1) mm = fmaxf(mm, S.T[u1 * bs + v2] - tb[u1 * h]);
                        float ss = 0.f;
                        for (int u1 = 0; u1 < hx; ++u1) ss += ex2f(S.T[u1 * bs + v2] - tb[u1 * h] - mm);
                        m[k] = mm;
                        sa[k] = ss;
                    }
                    out[k] = ln[k] - (m[k] + lg2f(sa[k]));
                }
                reinterpret_cast<float4*>(b_p)[v1 * bq + g4] = make_float4(out[0], out[1], out[2], out[3]);
            }
            __syncthreads();
            // X-update stage 1: R(v1, u2) = LSE_v2 [b(v1, v2) - K2(u2, v2)], float4 over
            // v2; PX adjacent lanes per line (strided float4 groups), combined by
            // warp shuffles, so that short row ranges (clusters) keep every lane busy
            for (int ph = 0; ph < 2; ++ph) {
            const int PXc = ph == 0 ? 1 : PX, lpxc = ph == 0 ? 0 : lpx;
            const int nl = ph == 0 ? xfull : nxl - xfull, l0 = ph == 0 ? 0 : xfull;
            for (int base = 0; base < nl * PXc; base += NT) {
                const int q = base + tid;
                const bool act = q < nl * PXc;
                const int ql = act ? l0 + (q >> lpxc) : 0, p = q & (PXc - 1);
                const int line = rlo * wx + ql;
                const int v1 = line / wx, u2 = line - v1 * wx;
                const float4* br = b4 + v1 * bq;
                const float4* tr = t24 + u2 * bq;
                float m = (first || !act) ? 0.f : S.R[line];
                float sacc = 0.f;
                if (act && !first) {
                    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
                    int g = p;
                    for (; g + PXc < nq; g += 2 * PXc) {
                        const float4 bb = br[g], tt = tr[g], bc = br[g + PXc], tc = tr[g + PXc];
                        s0 += ex2f(bb.x - tt.x - m) + ex2f(bb.y - tt.y - m);
                        s1 += ex2f(bb.z - tt.z - m) + ex2f(bb.w - tt.w - m);
                        s2 += ex2f(bc.x - tc.x - m) + ex2f(bc.y - tc.y - m);
                        s3 += ex2f(bc.z - tc.z - m) + ex2f(bc.w - tc.w - m);
                    }
                    if (g < nq) {
                        const float4 bb = br[g], tt = tr[g];
                        s0 += ex2f(bb.x - tt.x - m) + ex2f(bb.y - tt.y - m);
                        s1 += ex2f(bb.z - tt.z - m) + ex2f(bb.w - tt.w - m);
                    }
                    sacc = (s0 + s1) + (s2 + s3);
                }
                for (int o = 1; o < PXc; o <<= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
                const bool bad = act && (first || !shift_ok(sacc));
                if (__any_sync(0xffffffffu, bad)) {
                    float mm = DD_NEG;
                    if (act)
                        for (int g = p; g < nq; g += PXc) {
                            const float4 bb = br[g], tt = tr[g];
                            mm = fmaxf(fmaxf(fmaxf(mm, bb.x - tt.x), fmaxf(bb.y - tt.y, bb.z - tt.z)), bb.w - tt.w);
                        }
                    for (int o = 1; o < PXc; o <<= 1) mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, o));
                    float ss = 0.f;
                    if (act)
                        for (int g = p; g < nq; g += PXc) {
                            const float4 bb = br[g], tt = tr[g];
                            ss += ex2f(bb.x - tt.x - mm) + ex2f(bb.y - tt.y - mm) + ex2f(bb.z - tt.z - mm) +
                                  ex2f(bb.w - tt.w - mm);
                        }
                    for (int o = 1; o < PXc; o <<= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
                    if (bad) { m = mm; sacc = ss; }
                }
                if (act && p == 0) S.R[line] = m + lg2f(sacc);
            }
            }
            __syncthreads();
            // X-update stage 2: a'(u) = log2 mu(u) - LSE_v1 [R(v1, u2) - K1(u1, v1)],
            // P2 adjacent lanes per line, combined by warp shuffles; L1 X error.
            // In a cluster each CTA first takes the log-sum over its own rows
            // (shifted by its own previous partial) into pm[it & 1].
            float e_loc = 0.f;
            // [buffer][rank][u]: every rank stores its partials into every rank's
            // buffer, so that the combine reads local shared memory
            float* const pcur = S.pm + (it & 1) * 4 * A.amax;
            const float* const pprev = S.pm + ((it + 1) & 1) * 4 * A.amax + crank * A.amax;
            for (int base = 0; base < nx * P2; base += NT) {
                const int q = base + tid;
                const bool act = q < nx * P2;
                const int line = act ? (q >> lp2) : 0, part = q & (P2 - 1);
                const int u1 = wx == 8 ? (line >> 3) : line / wx, u2 = line - u1 * wx;
                const float lg = act ? S.lgm[line] : DD_NEG;
                const bool live = lg > 0.5f * DD_NEG;
                const float* Rc = S.R + u2;
                const float* tb = S.tab1 + u1 * h;
                float m = (first || !live) ? 0.f : (CL > 1 ? pprev[line] : lg - aC[line]);
                float sacc = 0.f;
                if (live && !first) {
                    float s0 = 0.f, s1 = 0.f;
                    int v1 = rlo + part;
                    for (; v1 + P2 < rhi; v1 += 2 * P2) {
                        s0 += ex2f(Rc[v1 * wx] - tb[v1] - m);
                        s1 += ex2f(Rc[(v1 + P2) * wx] - tb[v1 + P2] - m);
                    }
                    if (v1 < rhi) s0 += ex2f(Rc[v1 * wx] - tb[v1] - m);
                    sacc = s0 + s1;
                }
                for (int o = 1; o < P2; o <<= 1) sacc += __shfl_xor_sync(0xffffffffu, sacc, o);
                const bool bad = live && (first || !shift_ok(sacc));
                if (__any_sync(0xffffffffu, bad)) {
                    float mm = DD_NEG;
                    if (live)
                        for (int v1 = rlo + part; v1 < rhi; v1 += P2) mm = fmaxf(mm, Rc[v1 * wx] - tb[v1]);
                    for (int o = 1; o < P2; o <<= 1) mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, o));
                    float ss = 0.f;
                    if (live)
                        for (int v1 = rlo + part; v1 < rhi; v1 += P2) ss += ex2f(Rc[v1 * wx] - tb[v1] - mm);
                    for (int o = 1; o < P2; o <<= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
                    if (bad) { m = mm; sacc = ss; }
                }
                if constexpr (CL > 1) {
                    if (act && part == 0) {
                        const float L = (live && sacc > 0.f) ? m + lg2f(sacc) : DD_NEG;
#pragma unroll
                        for (int r = 0; r < CL; ++r)
                            cg::this_cluster().map_shared_rank(pcur, (unsigned)r)[crank * A.amax + line] = L;
                    }
                } else {
                    if (act && part == 0) {
                        const float an = live ? lg - (m + lg2f(sacc)) : DD_NEG;
                        aN[line] = (live && om != 1.f) ? aC[line] + om * (an - aC[line]) : an;
                        if (live) e_loc += S.muxf[line] * fabsf(expm1f((aC[line] - an) * kLn2));
                    }
                }
            }
            if constexpr (CL > 1) {
                // combine the partials of all ranks (rank order: identical in every CTA)
                cg::cluster_group cl = cg::this_cluster();
                cl.sync();
                for (int u = tid; u < nx; u += NT) {
                    const float lg = S.lgm[u];
                    if (!(lg > 0.5f * DD_NEG)) {
                        aN[u] = DD_NEG;
                        continue;
                    }
                    float pr[CL];
                    float mx = DD_NEG;
#pragma unroll
                    for (int r = 0; r < CL; ++r) {
                        pr[r] = pcur[r * A.amax + u];
                        mx = fmaxf(mx, pr[r]);
                    }
                    float sm = 0.f;
#pragma unroll
                    for (int r = 0; r < CL; ++r) sm += ex2f(pr[r] - mx);
                    const float an = lg - (mx + lg2f(sm));
                    aN[u] = om != 1.f ? aC[u] + om * (an - aC[u]) : an;
                    e_loc += S.muxf[u] * fabsf(expm1f((aC[u] - an) * kLn2));
                }
            }
            for (int o = 16; o > 0; o >>= 1) e_loc += __shfl_down_sync(0xffffffffu, e_loc, o);
            float* const redf = reinterpret_cast<float*>(S.red);
            if (lane == 0) redf[wid] = e_loc;
            __syncthreads();
            err = 0.f;
#pragma unroll
            for (int k = 0; k < (NTB >> 5); ++k) err += redf[k];  // NTB == blockDim.x
            first = false;
            // stall: no 1% improvement for 64 iterations while already within
            // 50 tol (the FP32 rounding floor of this cell has been reached)
            if (err < 0.99f * best) { best = err; since = 0; } else ++since;
            stalled = A.fixed_iters <= 0 && since >= 64 && err <= 50.f * tolm;
            // the next iterate from the Anderson history (warp 0; every thread passes the barrier)
            const float err_last = err_prev;
            auto aa_update = [&]() {
                if (!aa_on) return;
                if (wid == 0) anderson_step(S, nx, A.amax, A.aa_m, err, err_last, aC, aN);
                __syncthreads();
            };
            if (A.omega < 0.f && !aa_on) {
                if (om > 1.f && err > 1.5f * err_prev) {  // diverging: back to plain steps
                    om = 1.f;
                    om_start = it + 5;
                } else if (it == om_start) {
                    err_mark = err;
                } else if (it == om_start + 5 && err_mark > 0.f) {
                    const float r = fminf(powf(err / err_mark, 0.2f), 0.999f);
                    om = fminf(1.85f, fmaxf(1.f, 2.f / (1.f + sqrtf(1.f - r))));
                }
            }
            err_prev = err;
            if (lev > 0) {
                // coarse level: refine once its error is within eps_tol (or it
                // stalls), a <- log2 mu + f (a' - log2 mu) with the newest X dual,
                // tables at the finer scale, exact shifts on the next iteration
                if (err <= eps_tolm || stalled || it >= A.max_iter) {
                    // out of iterations: straight to the target eps (one last
                    // iteration there keeps the outputs consistent)
                    float f = A.eps_factor;
                    if (it >= A.max_iter) {
                        f = 1.f / lev_scale;
                        lev = 1;
                    }
                    --lev;
                    lev_scale *= f;
                    __syncthreads();  // every thread has read aN / the error partials
                    for (int u = tid; u < nx; u += NT)
                        aC[u] = S.lgm[u] > 0.5f * DD_NEG ? S.lgm[u] + f * (aN[u] - S.lgm[u]) : DD_NEG;
                    build_tables(S, A.k2d * (double)lev_scale, h, w, bs, hx, wx, uc1, uc2, vc1, vc2, l1, l2);
                    for (int q = tid; q < hx * bs; q += NT) S.T[q] = DD_NEG;
                    first = true;
                    best = 3.0e38f;
                    since = 0;
                    stalled = false;
                    if (tid == 0) S.ctl[8] = 0;  // Anderson history restarts at the new level
                    __syncthreads();
                    continue;
                }
                aa_update();
                float* tmp = aC;
                aC = aN;
                aN = tmp;
                continue;
            }
            const bool done = (A.fixed_iters > 0) ? (it >= A.fixed_iters)
                                                  : (err <= tolm || it >= A.max_iter || stalled);
            if (done) break;
            aa_update();
            float* tmp = aC;
            aC = aN;
            aN = tmp;
        }
        __syncthreads();  // every thread has read the error partials in S.red
        if (A.trace && tid == 0 && lead) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_loop1));
        if (A.fixed_iters <= 0 && err > tolm && tid == 0 && lead) atomicAdd(&A.status[stalled ? 3 : 0], 1);
        if constexpr (CL == 1)
            if (A.targ && nx == kMlpBlock) write_targets(A, S, J, aC, h, w, bs, hx, wx, gm[5], uc1, uc2, q11, q12, q22);

        // ---- outputs of the solve: duals, objective --------------------------
        float* apo = A.alpha + (long long)A.amax * J;
        double eloc[1] = {0.0};
        // exact displacement of the float origins for the gauge conversion (FP64,
        // computed once per cell with the gauge)
        const double dx1 = S.clx[9], dx2 = S.clx[10], hd = S.clx[11];
        for (int u = tid; u < (lead ? nx : 0); u += NT) {  // X side: one CTA
            apo[u] = aC[u];
            const float lg = S.lgm[u];
            if (lg > 0.5f * DD_NEG) {
                const int u1 = u / wx, u2 = u - u1 * wx;
                const double r = S.mux[u] * (double)exp2f(aC[u] - aN[u]);
                const double ub1 = u1 - (double)uc1, ub2 = u2 - (double)uc2;
                const double al = kLn2d * ((double)aC[u] - A.k2d * ((l1 - 1.0) * ub1 * ub1 + (l2 - 1.0) * ub2 * ub2)
                                           + 2.0 * A.k2d * (dx1 * ub1 + dx2 * ub2) + hd)
                                  - A.lnmu[(r0 + u1) * A.N2 + (c0 + u2)];
                eloc[0] += al * r;
            }
        }
        // Y side of the objective: per entry ln2 b~ nu_J - ln(nu) nu_J in FP32
        // (per-thread partials), the separable gauge terms of b through row and
        // column sums of nu_J with FP64 weights, and the constant hd |nu_J|.
        float ef = 0.f;
        for (int v = rlo * w + tid; v < rhi * w; v += NT) {  // Y side: the own rows
            const int v1 = v / w, v2 = v - v1 * w;
            const float bv = b_p[v1 * bs + v2];
            A.comp_b[comp + (long long)v1 * stride + v2] = bv;
            if (lgnu_p[v1 * bs + v2] > 0.5f * DD_NEG) {
                const float nuJ = A.comp_nu[comp + (long long)v1 * stride + v2];
                ef += nuJ * (kLn2 * bv - A.lnnuf[(o1 + v1) * A.N2 + (o2 + v2)]);
            }
        }
        eloc[0] += (double)ef;
        // rows: B1 and the axis-1 gauge terms; columns: B2 and the axis-2 ones
        // (1 / l from the gauge's shared values: no FP64 division per row)
        for (int v1 = rlo + tid; v1 < rhi; v1 += NT) {
            float rs = 0.f;
            for (int v2 = 0; v2 < w; ++v2) rs += A.comp_nu[comp + (long long)v1 * stride + v2];
            const double vb1 = v1 - (double)vc1;
            eloc[0] += kLn2d * (S.B1[v1] - A.k2d * (S.clx[12] - 1.0) * vb1 * vb1 - 2.0 * A.k2d * dx1 * vb1 + hd) * rs;
        }
        for (int v2 = tid; v2 < w; v2 += NT) {
            float cs = 0.f;
            for (int v1 = rlo; v1 < rhi; ++v1) cs += A.comp_nu[comp + (long long)v1 * stride + v2];
            const double vb2 = v2 - (double)vc2;
            eloc[0] += kLn2d * (S.B2[v2] - A.k2d * (S.clx[13] - 1.0) * vb2 * vb2 - 2.0 * A.k2d * dx2 * vb2) * cs;
        }
        block_sum_d<1>(eloc, S.red);
        if constexpr (CL > 1) cluster_sum_d<1>(eloc, S.clx, 8);
        if (tid == 0 && lead) {
            float* gg = A.gauge + 8 * J;
            gg[0] = d1; gg[1] = d2; gg[2] = l1; gg[3] = l2;
            gg[4] = uc1; gg[5] = uc2; gg[6] = vc1; gg[7] = vc2;
            A.iters[J] = it;
            if (A.trace) {
                unsigned long long t_end;
                unsigned smid;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
                asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
                long long* tr = A.trace + 8LL * J;
                tr[0] = (long long)t_start;
                tr[1] = (long long)t_end;
                tr[2] = (long long)smid;
                tr[3] = (long long)blockDim.x * CL;
                tr[4] = (long long)t_gather;
                tr[5] = (long long)t_loop0;
                tr[6] = (long long)t_loop1;
                tr[7] = 0;
            }
            A.err[J] = err;
            A.Ecell[J] = A.eps * eloc[0];
        }
        // DD_FLAG_FUSED_C2B: CompositeToBasic of this cell right away (one-CTA
        // solves), its arrays T2, M2 (and L, E) in the box arrays and stage-1
        // buffers of the solve, which are dead after the outputs above; k_c2b
        // takes the cells that do not fit
        if constexpr (CL == 1) {
            if (A.fused && c2b_cell_floats(A.s, hx, wx, h, w, A.pmom != nullptr) <= (long long)(S.tab1 - S.lgnu)) {
                __syncthreads();  // outputs and gauge written, partials read
                C2bSmem C;
                C.red = S.red;
                C.T = S.lgnu;
                C.tab1 = S.tab1;
                C.tab2 = S.tab2;
                C.L = S.lgnu + 2LL * (wx / A.s) * hx * w;
                C.E = C.L + (long long)h * wx;
                C.coef = S.coef;
                C.ctl = S.ctl;
                c2b_cell_fused(A, J, C, aC);
                if (tid == 0) {
                    A.fused[J] = 1;
                    if (A.trace) {
                        unsigned long long t_c2b;
                        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_c2b));
                        A.trace[8LL * J + 7] = (long long)t_c2b;
                    }
                }
            }
        }
    }
    if constexpr (CL > 1) cg::this_cluster().sync();  // no CTA leaves while others read its shared memory
}

// Input features of the warm-start network for every cell with a full 8 x 8
// X block (one CTA per cell, before the solve), in BF16, DD_MLP_NIN per cell:
//   [0, 64)    log2(mu on the block / its mean) / 4,
//   [64, 320)  nu_J resampled to 16 x 16 by exact area overlap (output row i
//              covers box rows [i h / 16, (i + 1) h / 16), likewise columns):
//              log2(value / mean + 1/256) / 4,
//   [320, 336) scalars of the cell's change of gauge (box extent, barycentre
//              offset d, stretch l, barycentres, log2 k2, spreads, the
//              correlation of nu_J).
// nu_J is gathered from the member boxes as in BasicToComposite.
__global__ void __launch_bounds__(128) k_feat(HalfArgs A, __nv_bfloat16* __restrict__ feat) {
    __shared__ float rs[256];
    __shared__ double red[32 * 12 + 12];
    const int J = blockIdx.x, tid = threadIdx.x, NT = blockDim.x;
    if (A.guard && *A.guard) return;
    const int32_t* xb = A.xblk + XB_N * J;
    const int r0 = xb[XB_R0], c0 = xb[XB_C0], hx = xb[XB_HX], wx = xb[XB_WX];
    if (hx * wx != kMlpBlock) return;
    const int32_t* ch = A.chdr + CH_N * J;
    const int o1 = ch[CH_O1], o2 = ch[CH_O2], h = ch[CH_H], w = ch[CH_W];
    for (int k = tid; k < 256; k += NT) rs[k] = 0.f;
    int32_t mem[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) mem[k] = A.members[4 * J + k];
    __syncthreads();
    double g[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) g[k] = 0.0;
    for (int v = tid; v < h * w; v += NT) {
        const int v1 = v / w, v2 = v - v1 * w;
        const int y1 = o1 + v1, y2 = o2 + v2;
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (mem[k] < 0) continue;
            const int32_t* bh = A.bhdr_in + BH_N * mem[k];
            const int p1 = y1 - bh[BH_O1], p2 = y2 - bh[BH_O2];
            if (p1 >= 0 && p1 < bh[BH_H] && p2 >= 0 && p2 < bh[BH_W])
                acc += A.pool_in[(long long)bh[BH_START] + (long long)p1 * bh[BH_STRIDE] + p2];
        }
        if (!(acc > 0.f)) continue;
        const double a = acc;
        g[0] += a; g[1] += a * v1; g[2] += a * v2; g[3] += a * v1 * v1; g[4] += a * v2 * v2; g[10] += a * v1 * v2;
        // output rows / columns overlapping this pixel, and the overlap lengths
        const int i0 = (16 * v1) / h, i1 = (16 * (v1 + 1) - 1) / h;
        const int j0 = (16 * v2) / w, j1 = (16 * (v2 + 1) - 1) / w;
        for (int i = i0; i <= i1; ++i) {
            const float ov1 = fminf((float)(v1 + 1), (float)((i + 1) * h) / 16.f) - fmaxf((float)v1, (float)(i * h) / 16.f);
            for (int j = j0; j <= j1; ++j) {
                const float ov2 =
                    fminf((float)(v2 + 1), (float)((j + 1) * w) / 16.f) - fmaxf((float)v2, (float)(j * w) / 16.f);
                atomicAdd(&rs[16 * i + j], acc * ov1 * ov2);
            }
        }
    }
    for (int u = tid; u < hx * wx; u += NT) {
        const int u1 = u / wx, u2 = u - u1 * wx;
        const double m = A.mu[(r0 + u1) * A.N2 + (c0 + u2)];
        g[5] += m; g[6] += m * u1; g[7] += m * u2; g[8] += m * u1 * u1; g[9] += m * u2 * u2; g[11] += m * u1 * u2;
    }
    block_sum_d<12>(g, red);
    __nv_bfloat16* out = feat + (long long)DD_MLP_NIN * J;
    for (int u = tid; u < hx * wx; u += NT) {
        const int u1 = u / wx, u2 = u - u1 * wx;
        out[u] = __float2bfloat16_rn((float)(0.25 * log2(A.mu[(r0 + u1) * A.N2 + (c0 + u2)] * 64.0 / g[5])));
    }
    for (int k = tid; k < 256; k += NT)
        out[64 + k] = __float2bfloat16_rn((float)(0.25 * log2(rs[k] * 256.0 / g[0] + 1.0 / 256.0)));
    if (tid == 0) {
        const double uc1 = g[6] / g[5], uc2 = g[7] / g[5], vc1 = g[1] / g[0], vc2 = g[2] / g[0];
        const double vu1 = fmax(g[8] / g[5] - uc1 * uc1, 0.0), vu2 = fmax(g[9] / g[5] - uc2 * uc2, 0.0);
        const double vv1 = fmax(g[3] / g[0] - vc1 * vc1, 0.0), vv2 = fmax(g[4] / g[0] - vc2 * vc2, 0.0);
        const double cv = g[10] / g[0] - vc1 * vc2;
        const double l1 = vu1 > 1e-3 ? fmin(8.0, fmax(0.125, sqrt(vv1 / vu1))) : 1.0;
        const double l2 = vu2 > 1e-3 ? fmin(8.0, fmax(0.125, sqrt(vv2 / vu2))) : 1.0;
        const double d1 = (r0 - o1) + uc1 - vc1, d2 = (c0 - o2) + uc2 - vc2;
        const double rho = (vv1 > 0.0 && vv2 > 0.0) ? cv / sqrt(vv1 * vv2) : 0.0;
        const double sc[16] = {h / 32.0, w / 32.0, d1 / 8.0, d2 / 8.0, log2(l1), log2(l2), (uc1 - 3.5) / 4.0,
                               (uc2 - 3.5) / 4.0, (vc1 + 0.5) / h - 0.5, (vc2 + 0.5) / w - 0.5, log2(A.k2d),
                               sqrt(vu1) / 4.0, sqrt(vu2) / 4.0, sqrt(vv1) / 16.0, sqrt(vv2) / 16.0, rho};
        for (int k = 0; k < 16; ++k) out[320 + k] = __float2bfloat16_rn((float)sc[k]);
    }
}

// Graph mode: the size class and the processing order of every cell, on the
// device (one CTA). Two classes: 1 small boxes (area and sides within the tuned
// small-class limits), 0 all others, in one launch: boxes within the captured
// shared-memory capacity (a0, h0, w0) keep their arrays in shared memory, the
// rest in global scratch (offsets taken here). Within a class the order is
// longest expected solve first, by buckets of log2(box area x previous
// iteration count). Any box beyond what the captured launch holds, and
// composite / output pools beyond their capacity, set the guard to `stage`:
// every later kernel of the iteration then does nothing and the host redoes
// the iteration from that stage without the graph.
struct ClassCaps {
    long long a0, h0, w0, h2, w2, gscr, comp, pool, sa, ss;
    int cl_cap;          // most cells solved by clusters (0: none)
    long long cl_area;   // smallest box area h * w solved by a cluster
};

// Device classification of the cells of a half-iteration for the captured graph:
// class 1 small boxes, class 0 large boxes (global-scratch offsets for those
// beyond the shared-memory capacity), class 2 the largest-work cells solved by
// thread-block clusters. Work key = h w max(1, previous iterations); the cluster
// class takes whole quarter-octave key buckets from the top, and from the
// bucket that would exceed cl_cap its first cells in index order, cl_cap cells
// in all (dd_api.cu applies the same rule on the host). Each
// list is ordered by descending quarter-octave of the key (longest expected
// solves first).
__global__ void __launch_bounds__(1024) k_classify(int ncell, const int32_t* __restrict__ chdr,
                                                   const int32_t* __restrict__ iters, ClassCaps cc,
                                                   int32_t* __restrict__ corder, int* __restrict__ ccount,
                                                   long long* __restrict__ goff, const long long* __restrict__ tot,
                                                   int* __restrict__ guard, int stage) {
    constexpr int NFB = 192;  // quarter-octave buckets of the work key
    __shared__ int cnt[2][NFB];
    __shared__ int offs[2][NFB];
    __shared__ int cntf[NFB];
    __shared__ int bstar, clpos, fpart, npart, prank;
    __shared__ int wsum[32];
    __shared__ unsigned long long gsum;
    __shared__ int bad;
    const int tid = threadIdx.x, T = blockDim.x;
    for (int k = tid; k < 2 * NFB; k += T) (&cnt[0][0])[k] = 0;
    for (int k = tid; k < NFB; k += T) cntf[k] = 0;
    if (tid == 0) {
        gsum = 0;
        clpos = 0;
        prank = 0;
        bad = (tot[PT_COMP] > cc.comp || tot[PT_OUT] > cc.pool) ? 1 : 0;
    }
    __syncthreads();
    // cls: 0 large, 1 small; fb: quarter octave of the key (list order); el: may be clustered
    auto classify = [&](int J, int& cls, int& bk, int& fb, bool& el) {
        const int h = chdr[CH_N * J + CH_H], w = chdr[CH_N * J + CH_W];
        const long long a = (long long)h * padw(w);
        cls = (a <= cc.sa && w <= cc.ss && h <= cc.ss) ? 1 : 0;
        const long long key = (long long)h * w * max(1, iters[J]);
        cluster_key_bucket(key, bk, fb);
        el = cls == 0 && cc.cl_cap > 0 && (long long)h * w >= cc.cl_area;
    };
    for (int J = tid; J < ncell; J += T) {
        int cls, bk, fb;
        bool el;
        classify(J, cls, bk, fb, el);
        if (el)
            atomicAdd(&cntf[fb], 1);
        else
            atomicAdd(&cnt[cls][fb], 1);
        const int h = chdr[CH_N * J + CH_H], w = chdr[CH_N * J + CH_W];
        const long long a = (long long)h * padw(w);
        if (cls == 0 && !(a <= cc.a0 && h <= cc.h0 && w <= cc.w0)) {
            if (h > cc.h2 || w > cc.w2) atomicExch(&bad, 1);
            goff[J] = (long long)atomicAdd(&gsum, (unsigned long long)(2LL * h * padw(w)));
        } else {
            goff[J] = -1;
        }
    }
    __syncthreads();
    if (tid == 0) {
        if ((long long)gsum > cc.gscr) bad = 1;
        // whole buckets from the top, then the first cells (ascending index) of
        // the bucket that would overflow the cap
        int cum = 0, bs_ = NFB, fp = -1, np_ = 0;
        for (int f = NFB - 1; f >= 0; --f) {
            if (cntf[f] == 0) continue;
            if (cum + cntf[f] > cc.cl_cap) {
                fp = f;
                np_ = cc.cl_cap - cum;
                break;
            }
            cum += cntf[f];
            bs_ = f;
        }
        bstar = bs_;
        fpart = fp;
        npart = np_;
        for (int f = 0; f < bs_; ++f) cnt[0][f] += cntf[f] - (f == fp ? np_ : 0);
        cum += np_;
        for (int c = 0; c < 2; ++c) {
            int run = 0;
            for (int b = NFB - 1; b >= 0; --b) {  // descending keys
                offs[c][b] = run;
                run += cnt[c][b];
            }
            ccount[c] = run;
        }
        ccount[2] = cum;
        if (bad) atomicCAS(guard, 0, stage);
    }
    __syncthreads();
    // chunks of T cells in ascending index order: a block scan ranks the cells
    // of the partial bucket
    for (int base = 0; base < ncell; base += T) {
        const int J = base + tid;
        int cls = 1, bk = 0, fb = 0;
        bool el = false;
        if (J < ncell) classify(J, cls, bk, fb, el);
        const bool inpart = J < ncell && el && fb == fpart;
        const unsigned bal = __ballot_sync(0xffffffffu, inpart);
        const int lane = tid & 31, wid = tid >> 5;
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        int before = prank;
        for (int k = 0; k < wid; ++k) before += wsum[k];
        const int rank = before + __popc(bal & ((1u << lane) - 1u));
        if (J < ncell) {
            if (el && (fb >= bstar || (inpart && rank < npart))) {
                corder[2LL * ncell + atomicAdd(&clpos, 1)] = J;
            } else {
                const int pos = atomicAdd(&offs[cls][fb], 1);
                corder[(long long)cls * ncell + pos] = J;
            }
        }
        __syncthreads();
        if (tid == 0)
            for (int k = 0; k < (T >> 5); ++k) prank += wsum[k];
        __syncthreads();
    }
}

// rows of the cells in `idx` (features, targets) into packed caller buffers
__global__ void k_collect(int n, const int32_t* __restrict__ idx, const uint4* __restrict__ fsrc,
                          const uint4* __restrict__ tsrc, uint4* __restrict__ fdst, uint4* __restrict__ tdst) {
    constexpr int FQ = DD_MLP_NIN * 2 / 16, TQ = DD_MLP_NOUT * 4 / 16;
    const int r = blockIdx.x;
    if (r >= n) return;
    const long long J = idx[r];
    for (int q = threadIdx.x; q < FQ; q += blockDim.x) fdst[(long long)r * FQ + q] = fsrc[J * FQ + q];
    for (int q = threadIdx.x; q < TQ; q += blockDim.x) tdst[(long long)r * TQ + q] = tsrc[J * TQ + q];
}

// CompositeToBasic, D_i, balancing, truncation and compaction of one composite
// cell per CTA, from the duals k_sink left in global memory (alpha, b~ not
// needed: the member shares are ratios of partial sums over X).
constexpr int kC2bThreads = 256;  // k_c2b CTA size (3 per SM: 80 registers)
constexpr int kC2bBatch = 8;      // compaction strides per barrier pair

// CompositeToBasic, D_i, balancing, truncation and compaction of composite cell
// J by all threads of the calling CTA, from its X dual aC (shared memory) and
// the change of gauge of its solve (A.gauge, read after a block barrier). The
// member shares are ratios of partial sums over X, so the Y dual is not needed.
// Every return is uniform over the CTA.
__device__ __forceinline__ void c2b_cell(const HalfArgs& A, int J, const C2bSmem& S, const float* aC) {
    const int tid = threadIdx.x, NT = blockDim.x;
    const int s = A.s;
    const int32_t* xb = A.xblk + XB_N * J;
    const int r0 = xb[XB_R0], c0 = xb[XB_C0], hx = xb[XB_HX], wx = xb[XB_WX], nmem = xb[XB_NMEM];
    const int32_t* ch = A.chdr + CH_N * J;
    const int o1 = ch[CH_O1], o2 = ch[CH_O2], h = ch[CH_H], w = ch[CH_W], stride = ch[CH_STRIDE];
    const long long comp = ((long long)ch[CH_COMP_HI] << 32) | (unsigned int)ch[CH_COMP_LO];
    const long long slot0 = ch[CH_OUT_SLOT];
    const long long area = (long long)h * stride;
    const int nx = hx * wx, nA = h * w;
    const int bs = padw(w);
    if (nA == 0) return;  // handled (empty outputs) by k_sink
    if (comp + area > A.comp_cap || slot0 + nmem * area > A.out_cap || (A.pre && slot0 + nmem * area > A.pre_cap)) {
        if (tid == 0) atomicAdd(&A.status[4], 1);
        return;
    }
    int32_t mem[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) mem[k] = A.members[4 * J + k];
    // the change of gauge of this cell's solve, and its kernel tables
    const float* gg = A.gauge + 8 * J;
    const float l1 = gg[2], l2 = gg[3], uc1 = gg[4], uc2 = gg[5], vc1 = gg[6], vc2 = gg[7];
    // 1 / l as in the solve's tables (one FP64 division per cell, not per entry)
    if (tid == 0) {
        S.red[0] = 1.0 / (double)l1;
        S.red[1] = 1.0 / (double)l2;
    }
    __syncthreads();
    const double il1 = S.red[0], il2 = S.red[1];
    for (int v1 = tid; v1 < h; v1 += NT) {
        const double tt = (v1 - (double)vc1) * il1;
        const int us = min(hx - 1, max(0, (int)rint(tt + (double)uc1)));
        const double w0 = 2.0 * ((us - (double)uc1) - tt);
        const float w0f = (float)w0, kl = (float)(A.k2d * l1);
        for (int u1 = 0; u1 < hx; ++u1) {
            const float D = (float)(u1 - us);
            S.tab1[u1 * h + v1] = kl * D * (D + w0f);
        }
    }
    for (int v2 = tid; v2 < w; v2 += NT) {
        const double tt = (v2 - (double)vc2) * il2;
        const int us = min(wx - 1, max(0, (int)rint(tt + (double)uc2)));
        const double w0 = 2.0 * ((us - (double)uc2) - tt);
        const float w0f = (float)w0, kl = (float)(A.k2d * l2);
        for (int u2 = 0; u2 < wx; ++u2) {
            const float D = (float)(u2 - us);
            S.tab2[u2 * bs + v2] = kl * D * (D + w0f);
        }
    }
    __syncthreads();

    // ---- per-pixel moments of the cell plan (gluing candidates) ------------
    // pi(u, v) = 2^(a(u) + b~(v) - tab1(u1, v1) - tab2(u2, v2)) for the returned
    // pair (its Y-marginal is nu_J). For every pixel u of the block: the mass
    // r(u) = sum_v pi(u, v) and the mean displacement d(u) = E[y | u] - x(u),
    // separable like the X-update: per (v1, u2) the row sum over v2 and the mean
    // of v2 under it, then per u the sum over v1.
    if (A.pmom) {
        for (int q = tid; q < h * wx; q += NT) {
            const int v1 = q / wx, u2 = q - v1 * wx;
            const float* br = A.comp_b + comp + (long long)v1 * stride;
            const float* tb = S.tab2 + u2 * bs;
            float mx = DD_NEG;
            for (int v2 = 0; v2 < w; ++v2)
                if (br[v2] > 0.5f * DD_NEG) mx = fmaxf(mx, br[v2] - tb[v2]);
            float t0 = 0.f, t1 = 0.f;
            if (mx > 0.5f * DD_NEG)
                for (int v2 = 0; v2 < w; ++v2)
                    if (br[v2] > 0.5f * DD_NEG) {
                        const float e = ex2f(br[v2] - tb[v2] - mx);
                        t0 += e;
                        t1 += e * (float)v2;
                    }
            S.L[q] = t0 > 0.f ? mx + lg2f(t0) : DD_NEG;
            S.E[q] = t0 > 0.f ? t1 / t0 : 0.f;
        }
        __syncthreads();
        for (int u = tid; u < nx; u += NT) {
            const int u1 = u / wx, u2 = u - u1 * wx;
            const float* tb = S.tab1 + u1 * h;
            float mx = DD_NEG;
            for (int v1 = 0; v1 < h; ++v1)
                if (S.L[v1 * wx + u2] > 0.5f * DD_NEG) mx = fmaxf(mx, S.L[v1 * wx + u2] - tb[v1]);
            float t0 = 0.f, t1 = 0.f, t2 = 0.f;
            if (mx > 0.5f * DD_NEG)
                for (int v1 = 0; v1 < h; ++v1) {
                    const float Lv = S.L[v1 * wx + u2];
                    if (!(Lv > 0.5f * DD_NEG)) continue;
                    const float e = ex2f(Lv - tb[v1] - mx);
                    t0 += e;
                    t1 += e * (float)v1;
                    t2 += e * S.E[v1 * wx + u2];
                }
            const bool live = aC[u] > 0.5f * DD_NEG && t0 > 0.f;
            const double r = live ? exp2((double)aC[u] + (double)mx + (double)lg2f(t0)) : 0.0;
            const double e1 = live ? (double)(t1 / t0) : 0.0, e2 = live ? (double)(t2 / t0) : 0.0;
            const int rg = u1 / s, cg = u2 / s, k = rg * (wx / s) + cg;
            if (k >= nmem) continue;
            const int q = (u1 - rg * s) * s + (u2 - cg * s);
            double* pm = A.pmom + ((long long)mem[k] * s * s + q) * 3;
            pm[0] = r;
            pm[1] = live ? (double)(o1 - r0) + e1 - (double)u1 : 0.0;
            pm[2] = live ? (double)(o2 - c0) + e2 - (double)u2 : 0.0;
        }
    }

    // ---- 3. CompositeToBasic with D_i -----------------------------------
    // C1: per column group cg, T2(cg, u1, v2) = LSE over u2 in the group, and
    //     M2 = mean of (x2 - y2)^2 under that partial distribution.
    const int ncg = wx / s, nrg = hx / s;
    float* T2 = S.T;
    float* M2 = S.T + (long long)ncg * hx * w;
    for (int q = tid; q < ncg * hx * w; q += NT) {
        const int cg = q / (hx * w), rem = q - cg * hx * w;
        const int u1 = rem / w, v2 = rem - u1 * w;
        const float* ar = aC + u1 * wx + cg * s;
        const float* tb = S.tab2 + (cg * s) * bs + v2;
        const float lse = lse2(s, [&](int k) { return ar[k] - tb[k * bs]; });
        float mom = 0.f;
        for (int k = 0; k < s; ++k) {
            const float dd = (float)(c0 + cg * s + k - o2 - v2);
            mom += ex2f(ar[k] - tb[k * bs] - lse) * dd * dd;
        }
        T2[q] = lse;
        M2[q] = mom;
    }
    __syncthreads();
    // C2: each member's share of the column mass, as a ratio of partial sums
    // with one common shift, so that sum_i nu_i(v) = nu_J(v) up to FP32
    // rounding whatever the size of the log-domain values:
    //   nu_i(v) = nu_J(v) * sum_{u in X_i} pi(u, v) / sum_u pi(u, v),
    // and the mean squared displacement E_i(v) under pi(., v) restricted to X_i.
    float accm[4] = {0.f, 0.f, 0.f, 0.f}, accd[4] = {0.f, 0.f, 0.f, 0.f};
    // nu_J of the thread's next entry is loaded one entry ahead (its latency
    // overlaps the shared-memory work of the current one)
    auto nu_at = [&](int v) {
        const int v1 = v / w;
        return v < nA ? A.comp_nu[comp + (long long)v1 * stride + (v - v1 * w)] : 0.f;
    };
    float nuv_next = nu_at(tid);
    for (int v = tid; v < nA; v += NT) {
        const int v1 = v / w, v2 = v - v1 * w;
        const float* tb = S.tab1 + v1;
        const float nuv = nuv_next;
        nuv_next = nu_at(v + NT);
        float num[4] = {0.f, 0.f, 0.f, 0.f}, ew[4] = {0.f, 0.f, 0.f, 0.f};  // ew: sum_u pi(u, v) E_i(v)
        if (nuv > 0.f) {
            float mx = DD_NEG;
            for (int cg = 0; cg < ncg; ++cg)
                for (int u1 = 0; u1 < hx; ++u1) mx = fmaxf(mx, T2[(cg * hx + u1) * w + v2] - tb[u1 * h]);
            float den = 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k >= nmem) break;
                const int rg = k / ncg, cg = k - rg * ncg;
                const float* Tc = T2 + cg * hx * w + v2;
                const float* Mc = M2 + cg * hx * w + v2;
                float nk = 0.f, ek = 0.f;
                for (int kk = 0; kk < s; ++kk) {
                    const int u1 = rg * s + kk;
                    const float wt = ex2f(Tc[u1 * w] - tb[u1 * h] - mx);
                    const float dd = (float)(r0 + u1 - o1 - v1);
                    nk += wt;
                    ek += wt * (dd * dd + Mc[u1 * w]);
                }
                num[k] = nk;
                ew[k] = ek;
                den += nk;
            }
            const float sc = den > 0.f ? nuv / den : 0.f;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                num[k] *= sc;
                ew[k] *= sc;  // nu_i(v) E_i(v), without dividing by the member's share
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k >= nmem) break;
            A.pool_out[slot0 + k * area + (long long)v1 * stride + v2] = num[k];
            accm[k] += num[k];
            accd[k] += ew[k];
        }
    }
    float red8f[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) { red8f[k] = accm[k]; red8f[4 + k] = accd[k]; }
    double red8[8];
    block_sum_f<8>(red8f, red8, S.red);
    (void)nrg;

    // ---- 4. balancing coefficients (member order walk) -------------------
    if (tid == 0) {
        double mass[4], e[4];
        for (int k = 0; k < 4; ++k) {
            mass[k] = red8[k];
            e[k] = (k < nmem) ? mass[k] - A.m[mem[k]] : 0.0;
        }
        double cf[4][4];
        for (int j = 0; j < 4; ++j)
            for (int k = 0; k < 4; ++k) cf[j][k] = (j == k) ? 1.0 : 0.0;
        int pos[4], neg[4], np = 0, nn = 0;
        for (int k = 0; k < nmem; ++k) {
            if (e[k] > 0.0) pos[np++] = k;
            else if (e[k] < 0.0) neg[nn++] = k;
        }
        int p = 0, q = 0;
        double rp = np ? e[pos[0]] : 0.0, rq = nn ? -e[neg[0]] : 0.0;
        while (p < np && q < nn) {
            const int i = pos[p], j = neg[q];
            const double d = fmin(rp, rq);
            const double f = d / mass[i];
            cf[i][i] -= f;
            cf[j][i] += f;
            rp -= d;
            rq -= d;
            if (rp <= 0.0) { ++p; rp = p < np ? e[pos[p]] : 0.0; }
            if (rq <= 0.0) { ++q; rq = q < nn ? -e[neg[q]] : 0.0; }
        }
        for (int j = 0; j < 4; ++j)
            for (int k = 0; k < 4; ++k) S.coef[4 * j + k] = (float)cf[j][k];
        for (int k = 0; k < nmem; ++k) {
            double* bm = A.bmom + BM_N * mem[k];
            bm[BM_D] = A.h2 * red8[4 + k];
            bm[BM_PREMASS] = mass[k];
        }
        for (int k = 0; k < 16; ++k) S.ctl[4 + k] = 0;
        for (int k = 0; k < 4; ++k) {
            S.ctl[4 + 4 * k + 0] = INT32_MAX;  // min row
            S.ctl[4 + 4 * k + 1] = -1;         // max row
            S.ctl[4 + 4 * k + 2] = INT32_MAX;  // min col
            S.ctl[4 + 4 * k + 3] = -1;         // max col
        }
    }
    __syncthreads();

    // ---- 5. apply balancing, truncate, box and moments -------------------
    const double bc1 = 0.5 * (h - 1), bc2 = 0.5 * (w - 1);
    float cf[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k) cf[j][k] = S.coef[4 * j + k];
    int bb[4][4];
    float momf[16];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        bb[k][0] = INT32_MAX; bb[k][1] = -1; bb[k][2] = INT32_MAX; bb[k][3] = -1;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) momf[k] = 0.f;
    // the member values of four entries of the thread are loaded together (an
    // entry's values are only read and written by its own thread)
    constexpr int U5 = 2;
    for (int v0 = tid; v0 < nA; v0 += U5 * NT) {
        float vals[U5][4];
#pragma unroll
        for (int u = 0; u < U5; ++u) {
            const int v = v0 + u * NT, v1 = v / w;
            const long long off = slot0 + (long long)v1 * stride + (v - v1 * w);
#pragma unroll
            for (int k = 0; k < 4; ++k) vals[u][k] = (v < nA && k < nmem) ? A.pool_out[off + k * area] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U5; ++u) {
            const int v = v0 + u * NT;
            if (v >= nA) break;
            const int v1 = v / w, v2 = v - v1 * w;
            const long long off = slot0 + (long long)v1 * stride + v2;
            if (A.pre) {
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    if (k < nmem) A.pre[off + k * area] = vals[u][k];
            }
            const float y1 = (float)(v1 - bc1), y2 = (float)(v2 - bc2);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (j >= nmem) break;
                float nv = 0.f;
#pragma unroll
                for (int k = 0; k < 4; ++k) nv += cf[j][k] * vals[u][k];
                if (!(nv >= A.trunc)) nv = 0.f;
                A.pool_out[off + j * area] = nv;
                if (nv > 0.f) {
                    bb[j][0] = min(bb[j][0], v1); bb[j][1] = max(bb[j][1], v1);
                    bb[j][2] = min(bb[j][2], v2); bb[j][3] = max(bb[j][3], v2);
                    momf[4 * j + 0] += nv;
                    momf[4 * j + 1] += nv * y1;
                    momf[4 * j + 2] += nv * y2;
                    momf[4 * j + 3] += nv * (y1 * y1 + y2 * y2);
                }
            }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (k >= nmem) break;
        atomicMin(&S.ctl[4 + 4 * k + 0], bb[k][0]);
        atomicMax(&S.ctl[4 + 4 * k + 1], bb[k][1]);
        atomicMin(&S.ctl[4 + 4 * k + 2], bb[k][2]);
        atomicMax(&S.ctl[4 + 4 * k + 3], bb[k][3]);
    }
    double mom[16];
    block_sum_f<16>(momf, mom, S.red);  // contains __syncthreads

    // ---- compaction in place (dst index never exceeds src index) --------
    // Each member is rescaled to its basic mass m_i after truncation, so that
    // the removed entries do not leave later cell problems unbalanced. Thread k
    // does member k's scale, header and moments; then one pass compacts all
    // members (their slot regions are disjoint).
    if (tid < nmem) {
        const int k = tid;
        const int rlo = S.ctl[4 + 4 * k + 0], rhi = S.ctl[4 + 4 * k + 1];
        const int clo = S.ctl[4 + 4 * k + 2], chi = S.ctl[4 + 4 * k + 3];
        const bool empty = rhi < 0;
        const int hh = empty ? 0 : rhi - rlo + 1, ww = empty ? 0 : chi - clo + 1;
        const int i = mem[k];
        const double ms = mom[4 * k + 0], mi = A.m[i];
        S.coef[k] = ms > 0.0 ? (float)(mi / ms) : 1.f;
        int32_t* bo = A.bhdr_out + BH_N * i;
        bo[BH_O1] = empty ? 0 : o1 + rlo;
        bo[BH_O2] = empty ? 0 : o2 + clo;
        bo[BH_H] = hh;
        bo[BH_W] = ww;
        bo[BH_STRIDE] = (ww + 3) & ~3;
        bo[BH_START] = (int32_t)(slot0 + k * area);
        double* bm = A.bmom + BM_N * i;
        const double m1 = ms > 0 ? mom[4 * k + 1] / ms : 0.0, m2 = ms > 0 ? mom[4 * k + 2] / ms : 0.0;
        bm[BM_MASS] = ms > 0 ? mi : 0.0;
        bm[BM_Y1] = o1 + bc1 + m1;
        bm[BM_Y2] = o2 + bc2 + m2;
        bm[BM_VAR] = ms > 0 ? mom[4 * k + 3] / ms - m1 * m1 - m2 * m2 : 0.0;
    }
    __syncthreads();
    int nk[4], pre[5], rlo[4], clo[4], wk[4], stk[4];
    float fsc[4];
    pre[0] = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const bool live = k < nmem && S.ctl[4 + 4 * k + 1] >= 0;
        rlo[k] = S.ctl[4 + 4 * k + 0];
        clo[k] = S.ctl[4 + 4 * k + 2];
        const int hh = live ? S.ctl[4 + 4 * k + 1] - rlo[k] + 1 : 0;
        wk[k] = live ? S.ctl[4 + 4 * k + 3] - clo[k] + 1 : 0;
        stk[k] = (wk[k] + 3) & ~3;
        nk[k] = hh * stk[k];
        fsc[k] = k < nmem ? S.coef[k] : 1.f;
        pre[k + 1] = pre[k] + nk[k];
    }
    const int ntot = pre[4];
    // kC2bBatch strides of NT entries per barrier pair: every read of a batch
    // precedes its writes, and later batches read only beyond a member's last write
    for (int base = 0; base < ntot; base += kC2bBatch * NT) {
        float val[kC2bBatch];
        int kd[kC2bBatch];
#pragma unroll
        for (int j = 0; j < kC2bBatch; ++j) {
            const int dI = base + j * NT + tid;
            val[j] = 0.f;
            kd[j] = -1;
            if (dI < ntot) {
                const int k = (dI >= pre[1]) + (dI >= pre[2]) + (dI >= pre[3]);
                int p0 = pre[0], st = stk[0], wwk = wk[0], r0k = rlo[0], c0k = clo[0];
                float f = fsc[0];
#pragma unroll
                for (int t = 1; t < 4; ++t)
                    if (k == t) { p0 = pre[t]; st = stk[t]; wwk = wk[t]; r0k = rlo[t]; c0k = clo[t]; f = fsc[t]; }
                const int d = dI - p0, rr = d / st, cc = d - rr * st;
                const float* sl = A.pool_out + slot0 + (long long)k * area;
                if (cc < wwk) val[j] = sl[(long long)(r0k + rr) * stride + c0k + cc] * f;
                kd[j] = k;
            }
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kC2bBatch; ++j) {
            const int dI = base + j * NT + tid;
            if (kd[j] < 0) continue;
            int p0 = pre[0];
#pragma unroll
            for (int t = 1; t < 4; ++t)
                if (kd[j] == t) p0 = pre[t];
            A.pool_out[slot0 + (long long)kd[j] * area + (dI - p0)] = val[j];
        }
        __syncthreads();
    }
}

// the solving CTA's call (k_sink with A.fused): not inlined, so that the
// solver's register allocation does not carry CompositeToBasic's
__device__ __noinline__ void c2b_cell_fused(const HalfArgs& A, int J, const C2bSmem& S, const float* aC) {
    c2b_cell(A, J, C2bSmem(S), aC);
}

__global__ void __launch_bounds__(kC2bThreads, 3) k_c2b(HalfArgs A) {
    extern __shared__ __align__(16) char smem_raw[];
    int J = blockIdx.x;  // cells with the most work first, where an order is given
    if (A.c2b_order) {
        if (A.c2b_count) {
            const int b = blockIdx.x, n2 = A.c2b_count[2], n0 = A.c2b_count[0];
            J = b < n2 ? A.c2b_order[2LL * A.ncell + b]
                       : (b - n2 < n0 ? A.c2b_order[b - n2] : A.c2b_order[(long long)A.ncell + (b - n2 - n0)]);
        } else {
            J = A.c2b_order[blockIdx.x];
        }
    }
    // cells whose solving CTA already did this (k_sink with A.fused): clear the
    // mark for the next half-iteration and leave
    if (A.fused) {
        const int done = A.fused[J];
        __syncthreads();  // every thread has read the mark before it is cleared
        if (done) {
            if (threadIdx.x == 0) A.fused[J] = 0;
            return;
        }
    }
    if (A.guard && *A.guard) return;
    const int tid = threadIdx.x;
    // shared memory
    const int s = A.s, s2 = 2 * s, BS = padw(A.smaxW);
    double* dsm = reinterpret_cast<double*>(smem_raw);
    struct {
        double* red;
        float* T;
        float* tab1;
        float* tab2;
        float* a;
        float* L;  // gluing candidates: per (v1, u2) log2 of the row sum over v2, and
        float* E;  // the mean of v2 under it (h x 2s each)
        float* coef;
        int* ctl;
    } S;
    S.red = dsm;
    float* f = reinterpret_cast<float*>(dsm + 32 * 16 + 16);
    S.T = f; f += 4 * s2 * BS;
    S.tab1 = f; f += A.smaxH * s2;
    S.tab2 = f; f += BS * s2;
    S.a = f; f += A.amax;
    S.L = f; f += A.pmom ? A.smaxH * s2 : 0;
    S.E = f; f += A.pmom ? A.smaxH * s2 : 0;
    S.coef = f; f += 16;
    S.ctl = reinterpret_cast<int*>(f);
    if (reinterpret_cast<char*>(f + 32) - smem_raw > (long long)dyn_smem_bytes()) {
        if (tid == 0) atomicAdd(&A.status[2], 1);
        return;
    }
    const int32_t* xb = A.xblk + XB_N * J;
    const int nx = xb[XB_HX] * xb[XB_WX];
    const float* ap = A.alpha + (long long)A.amax * J;
    for (int u = tid; u < nx; u += blockDim.x) S.a[u] = ap[u];
    C2bSmem C;
    C.red = S.red; C.T = S.T; C.tab1 = S.tab1; C.tab2 = S.tab2; C.L = S.L; C.E = S.E; C.coef = S.coef; C.ctl = S.ctl;
    c2b_cell(A, J, C, S.a);
}

}  // namespace

size_t half_smem_bytes(dd_ctx* c, long long maxarea, long long maxh, long long maxw) {
    const size_t s2 = 2 * c->s, BS = (size_t)padw((int)maxw);
    maxarea = (maxarea + 3) & ~3LL;  // as in carve()
    size_t bytes = sizeof(double) * ((size_t)c->amax + 32 * 16 + 16 + (size_t)maxh + BS + 16) + 16;
    size_t fl = 2 * (size_t)maxarea + s2 * BS + 2 * (size_t)maxh * s2 + BS * s2 + 12 * (size_t)c->amax + 16 + 32 +
                (size_t)aa_floats(c->opt.fixed_iters > 0 ? 0 : c->opt.anderson, c->amax);
    return bytes + sizeof(float) * fl;
}

size_t c2b_smem_bytes(dd_ctx* c, long long maxh, long long maxw) {
    const size_t s2 = 2 * c->s, BS = (size_t)padw((int)maxw);
    size_t fl = 4 * s2 * BS + (size_t)maxh * s2 + BS * s2 + (size_t)c->amax + 16 + 32 +
                (c->opt.eps_gamma > 0.0 ? 2 * (size_t)maxh * s2 : 0);
    return sizeof(double) * (32 * 16 + 16) + sizeof(float) * fl;
}

namespace {
// deterministic block sum (fixed thread-to-element assignment and tree order)
__device__ double block_sum_fixed(double x, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[wid] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < nw; ++k) t += sh[k];
        sh[32] = t;
    }
    __syncthreads();
    const double r = sh[32];
    __syncthreads();
    return r;
}

// Stop budgets of the next solves (one CTA): b_J = tol ((1 - s) mu(X_J) + s mbar) w_J
// rescaled so that sum_J b_J = tol mu(X), with w_J = (it_J / mean it)^gamma from
// the previous iteration counts (w = 1 without them or for gamma = 0).
__global__ void __launch_bounds__(1024) k_budget(int ncell, const double* __restrict__ mJ,
                                                 const int32_t* __restrict__ iters, int use_iters, double tol,
                                                 double share, double mbar, double gamma,
                                                 double* __restrict__ budget) {
    __shared__ double sh[33];
    const int tid = threadIdx.x, T = blockDim.x;
    const bool weigh = use_iters && gamma > 0.0;
    double si = 0.0, sm = 0.0;
    for (int J = tid; J < ncell; J += T) {
        if (weigh) si += (double)max(1, iters[J]);
        sm += mJ[J];
    }
    const double mean_it = weigh ? block_sum_fixed(si, sh) / max(1, ncell) : 1.0;
    const double mtot = block_sum_fixed(sm, sh);
    // the weights are a heuristic: FP32 (an FP64 pow per cell on one SM took
    // ~70 us at GB300's FP64 rate); their sum and the rescale stay FP64, so the
    // budgets still add up to tol mu(X)
    const float inv_mean = (float)(1.0 / mean_it), gf = (float)gamma;
    double sw = 0.0;
    for (int J = tid; J < ncell; J += T) {
        double wj = (1.0 - share) * mJ[J] + share * mbar;
        if (weigh) {
            const float r = (float)max(1, iters[J]) * inv_mean;
            wj *= (double)(gf == 1.f ? r : exp2f(gf * __log2f(r)));
        }
        budget[J] = wj;
        sw += wj;
    }
    const double wsum = block_sum_fixed(sw, sh);
    const double scale = wsum > 0.0 ? tol * mtot / wsum : 0.0;
    for (int J = tid; J < ncell; J += T) budget[J] *= scale;
}

// a <- log2 mu + f (a - log2 mu) for the stored X duals of every cell (eps change)
__global__ void k_rescale_alpha(int ncell, int amax, int N2, const int32_t* __restrict__ xblk,
                                const float* __restrict__ lgmu, float* __restrict__ alpha, float f) {
    const int J = blockIdx.x;
    if (J >= ncell) return;
    const int32_t* xb = xblk + XB_N * J;
    const int r0 = xb[XB_R0], c0 = xb[XB_C0], hx = xb[XB_HX], wx = xb[XB_WX];
    for (int u = threadIdx.x; u < hx * wx && u < amax; u += blockDim.x) {
        const int u1 = u / wx, u2 = u - u1 * wx;
        const float lg = lgmu[(long long)(r0 + u1) * N2 + (c0 + u2)];
        float* a = alpha + (long long)amax * J + u;
        if (lg > 0.5f * DD_NEG) *a = lg + f * (*a - lg);
    }
}

}  // namespace

int launch_budget(dd_ctx* c, int part, cudaStream_t st) {
    const DevPart& P = c->part[part];
    if (P.ncell <= 0) return DD_OK;
    k_budget<<<1, 1024, 0, st ? st : c->stream>>>(P.ncell, P.mJ, P.iters, P.warm_valid ? 1 : 0, c->opt.tol, c->opt.tol_share,
                                        P.mbar, c->opt.tol_gamma, P.budget);
    return launch_status(__func__);
}

int launch_rescale_alpha(dd_ctx* c, int part, double f) {
    const DevPart& P = c->part[part];
    if (P.ncell <= 0) return DD_OK;
    k_rescale_alpha<<<P.ncell, 64, 0, c->stream>>>(P.ncell, c->amax, c->N2, P.xblk, c->d_lgmu, P.alpha, (float)f);
    return launch_status(__func__);
}

int half_kernel_max_smem() { return 227 * 1024; }

int launch_plan_half(dd_ctx* c, int part) {
    DevPart& P = c->part[part];
    k_plan_half<<<1, 1024, 0, c->stream>>>(P.ncell, P.members, c->bhdr[c->cur], P.chdr, P.xblk, c->d_tot);
    return launch_status(__func__);
}

int half_padw(int w) { return padw(w); }

namespace {
bool g_attr_set = false;

int set_attrs() {
    if (g_attr_set) return DD_OK;
    const int mx = half_kernel_max_smem();
    if (cudaFuncSetAttribute(k_sink<64, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
        cudaFuncSetAttribute(k_sink<128, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
        cudaFuncSetAttribute(k_sink<256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
        cudaFuncSetAttribute(k_sink<512, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
        cudaFuncSetAttribute(k_sink<256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
        cudaFuncSetAttribute(k_sink<256, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
        cudaFuncSetAttribute(k_sink<512, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
        cudaFuncSetAttribute(k_sink<512, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess ||
        cudaFuncSetAttribute(k_c2b, cudaFuncAttributeMaxDynamicSharedMemorySize, mx) != cudaSuccess)
        return DD_ERR_CUDA;
    g_attr_set = true;
    return DD_OK;
}

HalfArgs make_args(dd_ctx* c, int part) {
    DevPart& P = c->part[part];
    HalfArgs A;
    A.N1 = c->N1; A.N2 = c->N2; A.s = c->s; A.ncell = P.ncell; A.amax = c->amax;
    A.k2 = c->k2; A.k2d = c->k2d; A.eps = c->eps; A.h2 = c->h * c->h;
    A.members = P.members; A.xblk = P.xblk; A.mJ = P.mJ; A.order = P.order;
    A.c2b_order = nullptr; A.c2b_count = nullptr;
    A.bhdr_in = c->bhdr[c->cur]; A.pool_in = c->pool[c->cur];
    A.bhdr_out = c->bhdr[1 - c->cur]; A.pool_out = c->pool[1 - c->cur];
    A.chdr = P.chdr; A.comp_b = P.comp_b; A.comp_nu = P.comp_nu;
    A.alpha = P.alpha; A.gauge = P.gauge;
    A.warm = ((c->opt.warm == DD_WARM_PREV || c->opt.warm == DD_WARM_MLP) && P.warm_valid) ? 1 : 0;
    A.lgmu = c->d_lgmu; A.mu = c->d_mu; A.nu = c->d_nu; A.m = c->d_m;
    A.lnmu = c->d_lnmu; A.lnnu = c->d_lnnu; A.lnnuf = c->d_lnnuf;
    A.tol = c->opt.tol; A.max_iter = c->opt.max_iter; A.fixed_iters = c->opt.fixed_iters;
    A.tol_share = c->opt.tol_share; A.mbar = P.mbar;
    A.budget = P.budget;
    A.omega = (float)c->opt.omega;
    A.trunc = (float)c->opt.trunc;
    A.iters = P.iters; A.err = P.err; A.Ecell = P.Ecell; A.bmom = c->d_bmom;
    A.pre = (c->opt.flags & DD_FLAG_KEEP_PREBALANCE) ? c->d_pre : nullptr;
    A.queue = c->d_queue; A.status = c->d_status + 8 * c->status_slot;
    A.guard = c->capturing ? c->d_guard : nullptr;
    A.count = nullptr;
    A.trace = (c->opt.flags & DD_FLAG_TRACE) ? c->d_trace[part] : nullptr;
    A.aa_m = c->opt.fixed_iters > 0 ? 0 : c->opt.anderson;
    A.fused = (c->fuse_c2b && (c->opt.flags & DD_FLAG_FUSED_C2B)) ? c->d_fused : nullptr;
    A.pmom = c->opt.eps_gamma > 0.0 ? c->d_pmom : nullptr;
    A.eps_levels = c->opt.eps_levels;
    A.eps_factor = (float)c->opt.eps_factor;
    A.eps_tol = c->opt.eps_tol;
    A.comp_cap = (long long)P.comp_cap;
    A.out_cap = (long long)c->pool_cap[1 - c->cur];
    A.gscr_cap = (long long)c->gscr_cap;
    A.pre_cap = (long long)c->pre_cap;
    A.gscratch = nullptr; A.goff = nullptr;
    A.affine = (c->opt.warm == DD_WARM_AFFINE || c->opt.warm == DD_WARM_MLP) ? 1 : 0;
    A.pred = mlp_active(c, part) ? c->d_pred : nullptr;
    A.pred_old = (mlp_active(c, part) && mlp_keeps_old(c) && P.pred_old_valid) ? c->d_pred_old[part] : nullptr;
    A.targ = (c->opt.flags & DD_FLAG_COLLECT) ? c->d_targ : nullptr;
    return A;
}
}  // namespace

int launch_feat(dd_ctx* c, int part) {
    HalfArgs A = make_args(c, part);
    k_feat<<<c->part[part].ncell, 128, 0, c->stream>>>(A, reinterpret_cast<__nv_bfloat16*>(c->d_feat));
    return launch_status(__func__);
}

int launch_collect(dd_ctx* c, int n, const int32_t* idx, uint16_t* feat, float* targ) {
    if (n <= 0) return DD_OK;
    k_collect<<<n, 64, 0, c->stream>>>(n, idx, reinterpret_cast<const uint4*>(c->d_feat),
                                       reinterpret_cast<const uint4*>(c->d_targ), reinterpret_cast<uint4*>(feat),
                                       reinterpret_cast<uint4*>(targ));
    return launch_status(__func__);
}

int half_threads(int requested) {
    return requested <= 64 ? 64 : (requested <= 128 ? 128 : (requested <= 256 ? 256 : 512));
}

int launch_classify(dd_ctx* c, int part, int stage) {
    const DevPart& P = c->part[part];
    ClassCaps cc{c->gcap.a0, c->gcap.h0, c->gcap.w0, c->gcap.h2, c->gcap.w2, c->gcap.gscr, c->gcap.comp[part],
                 c->gcap.pool, c->tune.small_area, c->tune.small_side, c->gcap.cl_cap, kClusterMinArea};
    k_classify<<<1, 1024, 0, c->stream>>>(P.ncell, P.chdr, P.iters, cc, c->d_corder[part], c->d_ccount[part],
                                          c->d_goff, c->d_tot, c->d_guard, stage);
    return launch_status(__func__);
}

int launch_half(dd_ctx* c, int part, const int32_t* order, int ncell, int* queue, const long long dims[3],
                int threads, size_t smem, int grid, cudaStream_t stream, bool global_boxes, const int* count_dev) {
    RET_IF(set_attrs());
    HalfArgs A = make_args(c, part);
    A.count = count_dev;
    if (global_boxes) {
        A.gscratch = c->d_gscr;
        A.goff = c->d_goff;
    }
    A.ncell = ncell;
    A.order = order;
    A.queue = queue;
    A.smaxA = (int)dims[0];
    A.smaxH = (int)dims[1];
    A.smaxW = (int)dims[2];
    switch (half_threads(threads)) {
        case 64: k_sink<64, 1><<<grid, 64, smem, stream>>>(A); break;
        case 128: k_sink<128, 1><<<grid, 128, smem, stream>>>(A); break;
        case 256: k_sink<256, 1><<<grid, 256, smem, stream>>>(A); break;
        default: k_sink<512, 1><<<grid, 512, smem, stream>>>(A); break;
    }
    return launch_status(__func__);
}

int half_cluster_size(int requested) { return requested >= 4 ? 4 : (requested >= 2 ? 2 : 1); }

int launch_half_cluster(dd_ctx* c, int part, const int32_t* order, int ncell, int* queue, const long long dims[3],
                        int threads, int cl, size_t smem, int nclusters, cudaStream_t stream, const int* count_dev) {
    RET_IF(set_attrs());
    HalfArgs A = make_args(c, part);
    A.count = count_dev;
    A.gscratch = c->d_gscr;
    A.goff = c->d_goff;
    A.ncell = ncell;
    A.order = order;
    A.queue = queue;
    A.smaxA = (int)dims[0];
    A.smaxH = (int)dims[1];
    A.smaxW = (int)dims[2];
    A.targ = nullptr;  // training targets come from one-CTA solves only
    const int nt = half_threads(threads) >= 512 ? 512 : 256;
    cl = half_cluster_size(cl);
    if (cl < 2 || nclusters < 1) return DD_ERR_ARG;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclusters * cl), 1, 1);
    cfg.blockDim = dim3((unsigned)nt, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (nt == 512)
        e = cl == 4 ? cudaLaunchKernelEx(&cfg, k_sink<512, 4>, A) : cudaLaunchKernelEx(&cfg, k_sink<512, 2>, A);
    else
        e = cl == 4 ? cudaLaunchKernelEx(&cfg, k_sink<256, 4>, A) : cudaLaunchKernelEx(&cfg, k_sink<256, 2>, A);
    if (e != cudaSuccess) return dd_record_cuda_error(e, __func__);
    return launch_status(__func__);
}

int launch_c2b(dd_ctx* c, int part, const long long dims[3], size_t smem, const int32_t* order, const int* count) {
    RET_IF(set_attrs());
    HalfArgs A = make_args(c, part);
    A.c2b_order = order;
    A.c2b_count = count;
    A.smaxA = (int)dims[0];
    A.smaxH = (int)dims[1];
    A.smaxW = (int)dims[2];
    A.fused = c->d_fused;  // skips (and clears) the cells done by their solving CTAs
    k_c2b<<<c->part[part].ncell, kC2bThreads, smem, c->stream>>>(A);
    return launch_status(__func__);
}

int half_occupancy(int threads, size_t smem) {
    if (set_attrs() != DD_OK) return 0;
    int nb = 0;
    switch (half_threads(threads)) {
        case 64: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sink<64, 1>, 64, smem); break;
        case 128: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sink<128, 1>, 128, smem); break;
        case 256: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sink<256, 1>, 256, smem); break;
        default: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_sink<512, 1>, 512, smem); break;
    }
    return nb;
}
