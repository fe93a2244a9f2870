// Flow update kernels (Section 3.2 and the steps of Section 5.1) and the
// Y-marginal error reduction.
//
//  k_cbar            edge costs Eq. (edge-cost) for product gluing candidates
//                    (Remark 3.8): for j != i
//                      c_bar_ij = q_i h^2 (|xbar_j - ybar_i|^2 + Var_x(j) + Var_y(i)) - D_i / m_i,
//                    the mean of |x - y|^2 under mu_j/m_j (x) nu_i/|nu_i| times
//                    q_i = |nu_i| / m_i, minus <c, pi_i> / m_i; c_bar_ii = 0.
//                    One thread per basic cell, FP64.
//  k_xbox            one thread per target j: union box of the sources i in
//                    N(j) with w_ij > 0.
//  k_plan_exchange   one CTA: pool offsets of the union boxes (prefix sum).
//  k_exchange        one CTA per target j: nu_hat_j = sum_i (w_ij / m_i) nu_i
//                    (Eq. flow-update-cell-marginals), truncation and the minimal
//                    box, written compactly: one gather over the union box (values
//                    kept in shared memory up to 4096 entries, else gathered again
//                    for the compact write).
//  k_scatter_y / k_l1y   sum_y |sum_i nu_i(y) - nu(y)| in FP64.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"

namespace {

__global__ void k_cbar(int nb, const int32_t* __restrict__ nbr, const double* __restrict__ xmom,
                       const double* __restrict__ bmom, const double* __restrict__ m, double h2,
                       double* __restrict__ cbar, const int* __restrict__ guard) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nb || (guard && *guard)) return;
    const double* bi = bmom + BM_N * i;
    const double q = bi[BM_MASS] / m[i];
    const double Di = bi[BM_D] / m[i];
    for (int k = 0; k < 5; ++k) {
        int j = nbr[5 * i + k];
        double c = 0.0;
        if (j >= 0 && j != i) {
            const double* xj = xmom + 3 * j;
            const double d1 = xj[0] - bi[BM_Y1], d2 = xj[1] - bi[BM_Y2];
            c = q * h2 * (d1 * d1 + d2 * d2 + xj[2] + bi[BM_VAR]) - Di;
        }
        cbar[5 * i + k] = c;
    }
}

__device__ long long block_exscan_x(long long x, long long* sh, long long* total) {
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
        if (lane < nw) sh[lane] = s;
    }
    __syncthreads();
    long long base = wid > 0 ? sh[wid - 1] : 0;
    *total = sh[nw - 1];
    __syncthreads();
    return base + inc - x;
}

// rev[5*j + k] = position of j in the neighbour list of i = nbr[5*j + k]
// union box of the sources i in N(j) with w_ij > 0 of every target j, one
// thread per target: CH_O1, CH_O2, CH_H, CH_W, CH_STRIDE of xhdr, and in
// CH_COMP_LO the entries of those source boxes (read by the exchange)
__global__ void k_xbox(int nb, const int32_t* __restrict__ nbr, const int32_t* __restrict__ rev,
                       const double* __restrict__ w, const int32_t* __restrict__ bhdr, int32_t* __restrict__ xhdr,
                       const int* __restrict__ guard) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nb || (guard && *guard)) return;
    // the five neighbour slots' loads are independent: issue them together
    int src[5], rv[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        src[k] = nbr[5 * j + k];
        rv[k] = rev[5 * j + k];
    }
    double wk[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) wk[k] = src[k] >= 0 ? w[5 * src[k] + rv[k]] : 0.0;
    int bo1[5], bo2[5], bh[5], bw[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const bool use = src[k] >= 0 && wk[k] > 0.0;
        const int32_t* b = bhdr + BH_N * (use ? src[k] : 0);
        bo1[k] = use ? b[BH_O1] : 0;
        bo2[k] = use ? b[BH_O2] : 0;
        bh[k] = use ? b[BH_H] : 0;
        bw[k] = use ? b[BH_W] : 0;
    }
    int lo1 = INT32_MAX, lo2 = INT32_MAX, hi1 = INT32_MIN, hi2 = INT32_MIN, sin = 0;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        if (bh[k] <= 0 || bw[k] <= 0) continue;
        sin += bh[k] * bw[k];
        lo1 = min(lo1, bo1[k]);
        lo2 = min(lo2, bo2[k]);
        hi1 = max(hi1, bo1[k] + bh[k]);
        hi2 = max(hi2, bo2[k] + bw[k]);
    }
    int h = 0, ww = 0;
    if (hi1 > lo1) { h = hi1 - lo1; ww = hi2 - lo2; } else { lo1 = lo2 = 0; }
    int32_t* x = xhdr + CH_N * j;
    x[CH_O1] = lo1; x[CH_O2] = lo2; x[CH_H] = h; x[CH_W] = ww; x[CH_STRIDE] = (ww + 3) & ~3;
    x[CH_COMP_LO] = sin;
}

// one CTA: pool offsets of the exchange outputs (prefix sum of the union boxes
// k_xbox wrote) and the totals
__global__ void k_plan_exchange(int nb, int32_t* __restrict__ xhdr, long long* __restrict__ tot,
                                int* __restrict__ guard, long long pool_cap, int stage) {
    __shared__ long long sh[64];
    if (guard && *guard) return;
    const int T = blockDim.x;
    const int per = (nb + T - 1) / T;
    const int c0 = min(nb, threadIdx.x * per), c1 = min(nb, c0 + per);
    long long sa = 0, sin = 0, sout = 0;
    for (int j = c0; j < c1; ++j) {
        const int32_t* x = xhdr + CH_N * j;
        const int h = x[CH_H];
        sa += (long long)h * x[CH_STRIDE];
        sout += (long long)h * x[CH_W];
        sin += x[CH_COMP_LO];
    }
    long long ta, tin, tout;
    (void)block_exscan_x(sin, sh, &tin);
    (void)block_exscan_x(sout, sh, &tout);
    long long ea = block_exscan_x(sa, sh, &ta);
    for (int j = c0; j < c1; ++j) {
        int32_t* x = xhdr + CH_N * j;
        x[CH_OUT_SLOT] = (int32_t)ea;
        ea += (long long)x[CH_H] * x[CH_STRIDE];
    }
    if (threadIdx.x == 0) {
        tot[PT_OUT] = ta;
        tot[PT_PAD0] = tin;   // entries of the source boxes read (algorithmic bytes)
        tot[PT_PAD1] = tout;  // entries of the new boxes written
        // graph mode: the output pool was captured with a fixed capacity
        if (guard && ta > pool_cap) atomicCAS(guard, 0, stage);
    }
}

// sources of one exchange target in shared memory: box, pool start and w_ij / m_i
struct XchSrc {
    int o1[5], o2[5], h[5], w[5], stride[5];
    long long start[5];
    float coef[5];
    int n;
};

// sum_t coef_t nu_t(y) over the sources; the five loads are predicated and
// independent (issued together), the terms added in source order (a source
// whose box misses y adds +0, which leaves the non-negative sum unchanged)
__device__ __forceinline__ float gather_sum(int y1, int y2, const XchSrc& S, const float* __restrict__ pool) {
    float v[5];
#pragma unroll
    for (int t = 0; t < 5; ++t) {
        const int p1 = y1 - S.o1[t], p2 = y2 - S.o2[t];
        const bool in = p1 >= 0 && p1 < S.h[t] && p2 >= 0 && p2 < S.w[t];
        v[t] = in ? __ldg(pool + S.start[t] + (long long)p1 * S.stride[t] + p2) : 0.f;
    }
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < 5; ++t) acc += S.coef[t] * v[t];
    return acc;
}

constexpr int kXchThreads = 128;
constexpr int kXchCache = 4096;  // union-box values kept in shared memory; larger boxes are gathered twice

__global__ void __launch_bounds__(kXchThreads) k_exchange(int nb, const int32_t* __restrict__ nbr,
                                                          const int32_t* __restrict__ rev, const double* __restrict__ w,
                                                          const double* __restrict__ m,
                                                          const int32_t* __restrict__ bhdr_in,
                                                          const float* __restrict__ pool_in,
                                                          const int32_t* __restrict__ xhdr,
                                                          int32_t* __restrict__ bhdr_out, float* __restrict__ pool_out,
                                                          double* __restrict__ bmom, float trunc,
                                                          const int* __restrict__ guard, long long out_cap,
                                                          int* __restrict__ status) {
    if (guard && *guard) return;
    __shared__ XchSrc S;
    __shared__ int bb[4];
    __shared__ double red[kXchThreads / 32];
    __shared__ float fsc;
    __shared__ float vals[kXchCache];
    const int j = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int32_t* x = xhdr + CH_N * j;  // the target's union box (read while warp 0 gathers the sources)
    const int o1 = x[CH_O1], o2 = x[CH_O2], h = x[CH_H], ww = x[CH_W], xst = x[CH_STRIDE];
    const long long start = x[CH_OUT_SLOT];
    if (wid == 0) {
        // lane k < 5: neighbour slot k; the sources with w_ij > 0 keep the slot order
        int i = -1;
        double wij = 0.0;
        if (lane < 5) {
            i = nbr[5 * j + lane];
            if (i >= 0) wij = w[5 * i + rev[5 * j + lane]];
        }
        const bool ok = lane < 5 && i >= 0 && wij > 0.0;
        const unsigned msk = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const int t = __popc(msk & ((1u << lane) - 1u));
            const int32_t* b = bhdr_in + BH_N * i;
            S.o1[t] = b[BH_O1];
            S.o2[t] = b[BH_O2];
            S.h[t] = b[BH_H];
            S.w[t] = b[BH_W];
            S.stride[t] = b[BH_STRIDE];
            S.start[t] = b[BH_START];
            S.coef[t] = (float)(wij / m[i]);
        }
        if (lane == 0) {
            S.n = __popc(msk);
            for (int t = S.n; t < 5; ++t) {  // unused slots: an empty box and a zero weight
                S.o1[t] = S.o2[t] = S.h[t] = S.w[t] = S.stride[t] = 0;
                S.start[t] = 0;
                S.coef[t] = 0.f;
            }
            bb[0] = INT32_MAX; bb[1] = -1; bb[2] = INT32_MAX; bb[3] = -1;
        }
    }
    __syncthreads();
    if (start + (long long)h * xst > out_cap) {  // beyond the output pool: skip, report
        if (tid == 0) atomicAdd(status, 1);
        return;
    }
    // pass 1 over the union box: the values (kept in shared memory when they fit),
    // the minimal box of the entries >= trunc and their mass (FP64)
    const int area = h * ww;
    const bool cached = area <= kXchCache;
    int lo1 = INT32_MAX, hi1 = -1, lo2 = INT32_MAX, hi2 = -1;
    double ms = 0.0;
    constexpr int U = 4;  // pixels per thread whose gathers are in flight together
    for (int v0 = tid; v0 < area; v0 += U * kXchThreads) {
        float val[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int v = v0 + u * kXchThreads, v1 = v / ww, v2 = v - v1 * ww;
            val[u] = v < area ? gather_sum(o1 + v1, o2 + v2, S, pool_in) : 0.f;
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int v = v0 + u * kXchThreads, v1 = v / ww, v2 = v - v1 * ww;
            if (v >= area) break;
            if (cached) vals[v] = val[u];
            if (val[u] >= trunc) {
                lo1 = min(lo1, v1); hi1 = max(hi1, v1);
                lo2 = min(lo2, v2); hi2 = max(hi2, v2);
                ms += val[u];
            }
        }
    }
    lo1 = __reduce_min_sync(0xffffffffu, lo1);
    hi1 = __reduce_max_sync(0xffffffffu, hi1);
    lo2 = __reduce_min_sync(0xffffffffu, lo2);
    hi2 = __reduce_max_sync(0xffffffffu, hi2);
    for (int o = 16; o > 0; o >>= 1) ms += __shfl_down_sync(0xffffffffu, ms, o);
    if (lane == 0) {
        atomicMin(&bb[0], lo1); atomicMax(&bb[1], hi1); atomicMin(&bb[2], lo2); atomicMax(&bb[3], hi2);
        red[wid] = ms;
    }
    __syncthreads();
    // the compact box rescaled to the basic mass m_j (the inflow of the flow is
    // m_j, Eq. div-constraint-single-cell)
    if (tid == 0) {
        double t = 0.0;
        for (int k = 0; k < kXchThreads / 32; ++k) t += red[k];
        fsc = t > 0.0 ? (float)(m[j] / t) : 1.f;
        bmom[BM_N * j + BM_MASS] = t > 0.0 ? m[j] : 0.0;
    }
    __syncthreads();
    const bool empty = bb[1] < 0;
    const int r0 = bb[0], c0 = bb[2];
    const int hh = empty ? 0 : bb[1] - bb[0] + 1, w2 = empty ? 0 : bb[3] - bb[2] + 1;
    const int st = (w2 + 3) & ~3;
    const float f = fsc;
    for (int d = tid; d < hh * st; d += kXchThreads) {
        const int rr = d / st, cc = d - rr * st;
        float val = 0.f;
        if (cc < w2) {
            val = cached ? vals[(r0 + rr) * ww + c0 + cc] : gather_sum(o1 + r0 + rr, o2 + c0 + cc, S, pool_in);
            val = (val >= trunc) ? val * f : 0.f;
        }
        pool_out[start + d] = val;
    }
    if (tid == 0) {
        int32_t* bo = bhdr_out + BH_N * j;
        bo[BH_O1] = empty ? 0 : o1 + r0;
        bo[BH_O2] = empty ? 0 : o2 + c0;
        bo[BH_H] = hh;
        bo[BH_W] = w2;
        bo[BH_STRIDE] = st;
        bo[BH_START] = (int32_t)start;
    }
}

__global__ void k_scatter_y(int nb, int N2, const int32_t* __restrict__ bhdr, const float* __restrict__ pool,
                            double* __restrict__ acc) {
    const int i = blockIdx.x;
    const int32_t* b = bhdr + BH_N * i;
    const int h = b[BH_H], w = b[BH_W];
    for (int v = threadIdx.x; v < h * w; v += blockDim.x) {
        const int v1 = v / w, v2 = v - v1 * w;
        const float val = pool[(long long)b[BH_START] + (long long)v1 * b[BH_STRIDE] + v2];
        if (val != 0.f) atomicAdd(&acc[(long long)(b[BH_O1] + v1) * N2 + b[BH_O2] + v2], (double)val);
    }
}

__global__ void k_l1y(long long n, const double* __restrict__ acc, const double* __restrict__ nu,
                      double* __restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        s += fabs(acc[k] - nu[k]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        atomicAdd(out, t);
    }
}

}  // namespace

int launch_cbar(dd_ctx* c) {
    if (c->opt.eps_gamma > 0.0) return launch_cbar_glued(c);
    k_cbar<<<(c->nb + 255) / 256, 256, 0, c->stream>>>(c->nb, c->d_nbr, c->d_xmom, c->d_bmom, c->d_m,
                                                       c->h * c->h, c->d_cbar, c->capturing ? c->d_guard : nullptr);
    return launch_status(__func__);
}

int launch_plan_exchange(dd_ctx* c, int stage) {
    int* g = c->capturing ? c->d_guard : nullptr;
    k_xbox<<<(c->nb + 255) / 256, 256, 0, c->stream>>>(c->nb, c->d_nbr, c->d_rev, c->d_w, c->bhdr[c->cur], c->d_xhdr, g);
    const int r = launch_status("k_xbox");
    if (r != DD_OK) return r;
    k_plan_exchange<<<1, 1024, 0, c->stream>>>(c->nb, c->d_xhdr, c->d_tot, g, c->gcap.pool, stage);
    return launch_status(__func__);
}

int launch_exchange(dd_ctx* c) {
    k_exchange<<<c->nb, kXchThreads, 0, c->stream>>>(c->nb, c->d_nbr, c->d_rev, c->d_w, c->d_m, c->bhdr[c->cur],
                                             c->pool[c->cur], c->d_xhdr, c->bhdr[1 - c->cur], c->pool[1 - c->cur],
                                             c->d_bmom, (float)c->opt.trunc, c->capturing ? c->d_guard : nullptr,
                                             (long long)c->pool_cap[1 - c->cur], c->d_status + 5);
    return launch_status(__func__);
}

int launch_l1y(dd_ctx* c, double* out_dev) {
    const long long n = (long long)c->N1 * c->N2;
    if (cudaMemsetAsync(c->d_yacc, 0, sizeof(double) * n, c->stream) != cudaSuccess) return DD_ERR_CUDA;
    if (cudaMemsetAsync(out_dev, 0, sizeof(double), c->stream) != cudaSuccess) return DD_ERR_CUDA;
    k_scatter_y<<<c->nb, 128, 0, c->stream>>>(c->nb, c->N2, c->bhdr[c->cur], c->pool[c->cur], c->d_yacc);
    k_l1y<<<c->nsm * 2, 256, 0, c->stream>>>(n, c->d_yacc, c->d_nu, out_dev);
    return launch_status(__func__);
}
