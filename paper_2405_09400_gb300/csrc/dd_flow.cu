// Flow update kernels (Section 3.2 and the steps of Section 5.1) and the
// Y-marginal error reduction.
//
//  k_cbar            edge costs Eq. (edge-cost) for product gluing candidates
//                    (Remark 3.8): for j != i
//                      c_bar_ij = q_i h^2 (|xbar_j - ybar_i|^2 + Var_x(j) + Var_y(i)) - D_i / m_i,
//                    the mean of |x - y|^2 under mu_j/m_j (x) nu_i/|nu_i| times
//                    q_i = |nu_i| / m_i, minus <c, pi_i> / m_i; c_bar_ii = 0.
//                    One thread per basic cell, FP64.
//  k_plan_exchange   one CTA: union box of the sources i in N(j) with w_ij > 0
//                    for every target j, and pool offsets (prefix sum).
//  k_exchange        one CTA per target j: nu_hat_j = sum_i (w_ij / m_i) nu_i
//                    (Eq. flow-update-cell-marginals), truncation and the minimal
//                    box, written compactly (two passes over the union box).
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
__global__ void k_plan_exchange(int nb, const int32_t* __restrict__ nbr, const int32_t* __restrict__ rev,
                                const double* __restrict__ w, const int32_t* __restrict__ bhdr,
                                int32_t* __restrict__ xhdr, long long* __restrict__ tot, int* __restrict__ guard,
                                long long pool_cap, int stage) {
    __shared__ long long sh[64];
    if (guard && *guard) return;
    const int T = blockDim.x;
    const int per = (nb + T - 1) / T;
    const int c0 = min(nb, threadIdx.x * per), c1 = min(nb, c0 + per);
    long long sa = 0, sin = 0, sout = 0;
    for (int j = c0; j < c1; ++j) {
        int lo1 = INT32_MAX, lo2 = INT32_MAX, hi1 = INT32_MIN, hi2 = INT32_MIN;
        for (int k = 0; k < 5; ++k) {
            const int i = nbr[5 * j + k];
            if (i < 0) continue;
            if (!(w[5 * i + rev[5 * j + k]] > 0.0)) continue;
            const int32_t* b = bhdr + BH_N * i;
            if (b[BH_H] <= 0 || b[BH_W] <= 0) continue;
            sin += (long long)b[BH_H] * b[BH_W];
            lo1 = min(lo1, b[BH_O1]);
            lo2 = min(lo2, b[BH_O2]);
            hi1 = max(hi1, b[BH_O1] + b[BH_H]);
            hi2 = max(hi2, b[BH_O2] + b[BH_W]);
        }
        int h = 0, ww = 0;
        if (hi1 > lo1) { h = hi1 - lo1; ww = hi2 - lo2; } else { lo1 = lo2 = 0; }
        int32_t* x = xhdr + CH_N * j;
        x[CH_O1] = lo1; x[CH_O2] = lo2; x[CH_H] = h; x[CH_W] = ww; x[CH_STRIDE] = (ww + 3) & ~3;
        sa += (long long)h * ((ww + 3) & ~3);
        sout += (long long)h * ww;
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

__device__ __forceinline__ float gather_sum(int y1, int y2, int nsrc, const int* src, const float* coef,
                                            const int32_t* __restrict__ bhdr, const float* __restrict__ pool) {
    float acc = 0.f;
    for (int t = 0; t < nsrc; ++t) {
        const int32_t* b = bhdr + BH_N * src[t];
        const int p1 = y1 - b[BH_O1], p2 = y2 - b[BH_O2];
        if (p1 >= 0 && p1 < b[BH_H] && p2 >= 0 && p2 < b[BH_W])
            acc += coef[t] * pool[(long long)b[BH_START] + (long long)p1 * b[BH_STRIDE] + p2];
    }
    return acc;
}

__global__ void k_exchange(int nb, const int32_t* __restrict__ nbr, const int32_t* __restrict__ rev,
                           const double* __restrict__ w, const double* __restrict__ m,
                           const int32_t* __restrict__ bhdr_in, const float* __restrict__ pool_in,
                           const int32_t* __restrict__ xhdr, int32_t* __restrict__ bhdr_out,
                           float* __restrict__ pool_out, double* __restrict__ bmom, float trunc,
                           const int* __restrict__ guard, long long out_cap, int* __restrict__ status) {
    if (guard && *guard) return;
    __shared__ int src[5];
    __shared__ float coef[5];
    __shared__ int nsrc;
    __shared__ int bb[4];
    __shared__ double red[32];
    const int j = blockIdx.x;
    if (threadIdx.x == 0) {
        int n = 0;
        for (int k = 0; k < 5; ++k) {
            const int i = nbr[5 * j + k];
            if (i < 0) continue;
            const double wij = w[5 * i + rev[5 * j + k]];
            if (!(wij > 0.0)) continue;
            src[n] = i;
            coef[n] = (float)(wij / m[i]);
            ++n;
        }
        nsrc = n;
        bb[0] = INT32_MAX; bb[1] = -1; bb[2] = INT32_MAX; bb[3] = -1;
    }
    __syncthreads();
    const int32_t* x = xhdr + CH_N * j;
    const int o1 = x[CH_O1], o2 = x[CH_O2], h = x[CH_H], ww = x[CH_W];
    const long long start = x[CH_OUT_SLOT];
    if (start + (long long)h * x[CH_STRIDE] > out_cap) {  // beyond the output pool: skip, report
        if (threadIdx.x == 0) atomicAdd(status, 1);
        return;
    }
    // pass 1: minimal box of the entries >= trunc
    int lo1 = INT32_MAX, hi1 = -1, lo2 = INT32_MAX, hi2 = -1;
    for (int v = threadIdx.x; v < h * ww; v += blockDim.x) {
        const int v1 = v / ww, v2 = v - v1 * ww;
        const float val = gather_sum(o1 + v1, o2 + v2, nsrc, src, coef, bhdr_in, pool_in);
        if (val >= trunc) {
            lo1 = min(lo1, v1); hi1 = max(hi1, v1);
            lo2 = min(lo2, v2); hi2 = max(hi2, v2);
        }
    }
    atomicMin(&bb[0], lo1); atomicMax(&bb[1], hi1); atomicMin(&bb[2], lo2); atomicMax(&bb[3], hi2);
    __syncthreads();
    const bool empty = bb[1] < 0;
    const int r0 = bb[0], c0 = bb[2];
    const int hh = empty ? 0 : bb[1] - bb[0] + 1, w2 = empty ? 0 : bb[3] - bb[2] + 1;
    const int st = (w2 + 3) & ~3;
    // pass 2: the mass of the truncated box (FP64), then the compact box rescaled
    // to the basic mass m_j (the inflow of the flow is m_j, Eq. div-constraint-single-cell)
    double ms = 0.0;
    for (int d = threadIdx.x; d < hh * w2; d += blockDim.x) {
        const int rr = d / w2, cc = d - rr * w2;
        float val = gather_sum(o1 + r0 + rr, o2 + c0 + cc, nsrc, src, coef, bhdr_in, pool_in);
        if (val >= trunc) ms += val;
    }
    for (int o = 16; o > 0; o >>= 1) ms += __shfl_down_sync(0xffffffffu, ms, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = ms;
    __syncthreads();
    __shared__ float fsc;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        fsc = t > 0.0 ? (float)(m[j] / t) : 1.f;
        bmom[BM_N * j + BM_MASS] = t > 0.0 ? m[j] : 0.0;
    }
    __syncthreads();
    for (int d = threadIdx.x; d < hh * st; d += blockDim.x) {
        const int rr = d / st, cc = d - rr * st;
        float val = 0.f;
        if (cc < w2) {
            val = gather_sum(o1 + r0 + rr, o2 + c0 + cc, nsrc, src, coef, bhdr_in, pool_in);
            val = (val >= trunc) ? val * fsc : 0.f;
        }
        pool_out[start + d] = val;
    }
    if (threadIdx.x == 0) {
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
    k_plan_exchange<<<1, 1024, 0, c->stream>>>(c->nb, c->d_nbr, c->d_rev, c->d_w, c->bhdr[c->cur], c->d_xhdr,
                                               c->d_tot, c->capturing ? c->d_guard : nullptr, c->gcap.pool, stage);
    return launch_status(__func__);
}

int launch_exchange(dd_ctx* c) {
    k_exchange<<<c->nb, 128, 0, c->stream>>>(c->nb, c->d_nbr, c->d_rev, c->d_w, c->d_m, c->bhdr[c->cur],
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
