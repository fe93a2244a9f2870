// Device-side plan packing for dd_set_plan / dd_get_plan (kernels; the host
// side is in dd_api.cu).
//
// The caller's plan (basic-cell Y-marginals as packed float64 boxes) is copied
// to the device as it is and packed there into the FP32 pool layout (rows of
// stride ceil(w/4)*4, zero padding); the feasibility check of dd_set_plan (every
// entry finite and >= 0, |nu_i| = m_i and sum_i nu_i = nu within plan_tol, L1)
// runs on the device in FP64 on the caller's values. The packed plan goes to
// the pool that is not current and becomes current only when the check passes,
// so a rejected plan leaves the state as it was. dd_get_plan unpacks the current
// pool into float64 on the device and copies the packed array out once.
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"

namespace {

// one CTA per basic cell: FP64 entries -> FP32 pool rows, the cell's FP64 mass,
// the Y-marginal sum (FP64 atomics), and a flag for negative / non-finite values
__global__ void k_pack_plan(int nb, int N2, const int32_t* __restrict__ bhdr, const long long* __restrict__ soff,
                            const double* __restrict__ src, float* __restrict__ pool, double* __restrict__ cell_mass,
                            double* __restrict__ ym, int* __restrict__ bad) {
    __shared__ double red[32];
    const int i = blockIdx.x;
    if (i >= nb) return;
    const int32_t* b = bhdr + BH_N * i;
    const int h = b[BH_H], w = b[BH_W], st = b[BH_STRIDE];
    const long long s0 = soff[i];
    const long long d0 = b[BH_START];
    double mass = 0.0;
    for (int v = threadIdx.x; v < h * st; v += blockDim.x) {
        const int r = v / st, q = v - r * st;
        float out = 0.f;
        if (q < w) {
            const double x = src[s0 + (long long)r * w + q];
            if (!(x >= 0.0) || !isfinite(x)) {
                atomicExch(bad, 1);
            } else {
                out = (float)x;
                mass += x;
                if (ym && x != 0.0) atomicAdd(&ym[(long long)(b[BH_O1] + r) * N2 + b[BH_O2] + q], x);
            }
        }
        pool[d0 + v] = out;
    }
    if (!cell_mass) return;
    for (int o = 16; o > 0; o >>= 1) mass += __shfl_down_sync(0xffffffffu, mass, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mass;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        cell_mass[i] = t;
    }
}

// out[0] += sum_i |cell_mass_i - m_i|, out[1] += sum_y |ym - nu|
__global__ void k_plan_err(int nb, const double* __restrict__ cell_mass, const double* __restrict__ m, long long np,
                           const double* __restrict__ ym, const double* __restrict__ nu, double* __restrict__ out) {
    __shared__ double red[2][32];
    double sx = 0.0, sy = 0.0;
    const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, dt = (long long)gridDim.x * blockDim.x;
    for (long long k = t0; k < nb; k += dt) sx += fabs(cell_mass[k] - m[k]);
    for (long long k = t0; k < np; k += dt) sy += fabs(ym[k] - nu[k]);
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red[0][threadIdx.x >> 5] = sx;
        red[1][threadIdx.x >> 5] = sy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0.0, c = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            a += red[0][k];
            c += red[1][k];
        }
        atomicAdd(&out[0], a);
        atomicAdd(&out[1], c);
    }
}

// one CTA per basic cell: FP32 pool rows -> packed FP64 boxes
__global__ void k_unpack_plan(int nb, const int32_t* __restrict__ bhdr, const long long* __restrict__ soff,
                              const float* __restrict__ pool, double* __restrict__ dst) {
    const int i = blockIdx.x;
    if (i >= nb) return;
    const int32_t* b = bhdr + BH_N * i;
    const int h = b[BH_H], w = b[BH_W], st = b[BH_STRIDE];
    const long long s0 = soff[i], d0 = b[BH_START];
    for (int v = threadIdx.x; v < h * w; v += blockDim.x) {
        const int r = v / w, q = v - r * w;
        dst[s0 + v] = (double)pool[d0 + (long long)r * st + q];
    }
}

}  // namespace

int launch_pack_plan(dd_ctx* c, int dst, bool validate) {
    const int nb = c->nb;
    const long long np = (long long)c->N1 * c->N2;
    int* bad = reinterpret_cast<int*>(c->d_red + 2);
    k_pack_plan<<<nb, 128, 0, c->stream>>>(nb, c->N2, c->bhdr[dst], c->d_soff, c->d_plan64, c->pool[dst],
                                          validate ? c->d_cellmass : nullptr, validate ? c->d_yacc : nullptr, bad);
    int r = launch_status("k_pack_plan");
    if (r != DD_OK || !validate) return r;
    k_plan_err<<<c->nsm * 2, 256, 0, c->stream>>>(nb, c->d_cellmass, c->d_m, np, c->d_yacc, c->d_nu, c->d_red);
    return launch_status("k_plan_err");
}

int launch_unpack_plan(dd_ctx* c) {
    k_unpack_plan<<<c->nb, 128, 0, c->stream>>>(c->nb, c->bhdr[c->cur], c->d_soff, c->pool[c->cur], c->d_plan64);
    return launch_status("k_unpack_plan");
}
