// dd_probe_ex2_rate: throughput of the MUFU base-2 exponential (ex2.approx) on
// the current device, the unit that bounds the cell Sinkhorn kernel (every
// log-sum-exp term is one ex2). A persistent grid of independent ex2 chains,
// timed with CUDA events; the result calibrates the "alu" roofline of the cell
// kernels (ex2 per clock per SM = rate / (#SM x SM clock)).
#include <cuda_runtime.h>

#include <cstdint>

#include "dd_internal.h"

namespace {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 8 independent chains per thread: x <- -0.5 * 2^x stays in [-0.5, -0.25], so
// every ex2 sees a normal argument; the multiply runs on the FMA pipe, far
// below its own peak
__global__ void __launch_bounds__(512) k_ex2_rate(int iters, float* __restrict__ sink) {
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = -0.25f - 0.03f * k - 1e-7f * threadIdx.x;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = -0.5f * ex2_approx(a[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    if (s == 1.0f) sink[blockIdx.x] = s;  // never true; keeps the chains live
}

}  // namespace

extern "C" int dd_probe_ex2_rate(void* stream, double* ex2_per_s, double* ms_out) {
    if (!ex2_per_s) return DD_ERR_ARG;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return DD_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DD_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;
    const int threads = 512, per_sm = 4, iters = 4096;
    const int grid = nsm * per_sm;
    float* sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = DD_OK;
    float best = 0.f;
    if (cudaMalloc(&sink, sizeof(float) * grid) != cudaSuccess) return DD_ERR_OOM;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = DD_ERR_CUDA;
        goto done;
    }
    k_ex2_rate<<<grid, threads, 0, st>>>(iters, sink);  // warm-up
    for (int rep = 0; rep < 5; ++rep) {
        float ms = 0.f;
        cudaEventRecord(e0, st);
        k_ex2_rate<<<grid, threads, 0, st>>>(iters, sink);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            rc = dd_record_cuda_error(cudaGetLastError(), __func__);
            goto done;
        }
        if (rep == 0 || ms < best) best = ms;
    }
    *ex2_per_s = (double)grid * threads * 8.0 * iters / (best * 1e-3);
    if (ms_out) *ms_out = best;
done:
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(sink);
    return rc;
}
