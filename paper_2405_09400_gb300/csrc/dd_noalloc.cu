// dd_l1_y_error_static: the L1 Y-marginal error of a basic-cell box state,
// computed without allocating any device memory.
//
// Some callers cannot allocate: real-time or embedded pipelines that reserve all
// device memory up front and forbid allocation afterwards, and host frameworks
// whose own caching allocator owns the device memory (a cudaMalloc behind its
// back can fail or fragment its pool). For them
// this entry point uses a fixed scratch area that lives in a file-scope
// __device__ array instead of memory from cudaMalloc. The caller passes inputs
// and the output in device memory, as for dd_get_objective's Y error.
//
// Limits: at most DD_STATIC_MAX_PIXELS grid pixels and DD_STATIC_MAX_CELLS
// basic cells; the array (about 8.5 MB) stays resident on every GPU that loads
// the library, until the process exits. All calls share it, so two calls that
// overlap on the GPU (different streams, or different host threads on the same
// device) race; calls ordered on one stream are safe.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>

#include "../../include/ddflow.h"

namespace {

constexpr long long kMaxPixels = DD_STATIC_MAX_PIXELS;
constexpr int kMaxCells = DD_STATIC_MAX_CELLS;
constexpr int kMaxDevices = 64;

// scratch: the FP64 Y accumulator over the grid, then the box offsets
struct StaticScratch {
    double acc[kMaxPixels];
    long long offset[kMaxCells + 1];
};
static __device__ __align__(256) StaticScratch g_scratch;

// host-side device address of g_scratch, looked up once per device; host threads
// making their first call on one device at the same time may both look it up and
// store the same value
std::atomic<StaticScratch*> g_addr[kMaxDevices] = {};

// entries of a box: h * w, or 0 for a box with a non-positive extent
__device__ __forceinline__ long long box_size(const int32_t* __restrict__ hdr, int i) {
    const int h = hdr[4 * i + 2], w = hdr[4 * i + 3];
    return (h > 0 && w > 0) ? (long long)h * w : 0LL;
}

__global__ void k_offsets(int nb, const int32_t* __restrict__ hdr, StaticScratch* __restrict__ S) {
    // one CTA: exclusive prefix sum of the box sizes h * w (packed, unpadded boxes)
    __shared__ long long part[1024];
    const int T = blockDim.x, per = (nb + T - 1) / T;
    const int c0 = min(nb, (int)threadIdx.x * per), c1 = min(nb, c0 + per);
    long long s = 0;
    for (int i = c0; i < c1; ++i) s += box_size(hdr, i);
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long run = 0;
        for (int t = 0; t < T; ++t) {
            long long x = part[t];
            part[t] = run;
            run += x;
        }
        S->offset[nb] = run;
    }
    __syncthreads();
    long long run = part[threadIdx.x];
    for (int i = c0; i < c1; ++i) {
        S->offset[i] = run;
        run += box_size(hdr, i);
    }
}

__global__ void k_zero(long long n, StaticScratch* __restrict__ S, double* __restrict__ out) {
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        S->acc[k] = 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) *out = 0.0;
}

__global__ void k_scatter(int N1, int N2, const int32_t* __restrict__ hdr, const float* __restrict__ data,
                          StaticScratch* __restrict__ S) {
    const int i = blockIdx.x;
    const int o1 = hdr[4 * i], o2 = hdr[4 * i + 1], h = hdr[4 * i + 2], w = hdr[4 * i + 3];
    if (h <= 0 || w <= 0) return;
    const long long base = S->offset[i], n = (long long)h * w;
    for (long long v = threadIdx.x; v < n; v += blockDim.x) {
        const long long v1 = v / w, v2 = v - v1 * w;
        const long long y1 = o1 + v1, y2 = o2 + v2;
        if (y1 < 0 || y1 >= N1 || y2 < 0 || y2 >= N2) continue;  // outside the grid: ignored
        const float val = data[base + v];
        if (val != 0.f) atomicAdd(&S->acc[(long long)y1 * N2 + y2], (double)val);
    }
}

__global__ void k_reduce(long long n, const double* __restrict__ nu, const StaticScratch* __restrict__ S,
                         double* __restrict__ out) {
    __shared__ double red[32];
    double s = 0.0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x)
        s += fabs(S->acc[k] - nu[k]);
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

extern "C" int dd_l1_y_error_static(int32_t N1, int32_t N2, int32_t nbasic, const int32_t* hdr, const float* data,
                                    const double* nu, double* l1_out, void* stream) {
    if (N1 <= 0 || N2 <= 0 || nbasic <= 0 || !hdr || !data || !nu || !l1_out) return DD_ERR_ARG;
    const long long np = (long long)N1 * N2;
    if (np > kMaxPixels || nbasic > kMaxCells) return DD_ERR_ARG;  // beyond the static scratch
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DD_ERR_CUDA;
    StaticScratch* S = g_addr[dev].load(std::memory_order_acquire);
    if (!S) {
        // first call on this device: the host-side name g_scratch is not a device
        // address; ask the runtime for it (with this device current)
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return DD_ERR_CUDA;
        S = static_cast<StaticScratch*>(p);
        g_addr[dev].store(S, std::memory_order_release);
    }
    cudaStream_t st = (cudaStream_t)stream;
    int nsm = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return DD_ERR_CUDA;
    k_offsets<<<1, 1024, 0, st>>>(nbasic, hdr, S);
    k_zero<<<2 * nsm, 256, 0, st>>>(np, S, l1_out);
    k_scatter<<<nbasic, 128, 0, st>>>(N1, N2, hdr, data, S);
    k_reduce<<<2 * nsm, 256, 0, st>>>(np, nu, S, l1_out);
    return cudaGetLastError() == cudaSuccess ? DD_OK : DD_ERR_CUDA;
}
