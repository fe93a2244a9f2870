// The learned warm start's network on the GPU: a multilayer perceptron
// 336 -> 256 -> 256 -> 256 -> 320 (SiLU on the hidden layers, linear output)
// with BF16 weights and activations and FP32 accumulation, and its training
// (backpropagation, Adam). Not in the paper: it predicts the X dual that
// initialises each composite-cell Sinkhorn solve (alpha_init of Alg. 1 / Alg. 4).
//
// Every layer product is one tensor-core GEMM kernel,
//   C(m, n) = sum_k A(m, k) B(n, k),
// with A and B read as BF16 in either orientation (K contiguous or not), tiles
// of 64 x 64 x 32 staged in shared memory and mma.sync m16n8k16 BF16 -> FP32,
// and a fused epilogue (bias, SiLU, SiLU' of the next layer down, FP32/BF16
// stores). The forward pass of one layer, the two gradient products of the
// backward pass (dW = dZ^T H, dH = dZ W) and the bias sums are all of that form.
//
// Parameters: one flat FP32 vector (master copy), W_1 (256 x 336, row n = the
// weights into output n), b_1, W_2, b_2, W_3, b_3, W_4 (320 x 256), b_4; a BF16
// copy of the same vector feeds the GEMMs; biases are read in FP32.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "dd_internal.h"

namespace {

constexpr int kL = 4;
constexpr int kDims[kL + 1] = {DD_MLP_NIN, DD_MLP_NHID, DD_MLP_NHID, DD_MLP_NHID, DD_MLP_NOUT};

constexpr long long w_off(int l) {
    long long o = 0;
    for (int i = 0; i < l; ++i) o += (long long)kDims[i] * kDims[i + 1] + kDims[i + 1];
    return o;
}
constexpr long long b_off(int l) { return w_off(l) + (long long)kDims[l] * kDims[l + 1]; }
static_assert(w_off(kL) == DD_MLP_NPARAMS, "parameter count");

enum Epi { EPI_F32 = 0, EPI_BIAS_F32, EPI_BIAS_SILU, EPI_DSILU };

struct GemmArgs {
    int M, N, K;
    const __nv_bfloat16* A;
    long long lda;
    const __nv_bfloat16* B;
    long long ldb;
    int epi;
    const float* bias;    // EPI_BIAS_*: per n
    const float* zprev;   // EPI_DSILU: pre-activation (M x N) of the layer below
    float* outf;          // FP32 output (M x N, row stride ldc), may be null
    __nv_bfloat16* outh;  // BF16 output, may be null
    long long ldc;
};

__device__ __forceinline__ float silu_f(float z) { return z / (1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad_f(float z) {
    const float s = 1.f / (1.f + __expf(-z));
    return s * (1.f + z * (1.f - s));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

constexpr int BM = 64, BN = 64, BK = 32, SROW = BK + 8;  // SROW: padded row (bank spread)

// Stage a 64 x 32 tile X(r, c) = src(row0 + r, k0 + c) into shared memory, zero
// outside [0, R) x [0, K). KC: the source is K-contiguous (src[row * ld + k]),
// otherwise row-contiguous (src[k * ld + row]).
template <bool KC>
__device__ __forceinline__ void load_tile(uint16_t (*dst)[SROW], const __nv_bfloat16* src, long long ld, int row0,
                                          int R, int k0, int K) {
    const uint16_t* s = reinterpret_cast<const uint16_t*>(src);
    const int tid = threadIdx.x;
    if (KC) {
        const bool vec = (ld % 8 == 0) && ((reinterpret_cast<uintptr_t>(s) & 15) == 0);
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int id = tid + i * 128, r = id >> 2, c8 = (id & 3) * 8;
            const int row = row0 + r, k = k0 + c8;
            if (vec && row < R && k + 8 <= K) {
                *reinterpret_cast<uint4*>(&dst[r][c8]) = *reinterpret_cast<const uint4*>(s + row * ld + k);
            } else {
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    dst[r][c8 + e] = (row < R && k + e < K) ? s[row * ld + k + e] : (uint16_t)0;
            }
        }
    } else {
#pragma unroll 4
        for (int i = 0; i < 16; ++i) {
            const int id = tid + i * 128, r = id & 63, c = id >> 6;
            const int row = row0 + r, k = k0 + c;
            dst[r][c] = (row < R && k < K) ? s[(long long)k * ld + row] : (uint16_t)0;
        }
    }
}

template <bool AK, bool BKc>
__global__ void __launch_bounds__(128) k_gemm(GemmArgs g) {
    __shared__ __align__(16) uint16_t As[BM][SROW];
    __shared__ __align__(16) uint16_t Bs[BN][SROW];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int wm = (w >> 1) * 32, wn = (w & 1) * 32;
    const int gq = lane >> 2, tq = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

    for (int k0 = 0; k0 < g.K; k0 += BK) {
        load_tile<AK>(As, g.A, g.lda, m0, g.M, k0, g.K);
        load_tile<BKc>(Bs, g.B, g.ldb, n0, g.N, k0, g.K);
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + gq;
                af[i][0] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * tq]);
                af[i][1] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * tq]);
                af[i][2] = *reinterpret_cast<const uint32_t*>(&As[r][kk + 2 * tq + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t*>(&As[r + 8][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int n = wn + j * 8 + gq;
                bf[j][0] = *reinterpret_cast<const uint32_t*>(&Bs[n][kk + 2 * tq]);
                bf[j][1] = *reinterpret_cast<const uint32_t*>(&Bs[n][kk + 2 * tq + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }
    // epilogue: acc[i][j][e] is C(m0 + wm + 16 i + gq + 8 (e >> 1), n0 + wn + 8 j + 2 tq + (e & 1))
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int m = m0 + wm + 16 * i + gq + 8 * (e >> 1);
                const int n = n0 + wn + 8 * j + 2 * tq + (e & 1);
                if (m >= g.M || n >= g.N) continue;
                const long long o = (long long)m * g.ldc + n;
                float v = acc[i][j][e];
                if (g.epi == EPI_BIAS_F32 || g.epi == EPI_BIAS_SILU) v += g.bias[n];
                if (g.epi == EPI_DSILU) v *= silu_grad_f(g.zprev[o]);
                if (g.outf) g.outf[o] = v;
                if (g.outh) g.outh[o] = __float2bfloat16_rn(g.epi == EPI_BIAS_SILU ? silu_f(v) : v);
            }
}

int gemm(const GemmArgs& g, bool ak, bool bk, cudaStream_t st) {
    dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM);
    if (ak && bk) k_gemm<true, true><<<grid, 128, 0, st>>>(g);
    else if (ak) k_gemm<true, false><<<grid, 128, 0, st>>>(g);
    else if (bk) k_gemm<false, true><<<grid, 128, 0, st>>>(g);
    else k_gemm<false, false><<<grid, 128, 0, st>>>(g);
    return launch_status("mlp gemm");
}

// rows idx[b] of the data set into the batch buffers
__global__ void k_gather(int B, const int32_t* __restrict__ idx, const uint4* __restrict__ X, const uint4* __restrict__ T,
                         uint4* __restrict__ Xb, uint4* __restrict__ Tb) {
    constexpr int XQ = DD_MLP_NIN * 2 / 16, TQ = DD_MLP_NOUT * 4 / 16;
    const int b = blockIdx.x;
    if (b >= B) return;
    const long long r = idx[b];
    for (int q = threadIdx.x; q < XQ; q += blockDim.x) Xb[(long long)b * XQ + q] = X[r * XQ + q];
    for (int q = threadIdx.x; q < TQ; q += blockDim.x) Tb[(long long)b * TQ + q] = T[r * TQ + q];
}

// weighted squared error: L = (1/B) sum w_j (y - t)^2, dL/dy in FP32 and BF16
__global__ void k_loss(int B, const float* __restrict__ Y, const float* __restrict__ T, const float* __restrict__ wt,
                       float* __restrict__ dYf, __nv_bfloat16* __restrict__ dYh, double* __restrict__ L) {
    const long long n = (long long)B * DD_MLP_NOUT;
    double s = 0.0;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const int j = (int)(q % DD_MLP_NOUT);
        const float d = Y[q] - T[q];
        s += (double)wt[j] * d * d;
        const float gq = 2.f * wt[j] * d / (float)B;
        dYf[q] = gq;
        dYh[q] = __float2bfloat16_rn(gq);
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
        atomicAdd(L, t / B);
    }
}

// column sums of G (M x N, FP32) into out[N]: the bias gradient
__global__ void k_colsum(int M, int N, const float* __restrict__ G, float* __restrict__ out) {
    __shared__ float red[8][33];
    const int n = blockIdx.x * 32 + threadIdx.x;
    float s = 0.f;
    if (n < N)
        for (int m = threadIdx.y; m < M; m += 8) s += G[(long long)m * N + n];
    red[threadIdx.y][threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.y == 0 && n < N) {
        float t = 0.f;
        for (int k = 0; k < 8; ++k) t += red[k][threadIdx.x];
        out[n] = t;
    }
}

// Adam (Kingma & Ba) on the flat parameters; refreshes the BF16 copy
__global__ void k_adam(long long n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ p16, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        const float pq = p[q] - lr * (mq / c1) / (sqrtf(vq / c2) + eps);
        p[q] = pq;
        p16[q] = __float2bfloat16_rn(pq);
    }
}

__global__ void k_to_bf16(long long n, const float* __restrict__ p, __nv_bfloat16* __restrict__ p16) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < n; q += (long long)gridDim.x * blockDim.x)
        p16[q] = __float2bfloat16_rn(p[q]);
}

}  // namespace

struct dd_mlp {
    int max_batch = 0;
    cudaStream_t stream = nullptr;
    int nsm = 0;
    float* p = nullptr;           // FP32 master parameters
    __nv_bfloat16* p16 = nullptr; // BF16 copy
    float* g = nullptr;           // gradient
    float* am = nullptr;          // Adam moments
    float* av = nullptr;
    long long step = 0;
    // activations (max_batch rows)
    __nv_bfloat16* xb = nullptr;  // gathered batch input
    float* tb = nullptr;          // gathered targets
    __nv_bfloat16* hh[kL] = {};   // layer inputs: hh[0] = input, hh[l] = SiLU(z_l)
    float* z[kL] = {};            // pre-activations of the hidden layers
    float* y = nullptr;           // output
    float* dzf[2] = {};           // gradient wrt pre-activations (ping-pong), FP32
    __nv_bfloat16* dzh[2] = {};   // and BF16
    double* dloss = nullptr;
    double* hloss = nullptr;      // pinned
};

namespace {

void mlp_free(dd_mlp* m) {
    void* ptrs[] = {m->p, m->p16, m->g, m->am, m->av, m->xb, m->tb, m->y, m->dzf[0], m->dzf[1], m->dzh[0], m->dzh[1],
                    m->dloss};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    for (int l = 0; l < kL; ++l) {
        if (m->hh[l]) cudaFree(m->hh[l]);
        if (m->z[l]) cudaFree(m->z[l]);
    }
    if (m->hloss) cudaFreeHost(m->hloss);
}

// forward pass of the rows x (M x NIN, BF16) into y (M x NOUT, FP32); keeps the
// hidden pre-activations when `train`
int forward(dd_mlp* m, const __nv_bfloat16* x, int M, float* y, bool train) {
    const __nv_bfloat16* in = x;
    for (int l = 0; l < kL; ++l) {
        GemmArgs g{};
        g.M = M; g.N = kDims[l + 1]; g.K = kDims[l];
        g.A = in; g.lda = kDims[l];
        g.B = m->p16 + w_off(l); g.ldb = kDims[l];
        g.bias = m->p + b_off(l);
        g.ldc = kDims[l + 1];
        if (l < kL - 1) {
            g.epi = EPI_BIAS_SILU;
            g.outf = train ? m->z[l + 1] : nullptr;
            g.outh = m->hh[l + 1];
        } else {
            g.epi = EPI_BIAS_F32;
            g.outf = y;
        }
        int r = gemm(g, true, true, m->stream);
        if (r != DD_OK) return r;
        if (l < kL - 1) in = m->hh[l + 1];
    }
    return DD_OK;
}

// loss and gradient of the batch (x, t) already in place; gradient into m->g
int backward(dd_mlp* m, const __nv_bfloat16* x, const float* t, const float* wt, int M) {
    const cudaStream_t st = m->stream;
    int r = forward(m, x, M, m->y, true);
    if (r != DD_OK) return r;
    if (cudaMemsetAsync(m->dloss, 0, sizeof(double), st) != cudaSuccess) return dd_record_cuda_error(cudaGetLastError(), "mlp memset");
    k_loss<<<2 * m->nsm, 256, 0, st>>>(M, m->y, t, wt, m->dzf[0], m->dzh[0], m->dloss);
    if ((r = launch_status("mlp loss")) != DD_OK) return r;
    int cur = 0;
    for (int l = kL - 1; l >= 0; --l) {
        const int K = kDims[l], N = kDims[l + 1];
        const __nv_bfloat16* hin = l == 0 ? x : m->hh[l];
        // dW_l (N x K) = dZ^T H: A(n, b) = dZ[b][n], B(k, b) = H[b][k]
        GemmArgs gw{};
        gw.M = N; gw.N = K; gw.K = M;
        gw.A = m->dzh[cur]; gw.lda = N;
        gw.B = hin; gw.ldb = K;
        gw.epi = EPI_F32; gw.outf = m->g + w_off(l); gw.ldc = K;
        if ((r = gemm(gw, false, false, st)) != DD_OK) return r;
        k_colsum<<<(N + 31) / 32, dim3(32, 8), 0, st>>>(M, N, m->dzf[cur], m->g + b_off(l));
        if ((r = launch_status("mlp colsum")) != DD_OK) return r;
        if (l == 0) break;
        // dZ_{l-1} (M x K) = (dZ W_l) * SiLU'(z_l): A = dZ (K-contiguous over n), B(k, n) = W[n][k]
        GemmArgs gx{};
        gx.M = M; gx.N = K; gx.K = N;
        gx.A = m->dzh[cur]; gx.lda = N;
        gx.B = m->p16 + w_off(l); gx.ldb = K;
        gx.epi = EPI_DSILU; gx.zprev = m->z[l];
        gx.outf = m->dzf[1 - cur]; gx.outh = m->dzh[1 - cur]; gx.ldc = K;
        if ((r = gemm(gx, true, false, st)) != DD_OK) return r;
        cur = 1 - cur;
    }
    return DD_OK;
}

}  // namespace

int mlp_forward_dev(dd_mlp* m, const uint16_t* x, int M, float* y, cudaStream_t st) {
    if (!m || M < 0 || M > m->max_batch) return DD_ERR_ARG;
    if (M == 0) return DD_OK;
    cudaStream_t keep = m->stream;
    m->stream = st;
    int r = forward(m, reinterpret_cast<const __nv_bfloat16*>(x), M, y, false);
    m->stream = keep;
    return r;
}

extern "C" {

int dd_mlp_create(int32_t max_batch, void* stream, dd_mlp** out) {
    if (!out || max_batch <= 0) return DD_ERR_ARG;
    *out = nullptr;
    dd_mlp* m = new (std::nothrow) dd_mlp();
    if (!m) return DD_ERR_OOM;
    m->max_batch = max_batch;
    m->stream = (cudaStream_t)stream;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&m->nsm, cudaDevAttrMultiProcessorCount, dev);
    const long long P = DD_MLP_NPARAMS, B = max_batch;
    bool ok = cudaMalloc(&m->p, P * 4) == cudaSuccess && cudaMalloc(&m->p16, P * 2) == cudaSuccess &&
              cudaMalloc(&m->g, P * 4) == cudaSuccess && cudaMalloc(&m->am, P * 4) == cudaSuccess &&
              cudaMalloc(&m->av, P * 4) == cudaSuccess && cudaMalloc(&m->xb, B * DD_MLP_NIN * 2) == cudaSuccess &&
              cudaMalloc(&m->tb, B * DD_MLP_NOUT * 4) == cudaSuccess && cudaMalloc(&m->y, B * DD_MLP_NOUT * 4) == cudaSuccess &&
              cudaMalloc(&m->dloss, sizeof(double)) == cudaSuccess &&
              cudaMallocHost(&m->hloss, sizeof(double)) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k)
        ok = cudaMalloc(&m->dzf[k], B * DD_MLP_NOUT * 4) == cudaSuccess &&
             cudaMalloc(&m->dzh[k], B * DD_MLP_NOUT * 2) == cudaSuccess;
    for (int l = 1; l < kL && ok; ++l)
        ok = cudaMalloc(&m->hh[l], B * kDims[l] * 2) == cudaSuccess && cudaMalloc(&m->z[l], B * kDims[l] * 4) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        mlp_free(m);
        delete m;
        return DD_ERR_OOM;
    }
    cudaMemsetAsync(m->p, 0, P * 4, m->stream);
    cudaMemsetAsync(m->p16, 0, P * 2, m->stream);
    cudaMemsetAsync(m->am, 0, P * 4, m->stream);
    cudaMemsetAsync(m->av, 0, P * 4, m->stream);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) {
        dd_record_cuda_error(cudaGetLastError(), "dd_mlp_create");
        mlp_free(m);
        delete m;
        return DD_ERR_CUDA;
    }
    *out = m;
    return DD_OK;
}

int dd_mlp_set_params(dd_mlp* m, const float* params, int64_t n) {
    if (!m || !params || n != DD_MLP_NPARAMS) return DD_ERR_ARG;
    cudaStream_t st = m->stream;
    if (cudaMemcpyAsync(m->p, params, n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return dd_record_cuda_error(cudaGetLastError(), "dd_mlp_set_params");
    cudaMemsetAsync(m->am, 0, n * 4, st);
    cudaMemsetAsync(m->av, 0, n * 4, st);
    m->step = 0;
    k_to_bf16<<<2 * m->nsm, 256, 0, st>>>(n, m->p, m->p16);
    int r = launch_status("mlp to_bf16");
    if (r != DD_OK) return r;
    return cudaStreamSynchronize(st) == cudaSuccess ? DD_OK : dd_record_cuda_error(cudaGetLastError(), "dd_mlp_set_params");
}

int dd_mlp_get_params(dd_mlp* m, float* params, int64_t n) {
    if (!m || !params || n != DD_MLP_NPARAMS) return DD_ERR_ARG;
    if (cudaMemcpyAsync(params, m->p, n * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
        cudaStreamSynchronize(m->stream) != cudaSuccess)
        return dd_record_cuda_error(cudaGetLastError(), "dd_mlp_get_params");
    return DD_OK;
}

int dd_mlp_forward(dd_mlp* m, const uint16_t* x_dev, int32_t M, float* y_dev) {
    if (!m || M < 0 || M > m->max_batch || (M > 0 && (!x_dev || !y_dev))) return DD_ERR_ARG;
    if (M == 0) return DD_OK;
    return forward(m, reinterpret_cast<const __nv_bfloat16*>(x_dev), M, y_dev, false);
}

int dd_mlp_loss_grad(dd_mlp* m, const uint16_t* x_dev, const float* t_dev, const float* w_dev, int32_t M,
                     double* loss, float* grad_host) {
    if (!m || !x_dev || !t_dev || !w_dev || M <= 0 || M > m->max_batch) return DD_ERR_ARG;
    int r = backward(m, reinterpret_cast<const __nv_bfloat16*>(x_dev), t_dev, w_dev, M);
    if (r != DD_OK) return r;
    if (cudaMemcpyAsync(m->hloss, m->dloss, sizeof(double), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
        return dd_record_cuda_error(cudaGetLastError(), "dd_mlp_loss_grad");
    if (grad_host &&
        cudaMemcpyAsync(grad_host, m->g, (size_t)DD_MLP_NPARAMS * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess)
        return dd_record_cuda_error(cudaGetLastError(), "dd_mlp_loss_grad");
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return dd_record_cuda_error(cudaGetLastError(), "dd_mlp_loss_grad");
    if (loss) *loss = *m->hloss;
    return DD_OK;
}

int dd_mlp_train_step(dd_mlp* m, const uint16_t* x_all, const float* t_all, const int32_t* idx, int32_t B,
                      const float* w_dev, float lr, double* loss) {
    if (!m || !x_all || !t_all || !idx || !w_dev || B <= 0 || B > m->max_batch || !(lr > 0.f)) return DD_ERR_ARG;
    const cudaStream_t st = m->stream;
    k_gather<<<B, 128, 0, st>>>(B, idx, reinterpret_cast<const uint4*>(x_all), reinterpret_cast<const uint4*>(t_all),
                                reinterpret_cast<uint4*>(m->xb), reinterpret_cast<uint4*>(m->tb));
    int r = launch_status("mlp gather");
    if (r != DD_OK) return r;
    if ((r = backward(m, m->xb, m->tb, w_dev, B)) != DD_OK) return r;
    m->step += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
    k_adam<<<2 * m->nsm, 256, 0, st>>>(DD_MLP_NPARAMS, m->p, m->g, m->am, m->av, m->p16, lr, b1, b2, 1e-8f, c1, c2);
    if ((r = launch_status("mlp adam")) != DD_OK) return r;
    if (loss) {
        if (cudaMemcpyAsync(m->hloss, m->dloss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return dd_record_cuda_error(cudaGetLastError(), "dd_mlp_train_step");
        *loss = *m->hloss;
    }
    return DD_OK;
}

void dd_mlp_destroy(dd_mlp* m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    mlp_free(m);
    delete m;
}

}  // extern "C"
