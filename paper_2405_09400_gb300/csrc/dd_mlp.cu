// The learned warm start's network on the GPU: a multilayer perceptron
// 336 -> 256 -> 256 -> 256 -> 320 (SiLU on the hidden layers, linear output)
// with BF16 weights and activations and FP32 accumulation, and its training
// (backpropagation, Adam). Not in the paper: it predicts the X dual that
// initialises each composite-cell Sinkhorn solve (alpha_init of Alg. 1 / Alg. 4).
//
// Every layer product is one tensor-core GEMM kernel,
//   C(m, n) = sum_k A(m, k) B(n, k),
// with a fused epilogue (bias, SiLU, SiLU' of the next layer down, FP32/BF16
// stores). The forward products (A = activations, B = weights, both K
// contiguous) run on k_gemm_tc: TMA loads into 128-byte-swizzled shared memory,
// tcgen05.mma with the accumulator in tensor memory, tcgen05.ld epilogue. The
// two gradient products of the backward pass (dW = dZ^T H, dH = dZ W), whose
// operands are not all K-contiguous, run on k_gemm: tiles of 64 x 64 x 32 staged
// in shared memory and warp-level mma.sync m16n8k16 BF16 -> FP32, which also
// serves as the reference the forward kernel is tested against
// (dd_mlp_set_gemm).
//
// Parameters: one flat FP32 vector (master copy), W_1 (256 x 336, row n = the
// weights into output n), b_1, W_2, b_2, W_3, b_3, W_4 (320 x 256), b_4; a BF16
// copy of the same vector feeds the GEMMs; biases are read in FP32.
#include <cuda.h>  // CUtensorMap and its enums (declarations only; the encoder is looked up at run time)
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

// ---------------------------------------------------------------------------
// Forward products on the fifth-generation tensor cores: C = A B^T with A
// (M x K) and B (N x K) both K-contiguous BF16, FP32 accumulation in tensor
// memory. One CTA of 4 warps computes a 128 x 64 tile of C:
//  * thread 0 issues one TMA load (cp.async.bulk.tensor, 128-byte swizzle,
//    zero fill outside the matrix) per 64-wide K block of A and of B, all at
//    once (K <= 384: the whole K extent is resident, 24 KB per block), each
//    block on its own mbarrier;
//  * as each block lands, the same thread issues four tcgen05.mma (M = 128,
//    N = 64, K = 16) into a 64-column TMEM accumulator, then tcgen05.commit
//    arrives on a completion mbarrier;
//  * every warp reads its 32 TMEM lanes (rows) back with tcgen05.ld and applies
//    the epilogue (bias, SiLU, FP32 / BF16 stores) in registers.
// Every wait is bounded (~1 s of %globaltimer): on a timeout the kernel sets
// *err, waits (bounded) for its copies still in flight, frees its TMEM and
// returns without storing.
constexpr int TC_BM = 128, TC_BN = 64, TC_BK = 64, TC_KB_MAX = 6;
constexpr int TC_A_BYTES = TC_BM * TC_BK * 2, TC_B_BYTES = TC_BN * TC_BK * 2;
constexpr int TC_TMEM_COLS = 64;  // FP32 accumulator columns (power of two >= 32)
// instruction descriptor of kind::f16: D FP32 (bits 4-5), A and B BF16 (bits
// 7-9, 10-12), both K-major (bits 15, 16 zero), N >> 3 (bits 17-22), M >> 4 (bits 24-28)
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(TC_BM >> 4) << 24);

constexpr size_t tc_smem_bytes(int nkb) { return 1024 + (size_t)nkb * (TC_A_BYTES + TC_B_BYTES) + 8 * (TC_KB_MAX + 1) + 16; }

struct TcArgs {
    int M, N, nkb, epi;
    const float* bias;
    float* outf;
    __nv_bfloat16* outh;
    long long ldc;
    int* err;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for phase `parity` of the barrier; false after ~1 s without it
__device__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_test(bar, parity))
        if (global_ns() - t0 > 1000000000ull) return false;
    return true;
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int x, int y) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(bar), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1 (bits 46-48)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(128, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap tA, const __grid_constant__ CUtensorMap tB, TcArgs g) {
    extern __shared__ __align__(1024) uint8_t tc_smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * TC_BN, nkb = g.nkb;
    // tiles on 1024-byte boundaries (the swizzle pattern repeats every 8 rows of 128 bytes)
    const uint32_t raw = smem_addr(tc_smem), base = (raw + 1023u) & ~1023u;
    const uint32_t sA = base, sB = sA + nkb * TC_A_BYTES, sBar = sB + nkb * TC_B_BYTES, sDone = sBar + 8 * TC_KB_MAX;
    uint8_t* tail = tc_smem + (sDone + 8 - raw);
    volatile uint32_t* slot = reinterpret_cast<volatile uint32_t*>(tail);  // TMEM address from tcgen05.alloc
    volatile int* fail = reinterpret_cast<volatile int*>(tail + 4);
    if (tid == 0) {
        for (int kb = 0; kb < nkb; ++kb) mbar_init(sBar + 8 * kb, 1);
        mbar_init(sDone, 1);
        *fail = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr((const void*)slot)),
                     "r"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *slot;
    int issued = 0;  // K blocks whose loads thread 0 issued
    if (tid == 0) {
        for (int kb = 0; kb < nkb; ++kb) {
            mbar_expect_tx(sBar + 8 * kb, TC_A_BYTES + TC_B_BYTES);
            tma_load_2d(sA + kb * TC_A_BYTES, &tA, sBar + 8 * kb, kb * TC_BK, m0);
            tma_load_2d(sB + kb * TC_B_BYTES, &tB, sBar + 8 * kb, kb * TC_BK, n0);
            issued = kb + 1;
        }
        bool ok = true;
        for (int kb = 0; kb < nkb && ok; ++kb) {
            ok = mbar_wait(sBar + 8 * kb, 0);
            if (!ok) break;
            tc_fence_after();
#pragma unroll
            for (int j = 0; j < TC_BK / 16; ++j)  // K steps of 16: 32 bytes along the swizzled row
                umma_bf16(tmem, sw128_desc(sA + kb * TC_A_BYTES + 32 * j), sw128_desc(sB + kb * TC_B_BYTES + 32 * j),
                          (kb | j) != 0);
        }
        if (ok) {
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(sDone)
                         : "memory");
        } else {
            *fail = 1;
            atomicExch(g.err, 1);
            mbar_arrive(sDone);
        }
    }
    __syncwarp();
    const bool done = mbar_wait(sDone, 0);
    tc_fence_after();
    if (!done) {
        if (lane == 0) atomicExch(g.err, 1);
    } else if (!*fail) {
        // rows of this warp: TMEM lanes 32 warp .. 32 warp + 31
        const int m = m0 + 32 * warp + lane;
        const uint32_t trow = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll 1
        for (int c = 0; c < TC_BN / 16; ++c) {
            uint32_t r[16];
            tmem_ld16(trow + 16 * c, r);
            const int nb = n0 + 16 * c;
            if (m >= g.M || nb >= g.N) continue;
            float v[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                v[e] = __uint_as_float(r[e]);
                if (g.epi == EPI_BIAS_F32 || g.epi == EPI_BIAS_SILU) v[e] += g.bias[min(nb + e, g.N - 1)];
            }
            const long long o = (long long)m * g.ldc + nb;
            if (nb + 16 <= g.N) {
                if (g.outf) {
                    float4* q = reinterpret_cast<float4*>(g.outf + o);
#pragma unroll
                    for (int e = 0; e < 4; ++e) q[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
                }
                if (g.outh) {
                    uint32_t h[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float a = g.epi == EPI_BIAS_SILU ? silu_f(v[2 * e]) : v[2 * e];
                        const float b = g.epi == EPI_BIAS_SILU ? silu_f(v[2 * e + 1]) : v[2 * e + 1];
                        const __nv_bfloat162 p = __floats2bfloat162_rn(a, b);
                        h[e] = *reinterpret_cast<const uint32_t*>(&p);
                    }
                    uint4* q = reinterpret_cast<uint4*>(g.outh + o);
                    q[0] = make_uint4(h[0], h[1], h[2], h[3]);
                    q[1] = make_uint4(h[4], h[5], h[6], h[7]);
                }
            } else {
#pragma unroll
                for (int e = 0; e < 16; ++e) {
                    if (nb + e >= g.N) continue;
                    if (g.outf) g.outf[o + e] = v[e];
                    if (g.outh) g.outh[o + e] = __float2bfloat16_rn(g.epi == EPI_BIAS_SILU ? silu_f(v[e]) : v[e]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (tid == 0 && *fail)  // copies still in flight land before the CTA's shared memory is released
        for (int kb = 0; kb < issued; ++kb) mbar_wait(sBar + 8 * kb, 0);
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
    }
}

using TensorMapEncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                       const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                       CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// the driver's tensor-map encoder, looked up once through the runtime
TensorMapEncodeFn tensor_map_encoder() {
    static TensorMapEncodeFn fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        return reinterpret_cast<TensorMapEncodeFn>(p);
    }();
    return fn;
}

// rows x K BF16 matrix, row stride ld elements, read in boxes of 64 (K) x box_rows
bool encode_kmajor(CUtensorMap* map, const __nv_bfloat16* p, int rows, int K, long long ld, int box_rows) {
    const TensorMapEncodeFn fn = tensor_map_encoder();
    if (!fn) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TC_BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(p), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

// whether C = A B^T (both K-contiguous) can run on k_gemm_tc: the whole K extent
// resident, TMA-legal bases and row strides, vector-aligned epilogue stores
bool tc_eligible(const GemmArgs& g) {
    return g.M > 0 && g.N > 0 && g.K > 0 && g.K <= TC_KB_MAX * TC_BK && g.epi != EPI_DSILU && aligned16(g.A) &&
           aligned16(g.B) && g.lda % 8 == 0 && g.ldb % 8 == 0 && g.lda >= g.K && g.ldb >= g.K && g.ldc >= g.N && g.ldc % 8 == 0 &&
           (!g.outf || aligned16(g.outf)) && (!g.outh || aligned16(g.outh));
}

int gemm_tc(const GemmArgs& g, int* err, cudaStream_t st) {
    static const bool attr = [] {
        return cudaFuncSetAttribute(k_gemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes(TC_KB_MAX)) ==
               cudaSuccess;
    }();
    if (!attr) return dd_record_cuda_error(cudaGetLastError(), "mlp gemm (tensor memory): shared-memory attribute");
    CUtensorMap ta, tb;
    if (!encode_kmajor(&ta, g.A, g.M, g.K, g.lda, TC_BM) || !encode_kmajor(&tb, g.B, g.N, g.K, g.ldb, TC_BN))
        return dd_record_cuda_error(cudaErrorInvalidValue, "mlp gemm (tensor memory): tensor map");
    TcArgs a{};
    a.M = g.M; a.N = g.N; a.nkb = (g.K + TC_BK - 1) / TC_BK; a.epi = g.epi;
    a.bias = g.bias; a.outf = g.outf; a.outh = g.outh; a.ldc = g.ldc; a.err = err;
    dim3 grid((g.N + TC_BN - 1) / TC_BN, (g.M + TC_BM - 1) / TC_BM);
    k_gemm_tc<<<grid, 128, tc_smem_bytes(a.nkb), st>>>(ta, tb, a);
    return launch_status("mlp gemm (tensor memory)");
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
    int* d_err = nullptr;         // set by k_gemm_tc when a wait timed out
    int gemm_kind = DD_MLP_GEMM_UMMA;
};

namespace {

void mlp_free(dd_mlp* m) {
    void* ptrs[] = {m->p, m->p16, m->g, m->am, m->av, m->xb, m->tb, m->y, m->dzf[0], m->dzf[1], m->dzh[0], m->dzh[1],
                    m->dloss, m->d_err};
    for (void* q : ptrs)
        if (q) cudaFree(q);
    for (int l = 0; l < kL; ++l) {
        if (m->hh[l]) cudaFree(m->hh[l]);
        if (m->z[l]) cudaFree(m->z[l]);
    }
    if (m->hloss) cudaFreeHost(m->hloss);
}

// forward pass of the rows x (M x NIN, BF16) into y (M x NOUT, FP32); keeps the
// hidden pre-activations when `train`; a timed-out wait of k_gemm_tc sets *err
int forward(dd_mlp* m, const __nv_bfloat16* x, int M, float* y, bool train, int* err) {
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
        int r;
        if (m->gemm_kind == DD_MLP_GEMM_MMA) r = gemm(g, true, true, m->stream);
        else if (tc_eligible(g)) r = gemm_tc(g, err, m->stream);
        else r = DD_ERR_ARG;  // a base or row stride the tensor maps cannot take
        if (r != DD_OK) return r;
        if (l < kL - 1) in = m->hh[l + 1];
    }
    return DD_OK;
}

// loss and gradient of the batch (x, t) already in place; gradient into m->g
int backward(dd_mlp* m, const __nv_bfloat16* x, const float* t, const float* wt, int M) {
    const cudaStream_t st = m->stream;
    int r = forward(m, x, M, m->y, true, m->d_err);
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

// after a synchronisation of the network's stream: DD_ERR_CUDA (and the flag
// cleared) if a k_gemm_tc wait timed out since the last check
int take_err(dd_mlp* m) {
    int e = 0;
    if (cudaMemcpy(&e, m->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return dd_record_cuda_error(cudaGetLastError(), "mlp error flag");
    if (!e) return DD_OK;
    cudaMemset(m->d_err, 0, sizeof(int));
    return dd_record_cuda_error(cudaErrorLaunchTimeout, "mlp gemm (tensor memory): a wait timed out");
}

}  // namespace

int mlp_forward_dev(dd_mlp* m, const uint16_t* x, int M, float* y, cudaStream_t st, int* err) {
    if (!m || M < 0 || M > m->max_batch) return DD_ERR_ARG;
    if (M == 0) return DD_OK;
    cudaStream_t keep = m->stream;
    m->stream = st;
    int r = forward(m, reinterpret_cast<const __nv_bfloat16*>(x), M, y, false, err ? err : m->d_err);
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
              cudaMalloc(&m->dloss, sizeof(double)) == cudaSuccess && cudaMalloc(&m->d_err, sizeof(int)) == cudaSuccess &&
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
    cudaMemsetAsync(m->d_err, 0, sizeof(int), m->stream);
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
    return take_err(m);
}

int dd_mlp_set_gemm(dd_mlp* m, int32_t kind) {
    if (!m || (kind != DD_MLP_GEMM_UMMA && kind != DD_MLP_GEMM_MMA)) return DD_ERR_ARG;
    m->gemm_kind = kind;
    return DD_OK;
}

int dd_mlp_forward(dd_mlp* m, const uint16_t* x_dev, int32_t M, float* y_dev) {
    if (!m || M < 0 || M > m->max_batch || (M > 0 && (!x_dev || !y_dev))) return DD_ERR_ARG;
    if (M == 0) return DD_OK;
    return forward(m, reinterpret_cast<const __nv_bfloat16*>(x_dev), M, y_dev, false, m->d_err);
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
    if ((r = take_err(m)) != DD_OK) return r;
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
        if ((r = take_err(m)) != DD_OK) return r;
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
