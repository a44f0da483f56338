// Learned surrogate: an MLP n_in -> H -> H -> n_out (SiLU) that maps the
// parameters of a magnetization family to its orientation-averaged log10 I(q),
// trained on data produced by the batched transform, with hand-written BF16
// kernels (FP32 accumulation, FP32 master weights, Adam).
//
// The paper has no learned component; here the exact transform generates
// the training targets and is the reference for the network's error.
//
// Kernels: for training, a BF16 tcgen05 GEMM (FP32 accumulation in TMEM)
// with the transposes the forward and backward passes need, plus
// element-wise SiLU / SiLU', MSE gradient, column sums for bias gradients,
// and Adam (the training GEMMs are small, B x 256 x 256); for inference, one
// fused tcgen05 kernel that runs the whole network per tile of 128 queries
// (k_mlp_infer).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>

#include <algorithm>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "nms.h"
#include "nms_internal.h"
#include "tc_ptx.cuh"

namespace nms {

// ------------------------------------------------------------------ GEMM
// C[m][n] (FP32, ldc) = sum_k A(m,k) B(n,k), A(m,k) = TA ? A[k*lda + m] :
// A[m*lda + k], B(n,k) = TB ? B[k*ldb + n] : B[n*ldb + k]; BF16 operands.
//
// On the 5th-generation tensor cores: one CTA of 8 warps per 128 x 128 tile
// of C.  For each 256-wide stretch of K the threads stage A and B into
// shared memory in the 128-byte-swizzled K-major layout (four k-blocks of 64
// per operand, 128 KB): every thread gathers 8 consecutive k of one row
// (one 16-byte load where the row is contiguous and aligned, 8 loads down a
// column where the operand is stored with K outermost; zero outside the
// matrix) and writes them as one 16-byte chunk.  One thread issues the
// tcgen05.mma (M = N = 128, K = 16, FP32 accumulation in 128 TMEM columns)
// and commits them to an mbarrier every thread waits on (bounded) before
// the buffers are reused; warp w reads TMEM lanes 32 (w mod 4) .. + 31 (rows
// of C), columns 64 (w / 4) .. + 63.  The training GEMMs are B x 256 x 256
// at most: a few CTAs, one or two K stretches.
constexpr int TG_BM = 128, TG_BN = 128, TG_BK = 64, TG_KB = 4, TG_THREADS = 256;
constexpr int TG_BLK = TG_BM * TG_BK * 2;              // 16 KB: one k-block of one operand
constexpr int TG_SMEM = 2 * TG_KB * TG_BLK + 1024;     // A and B, 4 k-blocks each

// 8 consecutive k (k0 .. k0 + 7) of row `row` as BF16x8, zero outside [0, R) x [0, K)
template <bool T>
__device__ __forceinline__ uint4 gather8(const __nv_bfloat16* __restrict__ P, int ld, int row, int R, int k0, int K)
{
    uint4 out = make_uint4(0u, 0u, 0u, 0u);
    if (row >= R) return out;
    if (!T && k0 + 8 <= K && (ld & 7) == 0 && ((reinterpret_cast<uintptr_t>(P) & 15) == 0))
        return *reinterpret_cast<const uint4*>(P + (int64_t)row * ld + k0);
    uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int k = k0 + e;
        if (k < K) {
            const __nv_bfloat16 v = T ? P[(int64_t)k * ld + row] : P[(int64_t)row * ld + k];
            w[e >> 1] |= (uint32_t)__bfloat16_as_ushort(v) << (16 * (e & 1));
        }
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

template <bool TA, bool TB>
__global__ void __launch_bounds__(TG_THREADS)
    k_mlp_gemm_tc(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda, const __nv_bfloat16* __restrict__ B,
                  int ldb, float* __restrict__ C, int ldc, int32_t* __restrict__ err, uint64_t limit_ns)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t s_taddr;
    __shared__ volatile int s_abort;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gA = smem_raw + (base - raw);
    uint8_t* gB = gA + TG_KB * TG_BLK;
    const uint32_t sA = base, sB = base + TG_KB * TG_BLK;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.y * TG_BM, n0 = blockIdx.x * TG_BN;
    if (tid == 0) {
        mbar_init(&bar, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tc_alloc<1>(smem_u32(&s_taddr), TG_BN);
        tc_relinquish<1>();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;
    const uint32_t idesc = idesc_bf16_f32(TG_BM, TG_BN);
    uint32_t phase = 0;
    bool aborted = false;
    for (int k0 = 0; k0 < K; k0 += TG_KB * TG_BK) {
        const int nkb = min(TG_KB, (K - k0 + TG_BK - 1) / TG_BK);
        // units: (k-block kb, row r, 8-wide chunk c); consecutive threads take
        // consecutive addresses of whichever index is contiguous in memory
        for (int u = tid; u < nkb * TG_BM * 8; u += TG_THREADS) {
            const int kb = u / (TG_BM * 8), v = u % (TG_BM * 8);
            const int r = TA ? v % TG_BM : v / 8, c = TA ? v / TG_BM : v % 8;
            const uint4 x = gather8<TA>(A, lda, m0 + r, M, k0 + kb * TG_BK + 8 * c, K);
            *reinterpret_cast<uint4*>(gA + kb * TG_BLK + swz_offset(r, 8 * c)) = x;
        }
        for (int u = tid; u < nkb * TG_BN * 8; u += TG_THREADS) {
            const int kb = u / (TG_BN * 8), v = u % (TG_BN * 8);
            const int r = TB ? v % TG_BN : v / 8, c = TB ? v / TG_BN : v % 8;
            const uint4 x = gather8<TB>(B, ldb, n0 + r, N, k0 + kb * TG_BK + 8 * c, K);
            *reinterpret_cast<uint4*>(gB + kb * TG_BLK + swz_offset(r, 8 * c)) = x;
        }
        fence_proxy_async_smem();
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            for (int kb = 0; kb < nkb; ++kb)
#pragma unroll
                for (int k16 = 0; k16 < 4; ++k16)
                    tc_mma_f16(taddr, sw128_desc(sA + kb * TG_BLK) + 2 * k16, sw128_desc(sB + kb * TG_BLK) + 2 * k16,
                               idesc, (k0 | kb | k16) ? 1u : 0u);
            tc_commit(&bar);
        }
        const bool ok = mbar_wait(&bar, phase, limit_ns, &s_abort);
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        phase ^= 1u;
        tc_fence_after();
    }
    if (!aborted) {
        const int quad = warp & 3, ch = warp >> 2;
        const int m = m0 + 32 * quad + lane;
#pragma unroll
        for (int c16 = 0; c16 < 4; ++c16) {
            float v[16];
            const int c0 = 64 * ch + 16 * c16;
            tmem_ld16(taddr + ((uint32_t)(32 * quad) << 16) + (uint32_t)c0, v);
            tmem_wait_ld();
            if (m < M) {
#pragma unroll
                for (int t = 0; t < 16; ++t) {
                    const int n = n0 + c0 + t;
                    if (n < N) C[(int64_t)m * ldc + n] = v[t];
                }
            }
        }
    } else if (tid == 0) {
        atomicExch(err, 2);
        // let the MMAs in flight finish (bounded) before TMEM is freed
        const uint64_t t0 = gtimer();
        while (!mbar_try_wait(&bar, phase) && gtimer() - t0 < 1000000000ull) {
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc<1>(taddr, TG_BN);
}

template <bool TA, bool TB>
static cudaError_t launch_gemm_tc(dim3 grid, int M, int N, int K, const __nv_bfloat16* A, int lda,
                                  const __nv_bfloat16* B, int ldb, float* C, int ldc, int32_t* err, cudaStream_t s)
{
    static bool attr = false;   // one-time opt-in to 129 KB of dynamic shared memory
    if (!attr) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_mlp_gemm_tc<TA, TB>, cudaFuncAttributeMaxDynamicSharedMemorySize, TG_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k_mlp_gemm_tc<TA, TB><<<grid, TG_THREADS, TG_SMEM, s>>>(M, N, K, A, lda, B, ldb, C, ldc, err, 4000000000ull);
    return cudaGetLastError();
}

static cudaError_t mlp_gemm(bool ta, bool tb, int M, int N, int K, const __nv_bfloat16* A, int lda,
                            const __nv_bfloat16* B, int ldb, float* C, int ldc, int32_t* err, cudaStream_t s)
{
    if (M <= 0 || N <= 0 || K <= 0) return cudaErrorInvalidValue;
    const dim3 grid((N + TG_BN - 1) / TG_BN, (M + TG_BM - 1) / TG_BM);
    if (!ta && !tb) return launch_gemm_tc<false, false>(grid, M, N, K, A, lda, B, ldb, C, ldc, err, s);
    if (!ta && tb) return launch_gemm_tc<false, true>(grid, M, N, K, A, lda, B, ldb, C, ldc, err, s);
    if (ta && !tb) return launch_gemm_tc<true, false>(grid, M, N, K, A, lda, B, ldb, C, ldc, err, s);
    return launch_gemm_tc<true, true>(grid, M, N, K, A, lda, B, ldb, C, ldc, err, s);
}

// ------------------------------------------------------------------ element-wise
__device__ __forceinline__ float silu(float z) { return z / (1.0f + expf(-z)); }

// SiLU with the fast exponential and the approximate division (two
// special-function operations; relative error a few FP32 ulp, and the
// result is rounded to BF16, 8 significant bits).  For z below about -88
// the denominator is infinite and the result is -0.
__device__ __forceinline__ float silu_fast(float z) { return __fdividef(z, 1.0f + __expf(-z)); }

// bf16x2 word of (a, b), a in the low half
__device__ __forceinline__ uint32_t bf16x2(float a, float b)
{
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// ------------------------------------------------------------------ fused inference
// Inference for H = 256, n_out <= 128 per launch, n_in <= 8 on the
// 5th-generation tensor cores, one kernel for the whole network.  A
// persistent CTA keeps W2 and W3 (BF16) in shared memory in the 128-byte
// swizzled K-major layout (160 or 192 KB: W3 for 64 or 128 outputs) and the
// activations in tensor memory,
// where the MMA reads them as its A operand (row m in lane m, two BF16 per
// 32-bit column).  Per tile of 128 queries:
//   layer 1 (threads, FP32):  H1 = bf16(silu(b1 + W1 xn))      -> TMEM Hb
//   layer 2 (tcgen05.mma):    D  = H1 W2^T   (128 x 256, FP32)  TMEM D
//   drain:                     H2 = bf16(silu(D + b2))          -> TMEM Hb
//   layer 3 (tcgen05.mma):    D  = H2 W3^T   (128 x n_out, FP32, D reused)
//   drain:                     Y  = (D + b3) ystd + ymean       -> global
// TMEM: D in columns 0-255, two activation buffers Hb[0], Hb[1] in 256-383
// and 384-511.  The layer-2 MMAs of tile i start as soon as tile i - 1's
// layer-3 accumulator has been read, and run under that tile's output
// stores and under layer 1 of tile i + 1, which the threads compute into the
// other buffer.  Warp w handles the rows
// 32 (w mod 4) .. + 31 (its TMEM lane quadrant) and the hidden units
// 32 (w / 4) .. + 31.  The arithmetic is that of the layer-by-layer path
// (BF16 operands, FP32 accumulation and activations); only the order of the
// FP32 sums differs.
constexpr int FI_THREADS = 1024;   // 32 warps (one per row of a 32-row output stage): the element-wise work needs many warps in flight
constexpr int FI_H = 256;
constexpr int FI_NO = 128;     // outputs per launch; W3 rows padded with zeros
constexpr int FI_TM = 128;     // queries per tile (the MMA's M)
constexpr int FI_W2_BYTES = 4 * FI_H * 128;   // 4 K-blocks of 256 rows x 128 B
constexpr uint32_t FI_HB = 256;               // TMEM column of activation buffer 0 (buffer 1: + 128)
// Dynamic shared memory after W2: W3 for 64 or 128 output rows, then the
// output stage (row stride odd: no bank conflicts).  With at most 64
// outputs the halved W3 leaves room to stage all 128 rows of a tile at once
// (one block barrier); otherwise 32 rows at a time.
__host__ __device__ constexpr int fi_w3_rows(int nout) { return nout <= 64 ? 64 : 128; }
__host__ __device__ constexpr int fi_stage_rows(int nout) { return nout <= 64 ? 128 : 32; }
__host__ __device__ constexpr int fi_smem(int nout)
{
    return FI_W2_BYTES + 4 * fi_w3_rows(nout) * 128 + fi_stage_rows(nout) * (fi_w3_rows(nout) + 1) * 4 + 1024;
}
static_assert(FI_THREADS == 32 * 32, "the 32-row output stage maps one warp to each row");

// Small per-launch tables in shared memory (read as warp-wide broadcasts):
// layer-1 weights padded to 8 inputs (with n_in < 8 the bias takes input
// slot 7, whose normalised input is 1), biases, the input normalisation
// xn = x * in_a + in_c, and the output map y = d * out_a + out_c.
struct FiSmall {
    float4 w1[FI_H][2];
    float b1[FI_H], b2[FI_H];
    float in_a[8], in_c[8];
    float out_a[FI_NO], out_c[FI_NO];
};

// layer 1 of one row for hidden units h0 .. h0 + 31, as 16 BF16 pairs
// (full8: n_in = 8, the bias is read separately)
__device__ __forceinline__ void fi_layer1(const float* xn, const FiSmall& sm, int h0, bool full8, uint32_t* w)
{
#pragma unroll 4
    for (int e = 0; e < 16; ++e) {
        float z[2];
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int h = h0 + 2 * e + t;
            const float4 u = sm.w1[h][0], v = sm.w1[h][1];
            float a0 = full8 ? sm.b1[h] : 0.f, a1 = 0.f;   // two chains of four
            a0 = fmaf(u.x, xn[0], a0);
            a1 = fmaf(v.x, xn[4], a1);
            a0 = fmaf(u.y, xn[1], a0);
            a1 = fmaf(v.y, xn[5], a1);
            a0 = fmaf(u.z, xn[2], a0);
            a1 = fmaf(v.z, xn[6], a1);
            a0 = fmaf(u.w, xn[3], a0);
            a1 = fmaf(v.w, xn[7], a1);
            z[t] = silu_fast(a0 + a1);
        }
        w[e] = bf16x2(z[0], z[1]);
    }
}

__global__ void __launch_bounds__(FI_THREADS, 1)
k_mlp_infer(int64_t n, int nin, int nout, int ystride, const float* __restrict__ X, const float* __restrict__ xlo,
            const float* __restrict__ xhi, const float* __restrict__ W1, const float* __restrict__ b1,
            const __nv_bfloat16* __restrict__ W2h, const float* __restrict__ b2, const __nv_bfloat16* __restrict__ W3h,
            const float* __restrict__ b3, const float* __restrict__ ymean, const float* __restrict__ ystd,
            float* __restrict__ Y, int32_t* __restrict__ err, uint64_t limit_ns)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_mma;
    __shared__ uint32_t s_taddr;
    __shared__ volatile int s_abort;
    __shared__ __align__(16) FiSmall sm;
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    uint8_t* gW2 = smem_raw + (base - raw);
    uint8_t* gW3 = gW2 + FI_W2_BYTES;
    const uint32_t sW2 = base, sW3 = base + FI_W2_BYTES;
    const int w3rows = fi_w3_rows(nout), srows = fi_stage_rows(nout), sstride = w3rows + 1;
    float* stag = reinterpret_cast<float*>(gW3 + 4 * w3rows * 128);   // srows x sstride
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    for (int h = tid; h < FI_H; h += FI_THREADS) {
        float w[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) w[i] = i < nin ? W1[h * nin + i] : 0.f;
        if (nin < 8) w[7] = b1[h];
        sm.w1[h][0] = make_float4(w[0], w[1], w[2], w[3]);
        sm.w1[h][1] = make_float4(w[4], w[5], w[6], w[7]);
        sm.b1[h] = b1[h];
        sm.b2[h] = b2[h];
    }
    if (tid < 8) {
        // xn = 2 (x - lo) / (hi - lo) - 1 as one FMA; inputs past n_in are
        // 0, except slot 7 (the bias) when n_in < 8
        const float a = tid < nin ? 2.0f / (xhi[tid] - xlo[tid]) : 0.f;
        sm.in_a[tid] = a;
        sm.in_c[tid] = tid < nin ? -fmaf(a, xlo[tid], 1.0f) : (tid == 7 ? 1.0f : 0.f);
    }
    for (int c = tid; c < FI_NO; c += FI_THREADS) {
        // y = (d + b3) ystd + ymean = d ystd + (b3 ystd + ymean)
        sm.out_a[c] = c < nout ? ystd[c] : 0.f;
        sm.out_c[c] = c < nout ? fmaf(b3[c], ystd[c], ymean[c]) : 0.f;
    }

    // W2 [256][256] and W3 [nout][256] (rows = outputs, K = inputs) into the
    // swizzled layout: K-block kb holds k in [64 kb, 64 kb + 64) of every row
    for (int u = tid; u < FI_H * 32; u += FI_THREADS) {
        const int r = u >> 5, j = u & 31, k = 8 * j;
        const uint4 v = reinterpret_cast<const uint4*>(W2h)[u];
        *reinterpret_cast<uint4*>(gW2 + (k >> 6) * (FI_H * 128) + swz_offset(r, k & 63)) = v;
    }
    for (int u = tid; u < w3rows * 32; u += FI_THREADS) {
        const int r = u >> 5, j = u & 31, k = 8 * j;
        const uint4 v = r < nout ? reinterpret_cast<const uint4*>(W3h)[u] : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(gW3 + (k >> 6) * (w3rows * 128) + swz_offset(r, k & 63)) = v;
    }
    if (tid == 0) {
        mbar_init(&bar_mma, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        tc_alloc<1>(smem_u32(&s_taddr), 512);
        tc_relinquish<1>();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;
    // layer 3 covers the outputs rounded up to the MMA's N granularity of 16
    const uint32_t id2 = idesc_bf16_f32(FI_TM, FI_H), id3 = idesc_bf16_f32(FI_TM, (nout + 15) & ~15);
    const int quad = warp & 3, cg = warp >> 2;        // TMEM lane quadrant, column group (0..7)
    const int row = 32 * quad + lane;                 // this thread's query row in the tile
    const uint32_t lanes = (uint32_t)(32 * quad) << 16;
    const int64_t ntiles = (n + FI_TM - 1) / FI_TM;
    // this thread's share of layer 1 for tile `tile` into buffer hb
    auto layer1 = [&](int64_t tile, uint32_t hb) {
        const int64_t q = tile * FI_TM + row;
        float xn[8];
#pragma unroll
        for (int i = 0; i < 8; ++i)
            xn[i] = (i < nin && q < n) ? fmaf(X[q * nin + i], sm.in_a[i], sm.in_c[i]) : sm.in_c[i];
        uint32_t w[16];
        fi_layer1(xn, sm, 32 * cg, nin == 8, w);
        tmem_st16(taddr + lanes + hb + 16u * (uint32_t)cg, w);
        tmem_wait_st();
    };
    // one thread issues the 16 K steps of a layer: D (+)= Hb x B^T
    auto mma_layer = [&](uint32_t hb, uint32_t sB, int brows, uint32_t idesc) {
        tc_fence_after();
#pragma unroll
        for (int kb = 0; kb < 4; ++kb)
#pragma unroll
            for (int k16 = 0; k16 < 4; ++k16)
                tc_mma_f16_ts(taddr, taddr + hb + (uint32_t)(8 * (4 * kb + k16)),
                              sw128_desc(sB + kb * (brows * 128)) + 2 * k16, idesc, (kb | k16) ? 1u : 0u);
        tc_commit(&bar_mma);
    };
    uint32_t phase = 0;
    bool aborted = false;
    // every thread waits for the MMAs committed last (bounded); false when
    // any thread of the block gave up
    auto wait_mma = [&]() {
        const bool ok = mbar_wait(&bar_mma, phase, limit_ns, &s_abort);
        const bool all = !__syncthreads_or(!ok);
        if (all) phase ^= 1u;
        return all;
    };
    int64_t tile = blockIdx.x;
    int buf = 0;
    if (tile < ntiles) {
        layer1(tile, FI_HB);
        tc_fence_before();
        __syncthreads();
        if (tid == 0) mma_layer(FI_HB, sW2, FI_H, id2);
    }
    for (; tile < ntiles; tile += gridDim.x, buf ^= 1) {
        const uint32_t hb = FI_HB + 128u * (uint32_t)buf, hn = FI_HB + 128u * (uint32_t)(buf ^ 1);
        const int64_t next = tile + gridDim.x;
        // layer 1 of the next tile into the other buffer, beside this tile's
        // layer-2 MMAs (that buffer's last reader, the previous tile's
        // layer-3 MMAs, has completed)
        if (next < ntiles) layer1(next, hn);
        if (!wait_mma()) {
            aborted = true;
            break;
        }
        tc_fence_after();
        // ---- drain D: bias, SiLU, BF16 into this tile's buffer (its
        // layer-2 MMAs, the buffer's readers, have completed)
        {
            float v[32];
            tmem_ld16(taddr + lanes + 32u * (uint32_t)cg, v);
            tmem_ld16(taddr + lanes + 32u * (uint32_t)cg + 16u, v + 16);
            tmem_wait_ld();
            uint32_t w[16];
            const float4* bb = reinterpret_cast<const float4*>(sm.b2 + 32 * cg);
#pragma unroll
            for (int e4 = 0; e4 < 8; ++e4) {
                const float4 b = bb[e4];
                w[2 * e4] = bf16x2(silu_fast(v[4 * e4] + b.x), silu_fast(v[4 * e4 + 1] + b.y));
                w[2 * e4 + 1] = bf16x2(silu_fast(v[4 * e4 + 2] + b.z), silu_fast(v[4 * e4 + 3] + b.w));
            }
            tmem_st16(taddr + lanes + hb + 16u * (uint32_t)cg, w);
            tmem_wait_st();
        }
        tc_fence_before();
        __syncthreads();
        // ---- layer 3 into D (columns 0 .. FI_NO - 1)
        if (tid == 0) mma_layer(hb, sW3, w3rows, id3);
        if (!wait_mma()) {
            aborted = true;
            break;
        }
        tc_fence_after();
        // ---- drain D: 16 output columns per warp, written out 32 rows at a
        // time through shared memory so that consecutive threads store
        // consecutive columns of a row (a warp's own values are 32 rows apart
        // in Y)
        {
            const int c0 = 16 * cg;
            const bool have = c0 < nout;   // the same for the whole warp
            float v[16];
            if (have) {
                tmem_ld16(taddr + lanes + (uint32_t)c0, v);
                tmem_wait_ld();
            }
            // D has been read: the next tile's layer-2 MMAs start now and run
            // under the output stores
            tc_fence_before();
            __syncthreads();
            if (next < ntiles && tid == 0) mma_layer(hn, sW2, FI_H, id2);
            if (srows == FI_TM) {
                // the whole tile at once; the stage is written again only
                // after the next tile's block barriers
                if (have)
#pragma unroll
                    for (int t = 0; t < 16; ++t) {
                        const int c = c0 + t;
                        if (c < nout) stag[row * sstride + c] = fmaf(v[t], sm.out_a[c], sm.out_c[c]);
                    }
                __syncthreads();
                for (int rr = warp; rr < FI_TM; rr += 32) {   // warp w writes rows w, w + 32, ...
                    const int64_t q = tile * FI_TM + rr;
                    if (q < n)
                        for (int c = lane; c < nout; c += 32) Y[q * ystride + c] = stag[rr * sstride + c];
                }
            } else {
                for (int qd = 0; qd < 4; ++qd) {
                    if (quad == qd && have) {
#pragma unroll
                        for (int t = 0; t < 16; ++t) {
                            const int c = c0 + t;
                            if (c < nout) stag[lane * sstride + c] = fmaf(v[t], sm.out_a[c], sm.out_c[c]);
                        }
                    }
                    __syncthreads();
                    // warp w writes staged row w, its lanes consecutive columns
                    const int64_t q = tile * FI_TM + 32 * qd + warp;
                    if (q < n)
                        for (int c = lane; c < nout; c += 32) Y[q * ystride + c] = stag[warp * sstride + c];
                    __syncthreads();
                }
            }
        }
    }
    if (aborted) {
        if (tid == 0) atomicExch(err, 1);
        // let the MMAs still in flight finish (bounded) before TMEM is freed
        if (tid == 0) {
            const uint64_t t0 = gtimer();
            while (!mbar_try_wait(&bar_mma, phase) && gtimer() - t0 < 1000000000ull) {
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tc_dealloc<1>(taddr, 512);
}
__device__ __forceinline__ float silu_grad(float z)
{
    const float s = 1.0f / (1.0f + expf(-z));
    return s * (1.0f + z * (1.0f - s));
}

// rows of X (FP32, raw) -> normalised input; layer 1 in FP32 (K = n_in is tiny)
__global__ void k_layer1(int B, int nin, int H, const float* __restrict__ X, const int32_t* __restrict__ perm,
                         const float* __restrict__ xlo, const float* __restrict__ xhi, const float* __restrict__ W1,
                         const float* __restrict__ b1, float* __restrict__ Xn, float* __restrict__ Z1,
                         __nv_bfloat16* __restrict__ H1)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)B * H) return;
    const int r = (int)(idx / H), h = (int)(idx % H);
    const int64_t src = perm ? perm[r] : r;
    float z = b1[h];
    for (int i = 0; i < nin; ++i) {
        const float xn = 2.0f * (X[src * nin + i] - xlo[i]) / (xhi[i] - xlo[i]) - 1.0f;
        if (h == 0) Xn[(int64_t)r * nin + i] = xn;
        z = fmaf(W1[h * nin + i], xn, z);
    }
    Z1[idx] = z;
    H1[idx] = __float2bfloat16(silu(z));
}

// Z = C + b (row-wise), H = bf16(silu(Z)) (act) or Y = Z (no act)
__global__ void k_bias_act(int B, int N, const float* __restrict__ C, const float* __restrict__ b, int act,
                           float* __restrict__ Z, __nv_bfloat16* __restrict__ H)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)B * N) return;
    const float z = C[idx] + b[idx % N];
    Z[idx] = z;
    if (act) H[idx] = __float2bfloat16(silu(z));
}

// dY = (Yn - Tn) / (B N) with Tn the standardised target; loss partial sums
__global__ void k_mse_grad(int B, int N, const float* __restrict__ Y, const float* __restrict__ T,
                           const int32_t* __restrict__ perm, const float* __restrict__ ymean,
                           const float* __restrict__ ystd, __nv_bfloat16* __restrict__ dY, float* __restrict__ dYf,
                           double* __restrict__ loss)
{
    __shared__ double red[256];
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (idx < (int64_t)B * N) {
        const int r = (int)(idx / N), o = (int)(idx % N);
        const int64_t src = perm ? perm[r] : r;
        const float t = (T[src * N + o] - ymean[o]) / ystd[o];
        const float d = Y[idx] - t;
        l = 0.5 * (double)d * (double)d;
        const float g = d / ((float)B * (float)N);
        dY[idx] = __float2bfloat16(g);
        dYf[idx] = g;
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, red[0]);
}

// dZ = dH * silu'(Z): BF16 copy for the next GEMM, FP32 copy for sums
__global__ void k_act_grad(int64_t n, const float* __restrict__ dH, const float* __restrict__ Z,
                           __nv_bfloat16* __restrict__ dZ, float* __restrict__ dZf)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n) return;
    const float g = dH[idx] * silu_grad(Z[idx]);
    if (dZ) dZ[idx] = __float2bfloat16(g);
    dZf[idx] = g;
}

// column sums: db[n] = sum_r G[r][n]
__global__ void k_col_sum(int B, int N, const float* __restrict__ G, float* __restrict__ db)
{
    const int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float acc = 0.f;
    for (int r = 0; r < B; ++r) acc += G[(int64_t)r * N + n];
    db[n] = acc;
}

// dW1[h][i] = sum_r dZ1[r][h] Xn[r][i] (FP32; K = batch)
__global__ void k_dw1(int B, int nin, int H, const float* __restrict__ dZ1, const float* __restrict__ Xn,
                      float* __restrict__ dW1)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= H * nin) return;
    const int h = idx / nin, i = idx % nin;
    float acc = 0.f;
    for (int r = 0; r < B; ++r) acc = fmaf(dZ1[(int64_t)r * H + h], Xn[(int64_t)r * nin + i], acc);
    dW1[idx] = acc;
}

__global__ void k_adam(int64_t n, float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_to_bf16(int64_t n, const float* __restrict__ a, __nv_bfloat16* __restrict__ b)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = __float2bfloat16(a[i]);
}

// de-normalise outputs: y = Yn * ystd + ymean
__global__ void k_denorm(int64_t n, int N, const float* __restrict__ Yn, const float* __restrict__ ymean,
                         const float* __restrict__ ystd, float* __restrict__ Y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) Y[i] = Yn[i] * ystd[i % N] + ymean[i % N];
}

// per-output mean and standard deviation of the targets (FP64 sums)
__global__ void k_target_stats(int64_t n, int N, const float* __restrict__ T, float* __restrict__ mean,
                               float* __restrict__ stdv)
{
    const int o = blockIdx.x;
    __shared__ double s1[256], s2[256];
    double a = 0.0, b = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += blockDim.x) {
        const double t = T[r * N + o];
        a += t;
        b += t * t;
    }
    s1[threadIdx.x] = a;
    s2[threadIdx.x] = b;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s1[threadIdx.x] += s1[threadIdx.x + w];
            s2[threadIdx.x] += s2[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mu = s1[0] / (double)n;
        const double var = fmax(s2[0] / (double)n - mu * mu, 1e-12);
        mean[o] = (float)mu;
        stdv[o] = (float)sqrt(var);
    }
}

}  // namespace nms

// ------------------------------------------------------------------ surrogate object
struct nms_surrogate_s {
    int nin = 0, H = 0, nout = 0;
    cudaStream_t stream = nullptr;
    int64_t nparam = 0;
    float* d_w = nullptr;      // master FP32: W1[H][nin] b1[H] W2[H][H] b2[H] W3[nout][H] b3[nout]
    float* d_g = nullptr;      // gradients, same layout
    float* d_m = nullptr;      // Adam moments
    float* d_v = nullptr;
    __nv_bfloat16* d_W2h = nullptr;
    __nv_bfloat16* d_W3h = nullptr;
    float* d_xlo = nullptr;
    float* d_xhi = nullptr;
    float* d_ymean = nullptr;
    float* d_ystd = nullptr;
    int64_t step = 0;
    // activations for a batch of capacity bcap
    int bcap = 0;
    float *d_Xn = nullptr, *d_Z1 = nullptr, *d_Z2 = nullptr, *d_Y = nullptr, *d_C = nullptr;
    float *d_dYf = nullptr, *d_dH = nullptr, *d_dZf = nullptr;
    __nv_bfloat16 *d_H1 = nullptr, *d_H2 = nullptr, *d_dY = nullptr, *d_dZ = nullptr;
    int32_t* d_perm = nullptr;
    int64_t perm_cap = 0;
    double* d_loss = nullptr;
    int32_t* d_err = nullptr;  // fused inference: a bounded wait gave up
    bool stats_set = false;
};

using namespace nms;

namespace {

float* W1p(nms_surrogate_s* s) { return s->d_w; }
float* b1p(nms_surrogate_s* s) { return s->d_w + (int64_t)s->H * s->nin; }
float* W2p(nms_surrogate_s* s) { return b1p(s) + s->H; }
float* b2p(nms_surrogate_s* s) { return W2p(s) + (int64_t)s->H * s->H; }
float* W3p(nms_surrogate_s* s) { return b2p(s) + s->H; }
float* b3p(nms_surrogate_s* s) { return W3p(s) + (int64_t)s->nout * s->H; }
int64_t off_b1(const nms_surrogate_s* s) { return (int64_t)s->H * s->nin; }
int64_t off_W2(const nms_surrogate_s* s) { return off_b1(s) + s->H; }
int64_t off_b2(const nms_surrogate_s* s) { return off_W2(s) + (int64_t)s->H * s->H; }
int64_t off_W3(const nms_surrogate_s* s) { return off_b2(s) + s->H; }
int64_t off_b3(const nms_surrogate_s* s) { return off_W3(s) + (int64_t)s->nout * s->H; }

unsigned nb(int64_t n) { return (unsigned)((n + 255) / 256); }

nms_status ensure_batch(nms_surrogate_s* s, int B)
{
    if (B <= s->bcap) return NMS_OK;
    void* bufs[] = {s->d_Xn, s->d_Z1, s->d_Z2, s->d_Y, s->d_C, s->d_dYf, s->d_dH, s->d_dZf, s->d_H1, s->d_H2, s->d_dY,
                    s->d_dZ};
    for (void* b : bufs)
        if (b) cudaFree(b);
    const int64_t w = std::max(s->H, s->nout);
    NMS_CUDA_TRY(cudaMalloc(&s->d_Xn, (size_t)B * s->nin * 4));
    NMS_CUDA_TRY(cudaMalloc(&s->d_Z1, (size_t)B * s->H * 4));
    NMS_CUDA_TRY(cudaMalloc(&s->d_Z2, (size_t)B * s->H * 4));
    NMS_CUDA_TRY(cudaMalloc(&s->d_Y, (size_t)B * s->nout * 4));
    NMS_CUDA_TRY(cudaMalloc(&s->d_C, (size_t)B * w * 4));
    NMS_CUDA_TRY(cudaMalloc(&s->d_dYf, (size_t)B * s->nout * 4));
    NMS_CUDA_TRY(cudaMalloc(&s->d_dH, (size_t)B * s->H * 4));
    NMS_CUDA_TRY(cudaMalloc(&s->d_dZf, (size_t)B * s->H * 4));
    NMS_CUDA_TRY(cudaMalloc(&s->d_H1, (size_t)B * s->H * 2));
    NMS_CUDA_TRY(cudaMalloc(&s->d_H2, (size_t)B * s->H * 2));
    NMS_CUDA_TRY(cudaMalloc(&s->d_dY, (size_t)B * s->nout * 2));
    NMS_CUDA_TRY(cudaMalloc(&s->d_dZ, (size_t)B * s->H * 2));
    s->bcap = B;
    return NMS_OK;
}

nms_status refresh_bf16(nms_surrogate_s* s)
{
    const int64_t n2 = (int64_t)s->H * s->H, n3 = (int64_t)s->nout * s->H;
    k_to_bf16<<<nb(n2), 256, 0, s->stream>>>(n2, W2p(s), s->d_W2h);
    k_to_bf16<<<nb(n3), 256, 0, s->stream>>>(n3, W3p(s), s->d_W3h);
    NMS_CUDA_TRY(cudaGetLastError());
    return NMS_OK;
}

// forward on rows perm[0..B) (or 0..B) of X; output normalised Y in d_Y
nms_status forward(nms_surrogate_s* s, const float* X, const int32_t* perm, int B)
{
    cudaStream_t st = s->stream;
    const int H = s->H, O = s->nout;
    k_layer1<<<nb((int64_t)B * H), 256, 0, st>>>(B, s->nin, H, X, perm, s->d_xlo, s->d_xhi, W1p(s), b1p(s), s->d_Xn,
                                                 s->d_Z1, s->d_H1);
    NMS_CUDA_TRY(cudaGetLastError());
    NMS_CUDA_TRY(mlp_gemm(false, false, B, H, H, s->d_H1, H, s->d_W2h, H, s->d_C, H, s->d_err, st));
    k_bias_act<<<nb((int64_t)B * H), 256, 0, st>>>(B, H, s->d_C, b2p(s), 1, s->d_Z2, s->d_H2);
    NMS_CUDA_TRY(cudaGetLastError());
    NMS_CUDA_TRY(mlp_gemm(false, false, B, O, H, s->d_H2, H, s->d_W3h, H, s->d_C, O, s->d_err, st));
    k_bias_act<<<nb((int64_t)B * O), 256, 0, st>>>(B, O, s->d_C, b3p(s), 0, s->d_Y, nullptr);
    NMS_CUDA_TRY(cudaGetLastError());
    return NMS_OK;
}

// backward after forward: gradients into d_g (overwritten), loss added to d_loss
nms_status backward(nms_surrogate_s* s, const float* T, const int32_t* perm, int B)
{
    cudaStream_t st = s->stream;
    const int H = s->H, O = s->nout, nin = s->nin;
    float* g = s->d_g;
    k_mse_grad<<<nb((int64_t)B * O), 256, 0, st>>>(B, O, s->d_Y, T, perm, s->d_ymean, s->d_ystd, s->d_dY, s->d_dYf,
                                                    s->d_loss);
    NMS_CUDA_TRY(cudaGetLastError());
    // layer 3: dW3 = dY^T H2, db3 = colsum dY, dH2 = dY W3
    NMS_CUDA_TRY(mlp_gemm(true, true, O, H, B, s->d_dY, O, s->d_H2, H, g + off_W3(s), H, s->d_err, st));
    k_col_sum<<<nb(O), 256, 0, st>>>(B, O, s->d_dYf, g + off_b3(s));
    NMS_CUDA_TRY(mlp_gemm(false, true, B, H, O, s->d_dY, O, s->d_W3h, H, s->d_dH, H, s->d_err, st));
    // layer 2
    k_act_grad<<<nb((int64_t)B * H), 256, 0, st>>>((int64_t)B * H, s->d_dH, s->d_Z2, s->d_dZ, s->d_dZf);
    NMS_CUDA_TRY(cudaGetLastError());
    NMS_CUDA_TRY(mlp_gemm(true, true, H, H, B, s->d_dZ, H, s->d_H1, H, g + off_W2(s), H, s->d_err, st));
    k_col_sum<<<nb(H), 256, 0, st>>>(B, H, s->d_dZf, g + off_b2(s));
    NMS_CUDA_TRY(mlp_gemm(false, true, B, H, H, s->d_dZ, H, s->d_W2h, H, s->d_dH, H, s->d_err, st));
    // layer 1 (FP32)
    k_act_grad<<<nb((int64_t)B * H), 256, 0, st>>>((int64_t)B * H, s->d_dH, s->d_Z1, nullptr, s->d_dZf);
    k_dw1<<<nb((int64_t)H * nin), 256, 0, st>>>(B, nin, H, s->d_dZf, s->d_Xn, g);
    k_col_sum<<<nb(H), 256, 0, st>>>(B, H, s->d_dZf, g + off_b1(s));
    NMS_CUDA_TRY(cudaGetLastError());
    return NMS_OK;
}

}  // namespace

extern "C" {

nms_status nms_surrogate_create(nms_surrogate_t* out, int32_t n_in, int32_t n_hidden, int32_t n_out,
                                const float* x_lo, const float* x_hi, uint64_t seed, void* cuda_stream)
{
    set_error("");
    if (!out) return NMS_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_in < 1 || n_in > 64 || n_hidden < 8 || n_hidden > 4096 || n_out < 1 || n_out > 4096 || !x_lo || !x_hi) {
        set_error("surrogate: need 1 <= n_in <= 64, 8 <= n_hidden <= 4096, 1 <= n_out <= 4096 and input bounds");
        return NMS_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n_in; ++i)
        if (!(x_hi[i] > x_lo[i])) {
            set_error("surrogate: x_hi must exceed x_lo");
            return NMS_ERR_INVALID_ARG;
        }
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
        cudaGetLastError();
        set_error("no CUDA device available (libnms has no CPU fallback)");
        return NMS_ERR_CUDA;
    }
    nms_surrogate_s* s = new nms_surrogate_s();
    s->nin = n_in;
    s->H = n_hidden;
    s->nout = n_out;
    s->stream = (cudaStream_t)cuda_stream;
    s->nparam = (int64_t)n_hidden * n_in + n_hidden + (int64_t)n_hidden * n_hidden + n_hidden +
                (int64_t)n_out * n_hidden + n_out;
    // He-style uniform initialisation from a seeded host generator
    std::vector<float> w(s->nparam, 0.f);
    std::mt19937_64 rng(seed);
    auto fill = [&](int64_t off, int64_t n, int fan_in) {
        const double a = sqrt(6.0 / fan_in);
        std::uniform_real_distribution<double> u(-a, a);
        for (int64_t i = 0; i < n; ++i) w[off + i] = (float)u(rng);
    };
    fill(0, (int64_t)n_hidden * n_in, n_in);
    fill(off_W2(s), (int64_t)n_hidden * n_hidden, n_hidden);
    fill(off_W3(s), (int64_t)n_out * n_hidden, n_hidden);
    std::vector<float> ones(n_out, 1.f), zeros(n_out, 0.f);
    auto bail = [&](nms_status st) {
        nms_surrogate_destroy(s);
        return st;
    };
    if (cudaMalloc(&s->d_w, s->nparam * 4) || cudaMalloc(&s->d_g, s->nparam * 4) ||
        cudaMalloc(&s->d_m, s->nparam * 4) || cudaMalloc(&s->d_v, s->nparam * 4) ||
        cudaMalloc(&s->d_W2h, (size_t)n_hidden * n_hidden * 2) || cudaMalloc(&s->d_W3h, (size_t)n_out * n_hidden * 2) ||
        cudaMalloc(&s->d_xlo, n_in * 4) || cudaMalloc(&s->d_xhi, n_in * 4) || cudaMalloc(&s->d_ymean, n_out * 4) ||
        cudaMalloc(&s->d_ystd, n_out * 4) || cudaMalloc(&s->d_loss, 8) || cudaMalloc(&s->d_err, 4)) {
        cudaGetLastError();
        set_error("surrogate: device allocation failed");
        return bail(NMS_ERR_OUT_OF_MEMORY);
    }
    cudaMemcpy(s->d_w, w.data(), s->nparam * 4, cudaMemcpyHostToDevice);
    cudaMemset(s->d_m, 0, s->nparam * 4);
    cudaMemset(s->d_v, 0, s->nparam * 4);
    cudaMemset(s->d_g, 0, s->nparam * 4);
    cudaMemcpy(s->d_xlo, x_lo, n_in * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(s->d_xhi, x_hi, n_in * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(s->d_ymean, zeros.data(), n_out * 4, cudaMemcpyHostToDevice);
    cudaMemcpy(s->d_ystd, ones.data(), n_out * 4, cudaMemcpyHostToDevice);
    nms_status st = refresh_bf16(s);
    if (st) return bail(st);
    if (cudaDeviceSynchronize() != cudaSuccess) return bail(cuda_fail(cudaGetLastError(), "surrogate init"));
    *out = s;
    return NMS_OK;
}

nms_status nms_surrogate_set_target_stats(nms_surrogate_t s, const float* y_mean, const float* y_std)
{
    set_error("");
    if (!s || !y_mean || !y_std) return NMS_ERR_INVALID_ARG;
    for (int o = 0; o < s->nout; ++o)
        if (!(y_std[o] > 0)) {
            set_error("surrogate: y_std must be > 0");
            return NMS_ERR_INVALID_ARG;
        }
    NMS_CUDA_TRY(cudaMemcpy(s->d_ymean, y_mean, s->nout * 4, cudaMemcpyHostToDevice));
    NMS_CUDA_TRY(cudaMemcpy(s->d_ystd, y_std, s->nout * 4, cudaMemcpyHostToDevice));
    s->stats_set = true;
    return NMS_OK;
}

nms_status nms_surrogate_train(nms_surrogate_t s, const float* X, const float* Y, int64_t n, int32_t batch,
                               int32_t epochs, float lr, uint64_t shuffle_seed, float* final_loss)
{
    set_error("");
    if (!s || !X || !Y || n < 1 || batch < 1 || epochs < 0 || !(lr > 0)) {
        set_error("surrogate train: bad arguments");
        return NMS_ERR_INVALID_ARG;
    }
    if (n > INT32_MAX) {
        set_error("surrogate train: n too large");
        return NMS_ERR_INVALID_ARG;
    }
    const int B = (int)std::min<int64_t>(batch, n);
    nms_status st = ensure_batch(s, B);
    if (st) return st;
    if (!s->stats_set) {
        k_target_stats<<<s->nout, 256, 0, s->stream>>>(n, s->nout, Y, s->d_ymean, s->d_ystd);
        NMS_CUDA_TRY(cudaGetLastError());
        s->stats_set = true;
    }
    if (n > s->perm_cap) {
        if (s->d_perm) cudaFree(s->d_perm);
        NMS_CUDA_TRY(cudaMalloc(&s->d_perm, n * sizeof(int32_t)));
        s->perm_cap = n;
    }
    std::vector<int32_t> perm(n);
    std::mt19937_64 rng(shuffle_seed);
    double last = 0.0;
    NMS_CUDA_TRY(cudaMemsetAsync(s->d_err, 0, 4, s->stream));
    for (int e = 0; e < epochs; ++e) {
        for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
        std::shuffle(perm.begin(), perm.end(), rng);
        NMS_CUDA_TRY(cudaMemcpyAsync(s->d_perm, perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s->stream));
        NMS_CUDA_TRY(cudaMemsetAsync(s->d_loss, 0, 8, s->stream));
        for (int64_t b0 = 0; b0 + B <= n; b0 += B) {
            if ((st = forward(s, X, s->d_perm + b0, B))) return st;
            if ((st = backward(s, Y, s->d_perm + b0, B))) return st;
            ++s->step;
            const float b1 = 0.9f, b2 = 0.999f;
            const float c1 = 1.f - powf(b1, (float)s->step), c2 = 1.f - powf(b2, (float)s->step);
            k_adam<<<nb(s->nparam), 256, 0, s->stream>>>(s->nparam, s->d_w, s->d_g, s->d_m, s->d_v, lr, b1, b2, 1e-8f,
                                                          c1, c2);
            NMS_CUDA_TRY(cudaGetLastError());
            if ((st = refresh_bf16(s))) return st;
        }
        double h = 0.0;
        int32_t herr = 0;
        NMS_CUDA_TRY(cudaMemcpyAsync(&h, s->d_loss, 8, cudaMemcpyDeviceToHost, s->stream));
        NMS_CUDA_TRY(cudaMemcpyAsync(&herr, s->d_err, 4, cudaMemcpyDeviceToHost, s->stream));
        NMS_CUDA_TRY(cudaStreamSynchronize(s->stream));
        if (herr) {
            set_error("surrogate train: a tensor-core GEMM's bounded wait gave up");
            return NMS_ERR_TIMEOUT;
        }
        last = h / (double)((n / B) * (int64_t)B * s->nout);
    }
    if (final_loss) *final_loss = (float)last;
    return NMS_OK;
}

nms_status nms_surrogate_gradients(nms_surrogate_t s, const float* X, const float* Y, int32_t n, float* grad,
                                   double* loss)
{
    set_error("");
    if (!s || !X || !Y || n < 1 || !grad) return NMS_ERR_INVALID_ARG;
    nms_status st = ensure_batch(s, n);
    if (st) return st;
    NMS_CUDA_TRY(cudaMemsetAsync(s->d_loss, 0, 8, s->stream));
    NMS_CUDA_TRY(cudaMemsetAsync(s->d_err, 0, 4, s->stream));
    if ((st = forward(s, X, nullptr, n))) return st;
    if ((st = backward(s, Y, nullptr, n))) return st;
    NMS_CUDA_TRY(cudaMemcpyAsync(grad, s->d_g, s->nparam * 4, cudaMemcpyDeviceToHost, s->stream));
    double h = 0.0;
    int32_t herr = 0;
    NMS_CUDA_TRY(cudaMemcpyAsync(&h, s->d_loss, 8, cudaMemcpyDeviceToHost, s->stream));
    NMS_CUDA_TRY(cudaMemcpyAsync(&herr, s->d_err, 4, cudaMemcpyDeviceToHost, s->stream));
    NMS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    if (herr) {
        set_error("surrogate gradients: a tensor-core GEMM's bounded wait gave up");
        return NMS_ERR_TIMEOUT;
    }
    if (loss) *loss = h / ((double)n * s->nout);
    return NMS_OK;
}

nms_status nms_surrogate_infer(nms_surrogate_t s, const float* X, int64_t n, float* Y)
{
    set_error("");
    if (!s || !X || !Y || n < 0) return NMS_ERR_INVALID_ARG;
    if (n == 0) return NMS_OK;
    if (s->H == FI_H && s->nout <= 2 * FI_NO && s->nin <= 8) {
        // the whole network in one tensor-core kernel per 128 outputs (W2 and
        // W3 fill the shared memory; more outputs run the hidden layers
        // again for the further 128)
        static bool attr = false;
        if (!attr) {
            NMS_CUDA_TRY(cudaFuncSetAttribute(k_mlp_infer, cudaFuncAttributeMaxDynamicSharedMemorySize, fi_smem(FI_NO)));
            attr = true;
        }
        NMS_CUDA_TRY(cudaMemsetAsync(s->d_err, 0, 4, s->stream));
        const int64_t tiles = (n + FI_TM - 1) / FI_TM;
        const int grid = (int)std::min<int64_t>(tiles, device_sm_count());
        for (int o0 = 0; o0 < s->nout; o0 += FI_NO) {
            const int part = std::min(FI_NO, s->nout - o0);
            k_mlp_infer<<<grid, FI_THREADS, fi_smem(part), s->stream>>>(
                n, s->nin, part, s->nout, X, s->d_xlo, s->d_xhi, W1p(s), b1p(s), s->d_W2h, b2p(s),
                s->d_W3h + (int64_t)o0 * FI_H, b3p(s) + o0, s->d_ymean + o0, s->d_ystd + o0, Y + o0, s->d_err,
                4000000000ull);
            NMS_CUDA_TRY(cudaGetLastError());
        }
        int32_t herr = 0;
        NMS_CUDA_TRY(cudaMemcpyAsync(&herr, s->d_err, 4, cudaMemcpyDeviceToHost, s->stream));
        NMS_CUDA_TRY(cudaStreamSynchronize(s->stream));
        if (herr) {
            set_error("surrogate inference: a bounded device wait gave up");
            return NMS_ERR_TIMEOUT;
        }
        return NMS_OK;
    }
    const int B = 65536;
    nms_status st = ensure_batch(s, (int)std::min<int64_t>(B, std::max<int64_t>(n, 1)));
    if (st) return st;
    for (int64_t b0 = 0; b0 < n; b0 += s->bcap) {
        const int nb_ = (int)std::min<int64_t>(s->bcap, n - b0);
        if ((st = forward(s, X + b0 * s->nin, nullptr, nb_))) return st;
        k_denorm<<<nb((int64_t)nb_ * s->nout), 256, 0, s->stream>>>((int64_t)nb_ * s->nout, s->nout, s->d_Y, s->d_ymean,
                                                                     s->d_ystd, Y + b0 * s->nout);
        NMS_CUDA_TRY(cudaGetLastError());
    }
    return NMS_OK;
}

nms_status nms_surrogate_get_params(nms_surrogate_t s, float* host, int64_t* count)
{
    set_error("");
    if (!s) return NMS_ERR_INVALID_ARG;
    if (count) *count = s->nparam;
    if (host) {
        NMS_CUDA_TRY(cudaStreamSynchronize(s->stream));
        NMS_CUDA_TRY(cudaMemcpy(host, s->d_w, s->nparam * 4, cudaMemcpyDeviceToHost));
    }
    return NMS_OK;
}

nms_status nms_surrogate_set_params(nms_surrogate_t s, const float* host, int64_t count)
{
    set_error("");
    if (!s || !host || count != s->nparam) {
        set_error("surrogate: parameter count mismatch");
        return NMS_ERR_INVALID_ARG;
    }
    NMS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    NMS_CUDA_TRY(cudaMemcpy(s->d_w, host, s->nparam * 4, cudaMemcpyHostToDevice));
    return refresh_bf16(s);
}

// Checkpoint: header, master weights, Adam moments, target statistics.
nms_status nms_surrogate_save(nms_surrogate_t s, const char* path)
{
    set_error("");
    if (!s || !path) return NMS_ERR_INVALID_ARG;
    std::vector<float> w(s->nparam), m(s->nparam), v(s->nparam), ym(s->nout), ys(s->nout), xl(s->nin), xh(s->nin);
    NMS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    NMS_CUDA_TRY(cudaMemcpy(w.data(), s->d_w, s->nparam * 4, cudaMemcpyDeviceToHost));
    NMS_CUDA_TRY(cudaMemcpy(m.data(), s->d_m, s->nparam * 4, cudaMemcpyDeviceToHost));
    NMS_CUDA_TRY(cudaMemcpy(v.data(), s->d_v, s->nparam * 4, cudaMemcpyDeviceToHost));
    NMS_CUDA_TRY(cudaMemcpy(ym.data(), s->d_ymean, s->nout * 4, cudaMemcpyDeviceToHost));
    NMS_CUDA_TRY(cudaMemcpy(ys.data(), s->d_ystd, s->nout * 4, cudaMemcpyDeviceToHost));
    NMS_CUDA_TRY(cudaMemcpy(xl.data(), s->d_xlo, s->nin * 4, cudaMemcpyDeviceToHost));
    NMS_CUDA_TRY(cudaMemcpy(xh.data(), s->d_xhi, s->nin * 4, cudaMemcpyDeviceToHost));
    FILE* f = fopen(path, "wb");
    if (!f) {
        set_error(std::string("cannot open ") + path);
        return NMS_ERR_INVALID_ARG;
    }
    const char magic[8] = {'N', 'M', 'S', 'S', 'U', 'R', '0', '1'};
    int64_t hdr[5] = {s->nin, s->H, s->nout, s->step, s->stats_set ? 1 : 0};
    bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, 8, 5, f) == 5 &&
              fwrite(w.data(), 4, s->nparam, f) == (size_t)s->nparam && fwrite(m.data(), 4, s->nparam, f) == (size_t)s->nparam &&
              fwrite(v.data(), 4, s->nparam, f) == (size_t)s->nparam && fwrite(ym.data(), 4, s->nout, f) == (size_t)s->nout &&
              fwrite(ys.data(), 4, s->nout, f) == (size_t)s->nout && fwrite(xl.data(), 4, s->nin, f) == (size_t)s->nin &&
              fwrite(xh.data(), 4, s->nin, f) == (size_t)s->nin;
    fclose(f);
    if (!ok) {
        set_error("short write");
        return NMS_ERR_INVALID_ARG;
    }
    return NMS_OK;
}

nms_status nms_surrogate_load(nms_surrogate_t s, const char* path)
{
    set_error("");
    if (!s || !path) return NMS_ERR_INVALID_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) {
        set_error(std::string("cannot open ") + path);
        return NMS_ERR_INVALID_ARG;
    }
    char magic[8];
    int64_t hdr[5];
    bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "NMSSUR01", 8) == 0 && fread(hdr, 8, 5, f) == 5 &&
              hdr[0] == s->nin && hdr[1] == s->H && hdr[2] == s->nout;
    std::vector<float> w(s->nparam), m(s->nparam), v(s->nparam), ym(s->nout), ys(s->nout), xl(s->nin), xh(s->nin);
    if (ok)
        ok = fread(w.data(), 4, s->nparam, f) == (size_t)s->nparam && fread(m.data(), 4, s->nparam, f) == (size_t)s->nparam &&
             fread(v.data(), 4, s->nparam, f) == (size_t)s->nparam && fread(ym.data(), 4, s->nout, f) == (size_t)s->nout &&
             fread(ys.data(), 4, s->nout, f) == (size_t)s->nout && fread(xl.data(), 4, s->nin, f) == (size_t)s->nin &&
             fread(xh.data(), 4, s->nin, f) == (size_t)s->nin;
    fclose(f);
    if (!ok) {
        set_error("not a surrogate checkpoint of this shape");
        return NMS_ERR_INVALID_ARG;
    }
    NMS_CUDA_TRY(cudaStreamSynchronize(s->stream));
    NMS_CUDA_TRY(cudaMemcpy(s->d_w, w.data(), s->nparam * 4, cudaMemcpyHostToDevice));
    NMS_CUDA_TRY(cudaMemcpy(s->d_m, m.data(), s->nparam * 4, cudaMemcpyHostToDevice));
    NMS_CUDA_TRY(cudaMemcpy(s->d_v, v.data(), s->nparam * 4, cudaMemcpyHostToDevice));
    NMS_CUDA_TRY(cudaMemcpy(s->d_ymean, ym.data(), s->nout * 4, cudaMemcpyHostToDevice));
    NMS_CUDA_TRY(cudaMemcpy(s->d_ystd, ys.data(), s->nout * 4, cudaMemcpyHostToDevice));
    NMS_CUDA_TRY(cudaMemcpy(s->d_xlo, xl.data(), s->nin * 4, cudaMemcpyHostToDevice));
    NMS_CUDA_TRY(cudaMemcpy(s->d_xhi, xh.data(), s->nin * 4, cudaMemcpyHostToDevice));
    s->step = hdr[3];
    s->stats_set = hdr[4] != 0;
    return refresh_bf16(s);
}

nms_status nms_surrogate_destroy(nms_surrogate_t s)
{
    if (!s) return NMS_OK;
    cudaStreamSynchronize(s->stream);
    void* bufs[] = {s->d_w, s->d_g, s->d_m, s->d_v, s->d_W2h, s->d_W3h, s->d_xlo, s->d_xhi, s->d_ymean, s->d_ystd,
                    s->d_Xn, s->d_Z1, s->d_Z2, s->d_Y, s->d_C, s->d_dYf, s->d_dH, s->d_dZf, s->d_H1, s->d_H2,
                    s->d_dY, s->d_dZ, s->d_perm, s->d_loss, s->d_err};
    for (void* b : bufs)
        if (b) cudaFree(b);
    delete s;
    return NMS_OK;
}

}  // extern "C"
