// Tensor-core path: the Fourier sum on a separable (Cartesian) detector grid
// as a split-FP16 real GEMM on tcgen05 (sm_103a).
//
// Paper, Sec. "Summation approach": F_c(q) = sum_j w_cj exp(-i q.r_j).  On the
// detector plane q = (0, q_y, q_z) the phase separates,
//   exp(-i (q_y Y + q_z Z)) = exp(-i q_y Y) exp(-i q_z Z),
// and with alpha = q_y Y_j, beta = q_z Z_j the four real sums
//   cc = sum_j w_cj cos(alpha) cos(beta)     cs = sum_j w_cj cos(alpha) sin(beta)
//   sc = sum_j w_cj sin(alpha) cos(beta)     ss = sum_j w_cj sin(alpha) sin(beta)
// give F_c(s_y q_y, s_z q_z) = (cc - s_y s_z ss) - i (s_z cs + s_y sc) for both
// signs s_y, s_z = +-1: cos is even and sin odd in q.  The GEMM is
//   D = A B^T,  A[2 (nch a + c) + p, j] = w_cj {cos, sin}_p(q_y,a Y_j),
//               B[2 b + r, j]           = {cos, sin}_r(q_z,b Z_j),
// K = cells, so D holds (cc, cs) in row p = 0 and (sc, ss) in row p = 1 of
// each (a, c).  On a detector axis that is symmetric about q = 0 (lo = -hi)
// the GEMM covers only the q >= 0 half of that axis and the epilogue writes
// both signs: a grid symmetric in q_y and q_z costs a quarter of the MMA work
// and 10 instead of 24 table bytes per cell and pixel pair (512^2 grid),
// with the same per-term arithmetic.  An asymmetric axis is covered in full
// and only the s = +1 combination is written.  When both axes are symmetric
// the -q_z half is not written at all: with real weights F(-q) = conj F(q),
// and the readers of the amplitudes take it from the q_z >= 0 half.
//
// Precision (GB300-specific choice): each operand x (scaled by a power of two
// to |x| <= 2^12) is split x = hi + lo with hi = fp16(x), lo = fp16(x - hi);
// three kind::f16 MMAs per K step give hi*hi (accumulator D0) and
// hi*lo + lo*hi (accumulator D1), a per-product error of ~3 * 2^-22 -- the
// precision of TF32x3 at the FP16 tensor rate.  FP32 accumulation in TMEM is
// limited to kc cells at a time: the accumulators are double-buffered and
// drained by 16 epilogue warps into two-float (hi, lo) registers.  Each
// chunk partial D0 + D1 is added to lo with one FP32 add and (hi, lo) is
// renormalised by TwoSum every TC_RENORM chunks, so lo holds at most a few
// chunk partials and its rounding stays far below the TMEM accumulation
// error.
//
// Phase tables use the two-float phase in turns t = q'.r (q' = q/2 pi) with
// the exact reduction t - rint(t), then sincospif.  Tables are written in the
// canonical K-major 128-byte-swizzled UMMA layout, 16 KB per (tile, k-block),
// so the GEMM moves them with plain 1D bulk copies (cp.async.bulk).
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "nms_internal.h"
#include "tc_ptx.cuh"

namespace nms {

constexpr int TC_BM = 128;          // rows of A per tile: 64 (q_y, channel) pairs x (cos, sin)
constexpr int TC_BN = 128;          // rows of B per tile: 64 q_z values x (cos, sin)
constexpr int TC_BK = 64;           // k per block = cells per block, one 128-byte swizzle row
constexpr int TC_BLOCK_BYTES = TC_BM * TC_BK * 2;   // 16 KB
constexpr int TC_STAGES = 3;
constexpr int TC_STAGE_BYTES = 4 * TC_BLOCK_BYTES;  // A_hi, A_lo, B_hi, B_lo
constexpr int TC_THREADS = 576;     // warp 0 producer, warp 1 MMA, warps 2..17 epilogue
constexpr int TC_EPI_WARPS = 16;    // 4 per TMEM lane quadrant, 32 accumulator columns each
#ifndef TC_RENORM
#define TC_RENORM 4                 // 0: TwoSum per chunk; G > 0: chunk partials add into lo, TwoSum every G chunks
#endif
#ifndef TC_DRAIN_W
#define TC_DRAIN_W 8                // accumulator columns per tcgen05.ld in the drain (4, 8 or 16)
#endif
constexpr float TC_SCALE = 4096.0f; // operand scale 2^12

// ------------------------------------------------------------------ tables
// Tables cover a list of k-blocks; k-block kb holds the cells
// [kb_cell0[kb], kb_cell0[kb] + kb_ncell[kb]) (kb_ncell <= 64) of the stacked
// per-rotation cell arrays, the rest of the block is zero padding.
__device__ __forceinline__ float turns_reduced(float2 q, float xh, float xl)
{
    // two-float product q' * coordinate (turns) reduced to [-1/2, 1/2]
    float p = q.x * xh;
    float e = fmaf(q.x, xh, -p) + fmaf(q.x, xl, q.y * xh);
    float n = rintf(p);
    return (p - n) + e;
}

// sin and cos of the phase 2 pi q x of a two-float node q (turns per unit
// length, passed as q4 = 4 q: scaling by 4 is exact) and a two-float
// coordinate x, for the fused ray form, where these values set the pace.
// The product in quarter turns p + e = q4 x (p = fl(q4.x x.h), e its error
// and the low parts) is split at the nearest quarter turn n = rint(p), the
// remainder r = (p - n) + e (p - n exact, Sterbenz; |r| <= 1/2 up to |e|)
// gives sin and cos of (pi/2) r by their Taylor series about 0 (odd terms
// to r^9, even terms to r^10: truncation below 2e-9 for |(pi/2) r| <= pi/4),
// and the quadrant n mod 4 swaps and negates them.  Coefficients are
// (pi/2)^k / k! rounded once to FP32, times the power of two SCALE (exact:
// the results come out scaled by SCALE at no cost).  Error about one unit in
// the last place (checked against exact values and sincospif).
template <int SCALE = 1>
__device__ __forceinline__ void sincos_node(float2 q4, float xh, float xl, float& sn, float& cs)
{
    static_assert(SCALE > 0 && (SCALE & (SCALE - 1)) == 0, "SCALE must be a power of two");
    constexpr double H = 1.5707963267948966192313216916398;   // pi / 2
    constexpr float K = (float)SCALE;
    constexpr float S1 = K * (float)H;
    constexpr float S3 = K * (float)(-H * H * H / 6.0);
    constexpr float S5 = K * (float)(H * H * H * H * H / 120.0);
    constexpr float S7 = K * (float)(-H * H * H * H * H * H * H / 5040.0);
    constexpr float S9 = K * (float)(H * H * H * H * H * H * H * H * H / 362880.0);
    constexpr float C2 = K * (float)(-H * H / 2.0);
    constexpr float C4 = K * (float)(H * H * H * H / 24.0);
    constexpr float C6 = K * (float)(-H * H * H * H * H * H / 720.0);
    constexpr float C8 = K * (float)(H * H * H * H * H * H * H * H / 40320.0);
    constexpr float C10 = K * (float)(-H * H * H * H * H * H * H * H * H * H / 3628800.0);
    const float p = q4.x * xh;
    const float e = fmaf(q4.x, xh, -p) + fmaf(q4.x, xl, q4.y * xh);
    const float qn = rintf(p);
    const float r = (p - qn) + e;
    const int n = (int)qn;
    const float r2 = r * r;
    float ps = fmaf(S9, r2, S7);
    ps = fmaf(ps, r2, S5);
    ps = fmaf(ps, r2, S3);
    ps = fmaf(ps, r2, S1);
    const float sr = ps * r;
    float pc = fmaf(C10, r2, C8);
    pc = fmaf(pc, r2, C6);
    pc = fmaf(pc, r2, C4);
    pc = fmaf(pc, r2, C2);
    const float cr = fmaf(pc, r2, K);
    // quadrant n: (sin, cos) = (s, c), (c, -s), (-s, -c), (-c, s)
    const bool swap = n & 1;
    const float a = swap ? cr : sr, b = swap ? sr : cr;
    sn = (n & 2) ? -a : a;
    cs = ((n + 1) & 2) ? -b : b;
}

// (x0, x1) -> hi = fp16x2(x0, x1), lo = fp16x2(x0 - hi.x, x1 - hi.y); x0 in
// the low half (the lower k index)
__device__ __forceinline__ void split_h2(float x0, float x1, uint32_t& h, uint32_t& l)
{
    const __half2 hh = __floats2half2_rn(x0, x1);
    const float2 f = __half22float2(hh);
    const __half2 ll = __floats2half2_rn(x0 - f.x, x1 - f.y);
    h = *reinterpret_cast<const uint32_t*>(&hh);
    l = *reinterpret_cast<const uint32_t*>(&ll);
}

// four consecutive k of one row: hi and lo halves as 8-byte words
__device__ __forceinline__ void split4(float x0, float x1, float x2, float x3, uint2& h, uint2& l)
{
    split_h2(x0, x1, h.x, l.x);
    split_h2(x2, x3, h.y, l.y);
}

// The tables are written one k-block (64 cells) per block of 256 threads:
// the cells' positions and weights are loaded once per k-block and every A
// and B row of that k-block is computed from them.  Thread t holds the
// cells 4 (t & 15) .. + 3 (one 8-byte half of a 16-byte swizzle chunk) and
// takes the row groups t / 16 + 16 i, so the 16 threads of a half-warp write
// one whole 128-byte row per store.  Stores are streaming (evict-first): a
// chunk's tables are read back by the GEMM only after the whole chunk is
// written.
constexpr int TAB_THREADS = 256;

// A tables: block (mt, kb) holds rows m = mt*128 + r, r < 128, with
// m = 2 (nch a + c) + p (GEMM q_y index a, channel c = 4 * set + {N, Mx, My,
// Mz}, p = cos/sin) and k = cell of the block.  A row group g is the 8 rows
// 8g..8g+7: one q_y node a and one weight set (g = spad a + set, spad =
// nch / 4).  Weight set st of cell j is cw[st * wstride + j].
//
// B tables: block (nt, kb) holds rows n = nt*128 + 2 b_loc + r, b_loc < 64,
// r = cos/sin of q_z,b Z_j.
__global__ void __launch_bounds__(TAB_THREADS, 3)
k_tables(const float4* __restrict__ cpos, const float4* __restrict__ cw, int64_t wstride, int nch,
         const int64_t* __restrict__ kb_cell0, const int32_t* __restrict__ kb_ncell, const float2* __restrict__ qy,
         int nyg, const float2* __restrict__ qz, int nzg, float4 wscale, int64_t nkb, int mtiles, int ntiles,
         uint8_t* __restrict__ A_hi, uint8_t* __restrict__ A_lo, uint8_t* __restrict__ B_hi,
         uint8_t* __restrict__ B_lo)
{
    const int r = threadIdx.x >> 4;
    const int q4 = threadIdx.x & 15;
    const int k0 = 4 * q4;                          // first cell of this thread in the k-block
    const int spad = nch >> 2;                      // weight sets per output (a power of two)
    // row group g = r + 16 i has weight set g mod spad: one set per thread
    // when spad <= 16, else spad / 16 passes over i with one set each
    const int passes = spad > 16 ? spad / 16 : 1;
    const int ngroups = mtiles * 16;
    const int nb = ntiles * 64;
    for (int64_t kb = blockIdx.x; kb < nkb; kb += gridDim.x) {
        const int64_t c0 = kb_cell0[kb];
        const int nc = kb_ncell[kb];
        float4 cp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cp[u] = k0 + u < nc ? cpos[c0 + k0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
        // ---- B rows; padding cells and rows stay zero
        for (int bi = r; bi < nb; bi += 16) {
            const int nt = bi >> 6, b_loc = bi & 63;
            const bool brow = bi < nzg;
            const float2 q = brow ? qz[bi] : make_float2(0.f, 0.f);
            float cs[4], sn[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float live = (brow && k0 + u < nc) ? TC_SCALE : 0.f;
                sincospif(2.0f * turns_reduced(q, cp[u].z, cp[u].w), &sn[u], &cs[u]);
                cs[u] *= live;
                sn[u] *= live;
            }
            uint2 ch, cl, sh, sl;
            split4(cs[0], cs[1], cs[2], cs[3], ch, cl);
            split4(sn[0], sn[1], sn[2], sn[3], sh, sl);
            const size_t blk = ((size_t)nt * nkb + kb) * TC_BLOCK_BYTES;
            const uint32_t oc = swz_offset(2 * b_loc, k0);
            const uint32_t os = swz_offset(2 * b_loc + 1, k0);
            __stcs(reinterpret_cast<uint2*>(B_hi + blk + oc), ch);
            __stcs(reinterpret_cast<uint2*>(B_lo + blk + oc), cl);
            __stcs(reinterpret_cast<uint2*>(B_hi + blk + os), sh);
            __stcs(reinterpret_cast<uint2*>(B_lo + blk + os), sl);
        }
        // ---- A rows, one weight set per pass
        for (int ps = 0; ps < passes; ++ps) {
            const int st = (r + 16 * ps) & (spad - 1);
            const float4* wset = cw + (int64_t)st * wstride;
            float4 w[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float4 v = k0 + u < nc ? wset[c0 + k0 + u] : make_float4(0.f, 0.f, 0.f, 0.f);
                w[u] = make_float4(v.x * wscale.x, v.y * wscale.y, v.z * wscale.z, v.w * wscale.w);
            }
            for (int g = r + 16 * ps; g < ngroups; g += 16 * passes) {
                const int a = g / spad;
                const bool arow = a < nyg;
                const float2 q = arow ? qy[a] : make_float2(0.f, 0.f);
                const float on = arow ? 1.f : 0.f;
                float cs[4], sn[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    sincospif(2.0f * turns_reduced(q, cp[u].x, cp[u].y), &sn[u], &cs[u]);
                    cs[u] *= on;
                    sn[u] *= on;
                }
                const int m0 = 8 * g;
                const size_t blk = ((size_t)(m0 >> 7) * nkb + kb) * TC_BLOCK_BYTES;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    float wv[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) wv[u] = c == 0 ? w[u].x : c == 1 ? w[u].y : c == 2 ? w[u].z : w[u].w;
                    uint2 h, l;
                    const uint32_t oc = swz_offset((m0 & 127) + 2 * c, k0);
                    split4(wv[0] * cs[0], wv[1] * cs[1], wv[2] * cs[2], wv[3] * cs[3], h, l);
                    __stcs(reinterpret_cast<uint2*>(A_hi + blk + oc), h);
                    __stcs(reinterpret_cast<uint2*>(A_lo + blk + oc), l);
                    const uint32_t os = swz_offset((m0 & 127) + 2 * c + 1, k0);
                    split4(wv[0] * sn[0], wv[1] * sn[1], wv[2] * sn[2], wv[3] * sn[3], h, l);
                    __stcs(reinterpret_cast<uint2*>(A_hi + blk + os), h);
                    __stcs(reinterpret_cast<uint2*>(A_lo + blk + os), l);
                }
            }
        }
    }
}

// ------------------------------------------------------------------ PTX helpers
// Teardown wait for this CTA's own asynchronous operations (bulk copies in
// flight, issued MMAs): it does not give up when another role aborted, only
// after TC_DRAIN_LIMIT_NS, so an aborting CTA still lets what it started land
// before it frees TMEM and exits.
constexpr uint64_t TC_DRAIN_LIMIT_NS = 1000000000ull;

__device__ __forceinline__ bool mbar_wait_drain(uint64_t* bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (gtimer() - t0 > TC_DRAIN_LIMIT_NS) return false;
    }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// all threads of both CTAs of the cluster
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Tensor copy of one box (row y of a 2D map whose rows are 128-byte table
// rows; the box is 16 or 8 KB of one table block) into this CTA's shared
// memory, its bytes completing on an mbarrier of the CTA pair that may be
// the peer's (cta_group::2: the operands of a two-SM MMA signal the issuing
// CTA's barrier directly).  The x coordinate is always 0 (16-byte aligned).
__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* tm, int32_t y, uint32_t bar_cluster)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2 [%0], [%1, {%2, "
        "%3}], [%4];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(0), "r"(y), "r"(bar_cluster)
        : "memory");
}

// address of the mbarrier at this offset in CTA `cta` of the cluster
__device__ __forceinline__ uint32_t mbar_cluster_addr(uint64_t* bar, uint32_t cta)
{
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(bar)), "r"(cta));
    return remote;
}

// Packed FP32x2 arithmetic (sm_100+): two lanes of a 64-bit register, RN.
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint64_t f2_sub(uint64_t a, uint64_t b)
{
    uint64_t d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint64_t f2_pack(float lo_lane, float hi_lane)
{
    return ((uint64_t)__float_as_uint(hi_lane) << 32) | (uint64_t)__float_as_uint(lo_lane);
}

__device__ __forceinline__ float f2_lane0(uint64_t v) { return __uint_as_float((uint32_t)v); }

// Two-float sum (a_hi, a_lo) + (b_hi, b_lo) with TwoSum on both words and
// renormalisation, so neither low word has to be small (a GEMM partial's low
// word can hold whole chunk partials); relative error ~2^-44.
__device__ __forceinline__ float2 tf_add(float ah, float al, float bh, float bl)
{
    float s = ah + bh;
    float bb = s - ah;
    float e = (ah - (s - bb)) + (bh - bb);
    const float t = al + bl;
    bb = t - al;
    const float f = (al - (t - bb)) + (bl - bb);
    e += t;
    float h = s + e;                 // FastTwoSum(s, e)
    e = e - (h - s);
    e += f;
    s = h + e;                       // FastTwoSum(h, e)
    return make_float2(s, e - (s - h));
}

// two-float complex (re hi, re lo, im hi, im lo) sum
__device__ __forceinline__ float4 tf_add4(float4 a, float4 b)
{
    const float2 re = tf_add(a.x, a.y, b.x, b.y);
    const float2 im = tf_add(a.z, a.w, b.z, b.w);
    return make_float4(re.x, re.y, im.x, im.y);
}

__device__ __forceinline__ float f2_lane1(uint64_t v) { return __uint_as_float((uint32_t)(v >> 32)); }

// two-SM MMA: arrive (once this thread's MMAs complete) on the mbarrier at
// this offset in the CTAs of the pair named by mask (bit 0 even, bit 1 odd;
// a barrier signal into each CTA's own shared memory, no data moves)
__device__ __forceinline__ void tc_commit_pair(uint64_t* bar, uint16_t mask)
{
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(mask)
        : "memory");
}

// The three products of one 16-wide k step: D0 (+)= A_hi B_hi, D1 (+)= A_hi B_lo,
// D1 += A_lo B_hi, in one asm block (one predicate for the first two, a
// constant-true one for the third), so the issuing thread spends few
// instructions per MMA.
template <int CG>
__device__ __forceinline__ void tc_mma3_f16(uint32_t d0, uint32_t d1, uint64_t ah, uint64_t al, uint64_t bh,
                                            uint64_t bl, uint32_t idesc, uint32_t accumulate)
{
    if constexpr (CG == 2)
        asm volatile(
            "{\n\t.reg .pred p, t;\n\t"
            "setp.ne.b32 p, %7, 0;\n\t"
            "setp.eq.b32 t, %6, %6;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%0], %2, %4, %6, p;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%1], %2, %5, %6, p;\n\t"
            "tcgen05.mma.cta_group::2.kind::f16 [%1], %3, %4, %6, t;\n\t}\n" ::"r"(d0),
            "r"(d1), "l"(ah), "l"(al), "l"(bh), "l"(bl), "r"(idesc), "r"(accumulate)
            : "memory");
    else
        asm volatile(
            "{\n\t.reg .pred p, t;\n\t"
            "setp.ne.b32 p, %7, 0;\n\t"
            "setp.eq.b32 t, %6, %6;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %2, %4, %6, p;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%1], %2, %5, %6, p;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%1], %3, %4, %6, t;\n\t}\n" ::"r"(d0),
            "r"(d1), "l"(ah), "l"(al), "l"(bh), "l"(bl), "r"(idesc), "r"(accumulate)
            : "memory");
}

// arrive on the mbarrier at this offset in CTA `cta` of the cluster
__device__ __forceinline__ void mbar_arrive_cluster(uint64_t* bar, uint32_t cta)
{
    uint32_t remote;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(remote) : "r"(smem_u32(bar)), "r"(cta));
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(remote) : "memory");
}

// try_wait that also acquires what other CTAs of the cluster released
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(200000u)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_cluster(uint64_t* bar, uint32_t parity, uint64_t limit_ns,
                                                  volatile int* abort_flag)
{
    if (mbar_try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = gtimer();
    while (true) {
        if (mbar_try_wait_cluster(bar, parity)) return true;
        if (*abort_flag) return false;
        if (gtimer() - t0 > limit_ns) return false;
    }
}

// ------------------------------------------------------------------ GEMM
// Persistent: gridDim.x CTAs (one per SM) each walk their own run of the
// work list (unit u, a CTA or a CTA pair, takes the items
// [unit_item0[u], unit_item0[u + 1]); the host balances the runs); TMEM,
// barriers and the stage ring stay live across items.  An item is one
// 128 x 128 output tile per CTA over a k-block range of the chunk's tables.
// Its two-float result either goes, unscaled, to the partial tile P[slot]
// (128 x 128: column pairs outermost, rows innermost) for k_gemm_reduce, or
// -- when the item covers the whole k-range of its output (slot < 0) -- is
// combined into amplitudes, scaled and stored (first piece) or added into
// F[-1 - slot] (FbView layout; no partial tile, no reduction pass).
//
// MODE 0: one CTA per item, tcgen05.mma.cta_group::1 with M = N = 128.
//
// MODE 2: the two-SM MMA.  A pair item covers the A tiles 2*mt and 2*mt + 1
// and one B tile: tcgen05.mma.cta_group::2 with M = 256, N = 128, issued by
// the even CTA, reads the A tile of each CTA and the B tile split in two
// 64-row halves, one in each CTA's shared memory, and accumulates each CTA's
// 128 rows in its own TMEM.  A stage is 48 KB per SM instead of 64 KB and an
// MMA reads 6 KB of shared memory per 128 x 128 x 16 product instead of 8 KB;
// the 48 KB stages also make room for a fourth stage.  The even CTA's "stage
// full" barrier counts the bytes of both CTAs: the odd CTA loads its
// operands with tensor copies of the CTA pair (cta_group::2) that complete
// on the even CTA's barrier, so the MMA issuer waits on one barrier.  The odd
// CTA's epilogue warps release accumulators on the even CTA's barrier.
struct GemmItem {
    int32_t mt, nt;       // A / B tile rows (MODE 2: mt indexes A tile pairs)
    int32_t kb0, kb1;     // k-block range (within this chunk's tables)
    int32_t slot;         // output slot in P (pairs: of rank 0); < 0: direct to output -1 - slot
    int32_t slot1;        // pairs: output slot of rank 1 (direct: equal to slot)
    int32_t store;        // direct: 1 = first piece of its output (store), 0 = add
    int32_t two;          // direct: 1 = the output has several pieces (two-float, both planes)
};

struct GemmArgs {
    const uint8_t* A_hi;
    const uint8_t* A_lo;
    const uint8_t* B_hi;
    const uint8_t* B_lo;
    int64_t nkb;          // k-blocks in the tables of this launch (block stride)
    const GemmItem* items;
    const int32_t* unit_item0;   // [units + 1]: first item of each unit (CTA, or CTA pair in MODE 2)
    int kcb;              // k-blocks per TMEM chunk (drain interval)
    double* P;            // [slots][64 column pairs][128 rows] float4 (col 2j hi, lo, col 2j+1 hi, lo)
    double* F;            // direct outputs, high plane: [out][nz][nch * ny] float2 (FbView layout)
    int64_t lo_off;       // float2 from the high to the low plane
    AxisMap ax;
    int nch;              // channels per output (4 per weight set), a power of two
    float scale[4];       // direct outputs: per-channel scale of the unscaled sums (powers of two)
    int32_t* err;
    uint64_t limit_ns;
    int mtiles, ntiles;   // tile rows of A and B (table layout)
};

template <int MODE>
struct GemmCfg {
    static constexpr int STAGES = MODE == 2 ? 4 : TC_STAGES;
    static constexpr int STAGE_BYTES = MODE == 2 ? 3 * TC_BLOCK_BYTES : TC_STAGE_BYTES;
    static constexpr int B_BYTES = MODE == 2 ? TC_BLOCK_BYTES / 2 : TC_BLOCK_BYTES;   // B piece per CTA
    static constexpr int CG = MODE == 2 ? 2 : 1;
};

// Amplitudes at (s_y q_y, s_z q_z) from the four real sums cc, cs, sc, ss
// (each a two-float (hi, lo) pair): F = (cc - s_y s_z ss) - i (s_z cs + s_y sc),
// as a normalised two-float complex value (re hi, re lo, im hi, im lo).
__device__ __forceinline__ float4 combine_tf(float2 cc, float2 cs, float2 sc, float2 ss, float sy, float sz)
{
    const float k = -sy * sz;
    const float2 re = tf_add(cc.x, cc.y, k * ss.x, k * ss.y);
    const float2 im = tf_add(-sz * cs.x, -sz * cs.y, -sy * sc.x, -sy * sc.y);
    return make_float4(re.x, re.y, im.x, im.y);
}

// The end of an item: its two-float column sums (hi[i], lo[i]: columns
// colh + 2i and colh + 2i + 1 of TMEM lane 32 quad + lane, row of A tile
// mtile) go to the partial tile P[slot] or, for an item that covers its
// output's whole k-range (slot < 0), into the amplitudes.
__device__ __forceinline__ void store_item(const GemmArgs& g, const GemmItem& item, int slot, int mtile, int quad,
                                           int lane, int colh, const uint64_t* hi, const uint64_t* lo)
{
    // results leave as two-float pairs (no FP64 arithmetic here: GB300
    // issues few FP64 operations per clock)
    if (slot >= 0) {
        // this item's tile, unscaled: (hi, lo) per element, column
        // pairs j = n / 2 outermost, rows innermost (a warp's stores
        // are contiguous)
        float4* out = reinterpret_cast<float4*>(g.P) + (int64_t)slot * (TC_BM * TC_BN / 2) +
                      (int64_t)(colh >> 1) * TC_BM + quad * 32 + lane;
#pragma unroll
        for (int i = 0; i < 16; ++i)
            out[i * TC_BM] =
                make_float4(f2_lane0(hi[i]), f2_lane0(lo[i]), f2_lane1(hi[i]), f2_lane1(lo[i]));
    } else {
        // the whole k-range of this output.  Row mg = 2 (nch a + c) + p:
        // the lanes 2i, 2i + 1 of a warp hold the cos and sin rows of
        // one (a, c); columns 2b + r hold cos, sin of q_z,b.  Each lane
        // takes its partner's pair and writes one or two amplitudes:
        // on a symmetric q_y axis lane p = 0 writes +q_y and lane 1
        // the mirrored -q_y node (both q_z signs where q_z is
        // symmetric); otherwise lane 0 writes +q_z and lane 1 -q_z.
        const AxisMap& ax = g.ax;
        const int mg = mtile * TC_BM + quad * 32 + lane;
        const int p = mg & 1;
        const int qi = mg >> 1;
        const int ag = qi / g.nch, ch = qi & (g.nch - 1);
        const int b0 = (item.nt * TC_BN + colh) >> 1;       // GEMM q_z index of column pair 0
        const int64_t mrows = (int64_t)g.nch * ax.ny;
        float2* Fo = reinterpret_cast<float2*>(g.F) + (int64_t)(-1 - slot) * (ax.nz - ax.zs0) * mrows + ch;
        // this lane's q_y node and sign, and which q_z signs it writes
        // (-q_z only where the q_z < 0 rows are stored)
        float sy = 1.f;
        int a_out = ax.hy + ag;
        bool act = ag < ax.nyg;
        int zfirst = 0, zlast = (ax.mz && ax.zs0 == 0) ? 1 : 0;   // 0: +q_z, 1: -q_z
        if (ax.my) {
            if (p) {
                sy = -1.f;
                a_out = ax.ny - 1 - ax.hy - ag;
                act = act && a_out != ax.hy + ag;      // q_y = 0 is its own mirror
            }
        } else {
            zfirst = zlast = p;
            act = act && (p == 0 || ax.mz);
        }
        const float sc = g.scale[ch & 3];
        if (!item.two) {
            // the output's only piece, rounded to FP32: the two-float
            // sums are rounded first (one word per column to exchange),
            // then combined; error <= 2^-24 (|cc| + |ss| + |F|)
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const uint64_t x = f2_add(hi[i], lo[i]);
                const uint64_t y = __shfl_xor_sync(0xffffffffu, x, 1);
                const float xc = f2_lane0(x), xs = f2_lane1(x), yc = f2_lane0(y), ys = f2_lane1(y);
                const float cc = p ? yc : xc, cs = p ? ys : xs, scs = p ? xc : yc, ss = p ? xs : ys;
                const int bg = b0 + i;
                if (!act || bg >= ax.nzg) continue;
                for (int zs = zfirst; zs <= zlast; ++zs) {
                    const float sz = zs ? -1.f : 1.f;
                    const int b_out = zs ? ax.nz - 1 - ax.hz - bg : ax.hz + bg;
                    if (zs && b_out == ax.hz + bg) continue;     // q_z = 0 is its own mirror
                    const float re = fmaf(-sy * sz, ss, cc);
                    const float im = -fmaf(sz, cs, sy * scs);
                    Fo[(int64_t)(b_out - ax.zs0) * mrows + (int64_t)g.nch * a_out] = make_float2(sc * re, sc * im);
                }
            }
        } else
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            // partner pair: all lanes take part in the exchange
            const uint64_t ph = __shfl_xor_sync(0xffffffffu, hi[i], 1);
            const uint64_t pl = __shfl_xor_sync(0xffffffffu, lo[i], 1);
            const float2 xc = make_float2(f2_lane0(hi[i]), f2_lane0(lo[i]));   // own row x cos(q_z Z)
            const float2 xs = make_float2(f2_lane1(hi[i]), f2_lane1(lo[i]));   // own row x sin(q_z Z)
            const float2 yc = make_float2(f2_lane0(ph), f2_lane0(pl));
            const float2 ys = make_float2(f2_lane1(ph), f2_lane1(pl));
            const float2 cc = p ? yc : xc, cs = p ? ys : xs, scs = p ? xc : yc, ss = p ? xs : ys;
            const int bg = b0 + i;
            if (!act || bg >= ax.nzg) continue;
            for (int zs = zfirst; zs <= zlast; ++zs) {
                const float sz = zs ? -1.f : 1.f;
                const int b_out = zs ? ax.nz - 1 - ax.hz - bg : ax.hz + bg;
                if (zs && b_out == ax.hz + bg) continue;     // q_z = 0 is its own mirror
                // an output of several pieces: two-float, stored by its
                // first piece and added by the later ones
                float2* oh = Fo + (int64_t)(b_out - ax.zs0) * mrows + (int64_t)g.nch * a_out;
                float4 v = combine_tf(cc, cs, scs, ss, sy, sz);
                v = make_float4(sc * v.x, sc * v.y, sc * v.z, sc * v.w);
                float2* ol = oh + g.lo_off;
                if (!item.store) {
                    const float2 h = *oh, l = *ol;
                    v = tf_add4(v, make_float4(h.x, l.x, h.y, l.y));
                }
                *oh = make_float2(v.x, v.z);
                *ol = make_float2(v.y, v.w);
            }
        }
    }
}

// tmA / tmB (MODE 2): 2D maps over the chunk's tables as 128-byte rows,
// boxes of 128 rows (an A block) and 64 rows (half a B block)
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_gemm_f16x3(const GemmArgs g, const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB)
{
    using C = GemmCfg<MODE>;
    constexpr bool CLUSTER = MODE == 2;
    constexpr int STG = C::STAGES;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[STG];     // MODE 2, even CTA: both CTAs' stage bytes
    __shared__ __align__(8) uint64_t bar_empty[STG];
    __shared__ __align__(8) uint64_t bar_acc_full[2];
    __shared__ __align__(8) uint64_t bar_acc_empty[2];
    __shared__ __align__(8) uint64_t bar_final;
    __shared__ uint32_t s_taddr;
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const int rank = CLUSTER ? (int)cluster_rank() : 0;
    const int unit = CLUSTER ? (int)(blockIdx.x >> 1) : (int)blockIdx.x;   // this CTA's (pair's) run of items
    const int it_begin = g.unit_item0[unit], it_end = g.unit_item0[unit + 1];

    if (threadIdx.x == 0) {
        for (int s = 0; s < STG; ++s) {
            mbar_init(&bar_full[s], 1);
            mbar_init(&bar_empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&bar_acc_full[b], 1);
            mbar_init(&bar_acc_empty[b], MODE == 2 ? 2 * TC_EPI_WARPS : TC_EPI_WARPS);
        }
        mbar_init(&bar_final, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        tc_alloc<C::CG>(smem_u32(&s_taddr), 512);
        tc_relinquish<C::CG>();
    }
    tc_fence_before();
    __syncthreads();
    if (CLUSTER) cluster_sync();    // both CTAs' barriers initialised before any remote arrival
    tc_fence_after();
    const uint32_t taddr = s_taddr;

    if (warp == 0) {
        // ---------------- producer: bulk copies of the operand blocks
        if (lane == 0) {
            int64_t i = 0;              // stage sequence number across items
            int s = 0;                  // its stage
            uint32_t par = 1u;          // parity of the stage's previous "empty" phase
            bool ok = true;
            for (int it = it_begin; it < it_end && ok; ++it) {
                const GemmItem item = g.items[it];
                for (int kb = item.kb0; kb < item.kb1; ++kb) {
                    if (!mbar_wait(&bar_empty[s], par, g.limit_ns, &s_abort)) {
                        s_abort = 1;
                        atomicExch(g.err, 1);
                        ok = false;
                        break;
                    }
                    const uint32_t st = sbase + (uint32_t)s * C::STAGE_BYTES;
                    const int mt = MODE == 2 ? 2 * item.mt + rank : item.mt;
                    const int nt = item.nt;
                    if (MODE == 2 && rank == 1) {
                        // table rows (128 B each) of this CTA's A block and B half
                        const int32_t nk = (int32_t)g.nkb;
                        const int32_t ra = (mt * nk + kb) * 128;
                        const int32_t rb = ((2 * g.mtiles + nt) * nk + kb) * 128 + 64;
                        const uint32_t lead = mbar_cluster_addr(&bar_full[s], 0);
                        tma_load_2d_pair(st, &tmA, ra, lead);
                        tma_load_2d_pair(st + TC_BLOCK_BYTES, &tmA, ra + g.mtiles * nk * 128, lead);
                        tma_load_2d_pair(st + 2 * TC_BLOCK_BYTES, &tmB, rb, lead);
                        tma_load_2d_pair(st + 2 * TC_BLOCK_BYTES + C::B_BYTES, &tmB, rb + g.ntiles * nk * 128, lead);
                        ++i;
                        if (++s == STG) {
                            s = 0;
                            par ^= 1u;
                        }
                        continue;
                    }
                    mbar_arrive_expect_tx(&bar_full[s], MODE == 2 ? 2 * C::STAGE_BYTES : C::STAGE_BYTES);
                    const size_t ao = ((size_t)mt * g.nkb + kb) * TC_BLOCK_BYTES;
                    // MODE 2: this CTA's 64-row half of the B block
                    const size_t bo = ((size_t)nt * g.nkb + kb) * TC_BLOCK_BYTES + (MODE == 2 ? rank * C::B_BYTES : 0);
                    bulk_g2s(st, g.A_hi + ao, TC_BLOCK_BYTES, &bar_full[s]);
                    bulk_g2s(st + TC_BLOCK_BYTES, g.A_lo + ao, TC_BLOCK_BYTES, &bar_full[s]);
                    bulk_g2s(st + 2 * TC_BLOCK_BYTES, g.B_hi + bo, C::B_BYTES, &bar_full[s]);
                    bulk_g2s(st + 2 * TC_BLOCK_BYTES + C::B_BYTES, g.B_lo + bo, C::B_BYTES, &bar_full[s]);
                    ++i;
                    if (++s == STG) {
                        s = 0;
                        par ^= 1u;
                    }
                }
            }
            // copies in flight must land before the CTA exits (bounded): only
            // the last STG issued stages can still be pending.  MODE 2, odd
            // CTA: its copies complete on the even CTA's barriers; without an
            // abort the even CTA's MMAs consumed them all before the final
            // cluster barrier, after an abort it gives them 2 ms to land.
            if (MODE == 2 && rank == 1) {
                if (!ok) {
                    const uint64_t t0 = gtimer();
                    while (gtimer() - t0 < 2000000ull) __nanosleep(1000);
                }
            } else {
                for (int64_t k = (i > STG ? i - STG : 0); k < i; ++k) {
                    const int s = (int)(k % STG);
                    const uint32_t par = (uint32_t)((k / STG) & 1);
                    mbar_wait_drain(&bar_full[s], par);
                }
            }
        }
    } else if (warp == 1) {
        if (MODE == 2 && rank == 1) {
            // odd CTA: no MMA issuer (its operands and accumulators are
            // driven by the even CTA)
        } else if (lane == 0) {
            // ---------------- MMA issuer (one thread; MODE 2: of the even CTA)
            constexpr int MM = MODE == 2 ? 2 * TC_BM : TC_BM;
            const uint32_t idesc = idesc_f16_f32(MM, TC_BN);
            const uint32_t bofs = 2 * TC_BLOCK_BYTES;             // B_hi in the stage
            const uint32_t lofs = bofs + C::B_BYTES;              // B_lo in the stage
            int s = 0;                  // stage of the next k-block
            uint32_t sph = 0;           // its phase bit (flips each pass over the ring)
            uint32_t c = 0;             // TMEM chunk sequence number
            bool ok = true;
            for (int it = it_begin; it < it_end && ok; ++it) {
                const GemmItem item = g.items[it];
                for (int k0 = item.kb0; k0 < item.kb1 && ok; k0 += g.kcb, ++c) {
                    const int b = (int)(c & 1);
                    const uint32_t apar = (uint32_t)((c >> 1) & 1) ^ 1u;
                    const bool oka = MODE == 2 ? mbar_wait_cluster(&bar_acc_empty[b], apar, g.limit_ns, &s_abort)
                                               : mbar_wait(&bar_acc_empty[b], apar, g.limit_ns, &s_abort);
                    if (!oka) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t d0 = taddr + (uint32_t)b * 256u;
                    const uint32_t d1 = d0 + 128u;
                    const int k1 = min(item.kb1, k0 + g.kcb);
                    bool first = true;
                    for (int kb = k0; kb < k1; ++kb) {
                        const bool okf = mbar_wait(&bar_full[s], sph, g.limit_ns, &s_abort);
                        if (!okf) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t st = sbase + (uint32_t)s * C::STAGE_BYTES;
                        // descriptors of the stage's four blocks; each 16-wide k
                        // step moves the start address field by 32 bytes (2 units)
                        const uint64_t ah0 = sw128_desc(st), al0 = sw128_desc(st + TC_BLOCK_BYTES);
                        const uint64_t bh0 = sw128_desc(st + bofs), bl0 = sw128_desc(st + lofs);
#pragma unroll
                        for (int k16 = 0; k16 < 4; ++k16) {
                            tc_mma3_f16<C::CG>(d0, d1, ah0 + 2 * k16, al0 + 2 * k16, bh0 + 2 * k16, bl0 + 2 * k16, idesc,
                                               first ? 0u : 1u);
                            first = false;
                        }
                        if (MODE == 2) tc_commit_pair(&bar_empty[s], (uint16_t)3);
                        else tc_commit(&bar_empty[s]);
                        if (++s == STG) {
                            s = 0;
                            sph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    if (MODE == 2) tc_commit_pair(&bar_acc_full[b], (uint16_t)3);
                    else tc_commit(&bar_acc_full[b]);
                }
            }
            if (!ok) {
                s_abort = 1;
                atomicExch(g.err, 2);
            }
            // every MMA issued by this thread completes before TMEM is freed
            if (MODE == 2) tc_commit_pair(&bar_final, (uint16_t)1);
            else tc_commit(&bar_final);
            mbar_wait_drain(&bar_final, 0);
        }
    } else {
        // ---------------- epilogue: drain TMEM chunks into two-float sums
        const int e = warp - 2;
        const int quad = warp & 3;                 // TMEM lane quadrant of this warp
        const int colh = (e >> 2) * 32;            // column quarter
        int64_t c = 0;
        bool ok = true;
        for (int it = it_begin; it < it_end && ok; ++it) {
            const GemmItem item = g.items[it];
            // two-float running sums, two columns per 64-bit register
            uint64_t hi[16], lo[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) { hi[i] = 0ull; lo[i] = 0ull; }
            for (int k0 = item.kb0; k0 < item.kb1; k0 += g.kcb, ++c) {
                const int b = (int)(c & 1);
                const uint32_t par = (uint32_t)((c >> 1) & 1);
                int okw = 0;
                if (lane == 0) okw = mbar_wait(&bar_acc_full[b], par, g.limit_ns, &s_abort) ? 1 : 0;
                okw = __shfl_sync(0xffffffffu, okw, 0);
                if (!okw) {
                    if (lane == 0) {
                        s_abort = 1;
                        atomicExch(g.err, 3);
                    }
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t base = taddr + ((uint32_t)(quad * 32) << 16) + (uint32_t)b * 256u + (uint32_t)colh;
#pragma unroll
                for (int cb = 0; cb < 32 / TC_DRAIN_W; ++cb) {
                    float v0[TC_DRAIN_W], v1[TC_DRAIN_W];
                    tmem_ld<TC_DRAIN_W>(base + cb * TC_DRAIN_W, v0);
                    tmem_ld<TC_DRAIN_W>(base + 128 + cb * TC_DRAIN_W, v1);
                    tmem_wait_ld();
#pragma unroll
                    for (int u = 0; u < TC_DRAIN_W / 2; ++u) {
                        const int idx = cb * (TC_DRAIN_W / 2) + u;
                        const uint64_t x =
                            f2_add(f2_pack(v0[2 * u], v0[2 * u + 1]), f2_pack(v1[2 * u], v1[2 * u + 1]));
#if TC_RENORM == 0
                        // TwoSum(hi, x) -> (s, er); hi = s; lo += er
                        const uint64_t sm = f2_add(hi[idx], x);
                        const uint64_t bb = f2_sub(sm, hi[idx]);
                        const uint64_t er = f2_add(f2_sub(hi[idx], f2_sub(sm, bb)), f2_sub(x, bb));
                        hi[idx] = sm;
                        lo[idx] = f2_add(lo[idx], er);
#else
                        lo[idx] = f2_add(lo[idx], x);   // chunk partial into the low word
#endif
                    }
                    // pace the drain: four drain warps share each scheduler with
                    // the producer or MMA thread; a short yield per column
                    // group keeps the single MMA-issuing thread from waiting
                    // behind their bursts.  Not in the two-SM form, whose MMAs
                    // wait for both CTAs' drains.
                    if (MODE != 2) __nanosleep(8 * TC_DRAIN_W);
                }
#if TC_RENORM > 0
                // every TC_RENORM chunks: TwoSum(hi, lo) -> (hi, lo), so lo
                // never holds more than a few chunk partials
                if (((k0 - item.kb0) / g.kcb + 1) % TC_RENORM == 0) {
#pragma unroll
                    for (int idx = 0; idx < 16; ++idx) {
                        const uint64_t sm = f2_add(hi[idx], lo[idx]);
                        const uint64_t bb = f2_sub(sm, hi[idx]);
                        lo[idx] = f2_add(f2_sub(hi[idx], f2_sub(sm, bb)), f2_sub(lo[idx], bb));
                        hi[idx] = sm;
                    }
                }
#endif
                tc_fence_before();
                __syncwarp();
                if (lane == 0) {
                    if (MODE == 2) mbar_arrive_cluster(&bar_acc_empty[b], 0);   // the MMA issuer's barrier
                    else mbar_arrive(&bar_acc_empty[b]);
                }
            }
            if (!ok) break;
            store_item(g, item, (CLUSTER && rank) ? item.slot1 : item.slot, MODE == 2 ? 2 * item.mt + rank : item.mt,
                       quad, lane, colh, hi, lo);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (CLUSTER) cluster_sync();    // no MMA, commit or remote arrival can still target this CTA
    tc_fence_after();
    if (warp == 1) tc_dealloc<C::CG>(taddr, 512);
}

// ------------------------------------------------------------------ fused ray GEMM
// Polar grid (rays, reading of Eq. qdef on the paper's polar detector) with
// one weight set, one B tile and up to three A tiles (at most 48 x 64 |q|
// nodes): each slot is one to three 128 x 128 output tiles, so with tables
// every table block is written to HBM once and read back once by one to
// three tiles.  Each work item covers one A tile (item.mt: coarse nodes
// 16 mt ..) and generates that tile and the B tile; since B is generated
// again for every A tile, a fourth tile would make the tables the faster
// form.  This form builds
// each k-block's four operand blocks in shared memory instead, from the cells'
// ray projections u and weights, with the arithmetic of k_tables (two-float
// phase, exact reduction, scaled FP16 hi/lo split) except that the phase is
// taken in quarter turns and its sine and cosine come from sincos_node
// instead of sincospif: generation, not the MMAs, sets this form's pace.
//
// Roles (704 threads):
//   warp 0           copies each k-block's cell data (64 positions, then 64
//                    weights, float4) into a ring of RF_CELL_SLOTS slots
//                    and lays each slot out for the generating threads (u
//                    as two float arrays, projected on the slot's ray when
//                    given the cells rotated once per rotation; weights
//                    scaled, even and odd cells apart; cells past the
//                    k-block's end zero) before releasing it;
//   warp 1, lane 0   issues the MMAs (as in k_gemm_f16x3);
//   warps 2..17      generate the operand stages;
//   warps 18..21     drain the accumulator (one warp per TMEM lane quadrant,
//                    all 128 columns) and write each item's result.
// Shared memory written by threads and read by the tensor cores, or read by
// threads and then refilled by a bulk copy, is ordered across the two
// proxies by fence.proxy.async before the mbarrier arrival that hands it on.
// The drain's two-float running sums live in tensor memory (columns 256..383
// hi, 384..511 lo), since a drain thread covers 128 columns; the accumulator
// (D0 columns 0..127, D1 128..255) is single-buffered, so the MMAs of chunk c
// wait for the drain of chunk c - 1, which runs beside the generation of
// chunk c's operands (generation is the slower of the two).
constexpr int RF_CELL_SLOTS = 4;
constexpr int RF_CELL_BYTES = 64 * 32;   // per slot: 64 float4 positions, then 64 float4 weights
constexpr int RF_GEN_WARPS = 16;
constexpr int RF_WORKERS = RF_GEN_WARPS * 32;   // generating threads
constexpr int RF_DRAIN_WARPS = 4;               // one per TMEM lane quadrant
constexpr int RF_THREADS = (2 + RF_GEN_WARPS + RF_DRAIN_WARPS) * 32;
constexpr int RF_SMEM = TC_STAGES * TC_STAGE_BYTES + RF_CELL_SLOTS * RF_CELL_BYTES + 1024;

constexpr int RF_MAX_SLOTS = 64;     // slots per launch when the loader projects
constexpr int RF_MAX_COARSE = 48;    // coarse |q| nodes: up to 3 A tiles of 16
constexpr int RF_PROJ_LAG = 2;       // k-blocks between a slot's copy and its final layout

struct RayFusedArgs {
    // project = 0: cpos holds (u hi, u lo, u hi, u lo) and cw the weights per
    // cell of the stacked slot arrays, indexed by kb_cell0.  project = 1: cpos
    // holds the rotated two-float (Y hi, Y lo, Z hi, Z lo) and cw the rotated
    // weights once per rotation ([n_rot][n_cells]); a k-block's first cell
    // c0 = rl n_cells + c belongs to slot s = slot0 + rl, that is rotation
    // s / n_rays and ray s mod n_rays, and is read at (s / n_rays) n_cells + c;
    // the loader warp then projects it, u = Y sin theta + Z cos theta in
    // two-float (ray_sc: sin hi, lo, cos hi, lo per ray).
    const float4* cpos;
    const float4* cw;
    const int64_t* kb_cell0;      // first cell of each k-block of the launch
    const int32_t* kb_ncell;      // its cells (<= 64)
    const float4* ray_sc;         // project: [n_rays]
    int64_t n_cells;
    int project, slot0, n_rays, n_rl;
    float4 wscale;                // per-channel weight scale (as in k_tables)
    int nyg, nzg;                 // live nodes: coarse (A rows, <= 48: A tile mt holds 16 mt ..), fine (B rows, <= 64)
    float2 qy[RF_MAX_COARSE];     // coarse nodes lo + 64 i1 dq in turns (two-float)
    float2 qz[64];                // fine offsets i2 dq in turns (two-float)
};

// all lanes wait (bounded); the warp continues only if every lane saw the phase
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns, volatile int* abort_flag)
{
    const bool ok = mbar_wait(bar, parity, limit_ns, abort_flag);
    return __all_sync(0xffffffffu, ok) != 0;
}

// One k-block of operands into the stage at st (generic pointer): thread
// (r, q4) of the 512 workers (nodes qb0, qb1, qa times 4, as sincos_node
// takes them) writes B rows 2b, 2b + 1 (b = r, r + 32) for the
// cells 4 q4 .. + 3 (8-byte stores: a half-warp fills a 128-byte row) and the
// eight A rows of coarse node a = r / 2 (four channels x cos, sin) for the
// cells 4 q4 + 2h, + 1 (h = r mod 2; 4-byte stores: a warp fills a row).
// Unlike the tables, B is not masked: a cell past the k-block's end has zero
// weights in A, so its products vanish, and rows past the live nodes
// (b >= nzg, a >= nyg) only feed output rows and columns nothing reads.
__device__ __forceinline__ void ray_gen_block(uint8_t* st, const float* uh, const float* ul, float4 w0, float4 w1,
                                              int q4, int r, float2 qb0, float2 qb1, float2 qa)
{
#pragma unroll
    for (int jb = 0; jb < 2; ++jb) {
        const float2 q = jb ? qb1 : qb0;
        const int b = r + 32 * jb;
        float cs[4], sn[4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
            sincos_node<(int)TC_SCALE>(q, uh[u], ul[u], sn[u], cs[u]);
        uint2 ch, cl, sh, sl;
        split4(cs[0], cs[1], cs[2], cs[3], ch, cl);
        split4(sn[0], sn[1], sn[2], sn[3], sh, sl);
        const uint32_t oc = swz_offset(2 * b, 4 * q4), os = swz_offset(2 * b + 1, 4 * q4);
        *reinterpret_cast<uint2*>(st + 2 * TC_BLOCK_BYTES + oc) = ch;
        *reinterpret_cast<uint2*>(st + 3 * TC_BLOCK_BYTES + oc) = cl;
        *reinterpret_cast<uint2*>(st + 2 * TC_BLOCK_BYTES + os) = sh;
        *reinterpret_cast<uint2*>(st + 3 * TC_BLOCK_BYTES + os) = sl;
    }
    const int h = r & 1, a = r >> 1;
    const int k = 4 * q4 + 2 * h;
    const float u0h = h ? uh[2] : uh[0], u0l = h ? ul[2] : ul[0];
    const float u1h = h ? uh[3] : uh[1], u1l = h ? ul[3] : ul[1];
    float s0, c0, s1, c1;
    sincos_node(qa, u0h, u0l, s0, c0);
    sincos_node(qa, u1h, u1l, s1, c1);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float x0 = c == 0 ? w0.x : c == 1 ? w0.y : c == 2 ? w0.z : w0.w;
        const float x1 = c == 0 ? w1.x : c == 1 ? w1.y : c == 2 ? w1.z : w1.w;
        const int row = 2 * (4 * a + c);
        uint32_t hh, ll;
        split_h2(x0 * c0, x1 * c1, hh, ll);
        const uint32_t oc = swz_offset(row, k), os = swz_offset(row + 1, k);
        *reinterpret_cast<uint32_t*>(st + oc) = hh;
        *reinterpret_cast<uint32_t*>(st + TC_BLOCK_BYTES + oc) = ll;
        split_h2(x0 * s0, x1 * s1, hh, ll);
        *reinterpret_cast<uint32_t*>(st + os) = hh;
        *reinterpret_cast<uint32_t*>(st + TC_BLOCK_BYTES + os) = ll;
    }
}

// Drain one chunk into the tensor-memory running sums of this warp's lane
// quadrant, all 128 columns (tb: column 0 of D0; D1 +128, hi +256, lo +384):
// lo += D0 + D1 (first chunk of an item: hi = 0, lo = D0 + D1), then, when
// renorm, a second pass TwoSum(hi, lo) -> (hi, lo).  The MMAs of the next
// chunk wait for this drain, so each TMEM load round trip covers two
// 8-column groups.
__device__ __forceinline__ void ray_drain_pair(uint32_t tb, int cb, bool first)
{
    float d0[16], d1[16], sl[16];
    tmem_ld8(tb + 8 * cb, d0);
    tmem_ld8(tb + 8 * cb + 8, d0 + 8);
    tmem_ld8(tb + 128 + 8 * cb, d1);
    tmem_ld8(tb + 128 + 8 * cb + 8, d1 + 8);
    if (!first) {
        tmem_ld8(tb + 384 + 8 * cb, sl);
        tmem_ld8(tb + 384 + 8 * cb + 8, sl + 8);
    }
    tmem_wait_ld();
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const uint64_t x = f2_add(f2_pack(d0[2 * u], d0[2 * u + 1]), f2_pack(d1[2 * u], d1[2 * u + 1]));
        const uint64_t lo = first ? x : f2_add(f2_pack(sl[2 * u], sl[2 * u + 1]), x);
        sl[2 * u] = f2_lane0(lo);
        sl[2 * u + 1] = f2_lane1(lo);
    }
#pragma unroll
    for (int z = 0; z < 16; z += 4) tmem_st4(tb + 384 + 8 * cb + z, sl + z);
    if (first) {
#pragma unroll
        for (int z = 0; z < 16; ++z) d0[z] = 0.f;
#pragma unroll
        for (int z = 0; z < 16; z += 4) tmem_st4(tb + 256 + 8 * cb + z, d0 + z);
    }
}

__device__ __forceinline__ void ray_drain_chunk(uint32_t tb, bool first, bool renorm)
{
    for (int cb = 0; cb < 16; cb += 2) ray_drain_pair(tb, cb, first);
    if (renorm) {
        tmem_wait_st();
        for (int cb = 0; cb < 16; cb += 2) {
            float sh[16], sl[16];
            tmem_ld8(tb + 256 + 8 * cb, sh);
            tmem_ld8(tb + 256 + 8 * cb + 8, sh + 8);
            tmem_ld8(tb + 384 + 8 * cb, sl);
            tmem_ld8(tb + 384 + 8 * cb + 8, sl + 8);
            tmem_wait_ld();
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint64_t hi = f2_pack(sh[2 * u], sh[2 * u + 1]);
                const uint64_t lo = f2_pack(sl[2 * u], sl[2 * u + 1]);
                const uint64_t sm = f2_add(hi, lo);
                const uint64_t bb = f2_sub(sm, hi);
                const uint64_t er = f2_add(f2_sub(hi, f2_sub(sm, bb)), f2_sub(lo, bb));
                sh[2 * u] = f2_lane0(sm);
                sh[2 * u + 1] = f2_lane1(sm);
                sl[2 * u] = f2_lane0(er);
                sl[2 * u + 1] = f2_lane1(er);
            }
#pragma unroll
            for (int z = 0; z < 16; z += 4) {
                tmem_st4(tb + 256 + 8 * cb + z, sh + z);
                tmem_st4(tb + 384 + 8 * cb + z, sl + z);
            }
        }
    }
    tmem_wait_st();
}

__global__ void __launch_bounds__(RF_THREADS, 1)
    k_gemm_ray_fused(const GemmArgs g, const __grid_constant__ RayFusedArgs ra)
{
    constexpr int STG = TC_STAGES;
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t bar_full[STG];       // RF_WORKERS arrivals: a stage is generated
    __shared__ __align__(8) uint64_t bar_empty[STG];      // MMA commit: a stage is consumed
    __shared__ __align__(8) uint64_t bar_cell_full[RF_CELL_SLOTS];
    __shared__ __align__(8) uint64_t bar_cell_empty[RF_CELL_SLOTS];
    __shared__ __align__(8) uint64_t bar_acc_full;
    __shared__ __align__(8) uint64_t bar_acc_empty;
    __shared__ __align__(8) uint64_t bar_final;
    __shared__ __align__(8) uint64_t bar_raw_full[RF_CELL_SLOTS];   // project: a slot's copy landed
    __shared__ int s_nc[RF_CELL_SLOTS];
    __shared__ int s_rl[RF_CELL_SLOTS];
    __shared__ float4 s_sc[RF_MAX_SLOTS];
    __shared__ uint32_t s_taddr;
    __shared__ volatile int s_abort;

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    uint8_t* const sgen = smem_raw + (sbase - smem_u32(smem_raw));      // the same address, generic
    uint8_t* const cells = sgen + STG * TC_STAGE_BYTES;
    const int it_begin = g.unit_item0[blockIdx.x], it_end = g.unit_item0[blockIdx.x + 1];

    if (threadIdx.x == 0) {
        for (int s = 0; s < STG; ++s) {
            mbar_init(&bar_full[s], RF_WORKERS);
            mbar_init(&bar_empty[s], 1);
        }
        for (int s = 0; s < RF_CELL_SLOTS; ++s) {
            mbar_init(&bar_cell_full[s], 1);
            mbar_init(&bar_cell_empty[s], RF_WORKERS);
            mbar_init(&bar_raw_full[s], 1);
        }
        mbar_init(&bar_acc_full, 1);
        mbar_init(&bar_acc_empty, RF_DRAIN_WARPS);
        mbar_init(&bar_final, 1);
        s_abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (ra.project && threadIdx.x < ra.n_rl) s_sc[threadIdx.x] = ra.ray_sc[(ra.slot0 + threadIdx.x) % ra.n_rays];
    if (warp == 1) {
        tc_alloc<1>(smem_u32(&s_taddr), 512);
        tc_relinquish<1>();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t taddr = s_taddr;

    if (warp == 0) {
        // ---------------- cell loader: bulk copies of each k-block's cells.
        // The warp reads the k-block descriptors 32 at a time (lane l holds
        // block kb0 + 32 i + l), so the copies never wait on those loads;
        // every lane follows the ring, lane 0 issues.  RF_PROJ_LAG k-blocks
        // after a slot's copy the warp rewrites it in the generating threads'
        // layout (with project = 1 projecting (Y, Z) on the slot's ray), then
        // releases it to them.
        int64_t i = 0;                      // k-block sequence number (copies issued)
        int cs = 0;                         // its cell slot
        uint32_t par = 1u;                  // parity of the slot's previous "empty" phase
        int64_t jp = 0;                     // project: k-blocks projected
        int csp = 0;
        uint32_t ppar = 0u;
        bool ok = true;
        // a slot's copy has landed: turn it into the layout the generating
        // threads read (u hi at 0, u lo at 256 bytes, 64 floats each; the
        // weights times the channel scale, cells 0, 2, .. at 1024 and 1, 3, ..
        // at 1536 bytes), every one of the 64 cells written, past nc zero
        auto finalize_next = [&]() -> bool {
            if (!warp_wait(&bar_raw_full[csp], ppar, g.limit_ns, &s_abort)) return false;
            const int nc = s_nc[csp];
            uint8_t* cl = cells + csp * RF_CELL_BYTES;
            const float4 W = ra.wscale;
            float uh[2], ul[2];
            float4 w[2];
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int k = lane + 32 * q;
                uh[q] = ul[q] = 0.f;
                w[q] = make_float4(0.f, 0.f, 0.f, 0.f);
                if (k < nc) {
                    const float4 x = *reinterpret_cast<const float4*>(cl + 16 * k);
                    if (ra.project) {
                        // u = Y sin theta + Z cos theta: two two-float products and a TwoSum
                        const float4 sc = s_sc[s_rl[csp]];
                        const float p1 = sc.x * x.x, p2 = sc.z * x.z;
                        const float e1 = fmaf(sc.x, x.x, -p1) + fmaf(sc.x, x.y, sc.y * x.x);
                        const float e2 = fmaf(sc.z, x.z, -p2) + fmaf(sc.z, x.w, sc.w * x.z);
                        const float sm = p1 + p2;
                        const float bb = sm - p1;
                        const float e = ((p1 - (sm - bb)) + (p2 - bb)) + (e1 + e2);
                        uh[q] = sm + e;
                        ul[q] = e - (uh[q] - sm);
                    } else {
                        uh[q] = x.x;
                        ul[q] = x.y;
                    }
                    const float4 v = *reinterpret_cast<const float4*>(cl + RF_CELL_BYTES / 2 + 16 * k);
                    w[q] = make_float4(v.x * W.x, v.y * W.y, v.z * W.z, v.w * W.w);
                }
            }
            __syncwarp();   // every lane has read its cells before any is overwritten
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int k = lane + 32 * q;
                reinterpret_cast<float*>(cl)[k] = uh[q];
                reinterpret_cast<float*>(cl + 256)[k] = ul[q];
                *reinterpret_cast<float4*>(cl + RF_CELL_BYTES / 2 + 512 * (k & 1) + 16 * (k >> 1)) = w[q];
            }
            fence_proxy_async_smem();       // these writes precede the slot's next bulk copy
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar_cell_full[csp]);
            ++jp;
            if (++csp == RF_CELL_SLOTS) {
                csp = 0;
                ppar ^= 1u;
            }
            return true;
        };
        for (int it = it_begin; it < it_end && ok; ++it) {
            const GemmItem item = g.items[it];
            for (int base = item.kb0; base < item.kb1 && ok; base += 32) {
                const int my = base + lane;
                const int64_t my_c0 = my < item.kb1 ? ra.kb_cell0[my] : 0;
                const int my_nc = my < item.kb1 ? ra.kb_ncell[my] : 0;
                const int cnt = min(32, item.kb1 - base);
                for (int j = 0; j < cnt; ++j) {
                    const int64_t c0 = __shfl_sync(0xffffffffu, my_c0, j);
                    const int nc = __shfl_sync(0xffffffffu, my_nc, j);
                    if (!warp_wait(&bar_cell_empty[cs], par, g.limit_ns, &s_abort)) {
                        ok = false;
                        break;
                    }
                    if (lane == 0) {
                        s_nc[cs] = nc;
                        int64_t src = c0;
                        uint64_t* landed = &bar_raw_full[cs];
                        if (ra.project) {
                            const int64_t rl = c0 / ra.n_cells;
                            const int slot = ra.slot0 + (int)rl;
                            src = (int64_t)(slot / ra.n_rays) * ra.n_cells + (c0 - rl * ra.n_cells);
                            s_rl[cs] = (int)rl;
                        }
                        uint8_t* dst = cells + cs * RF_CELL_BYTES;
                        if (nc > 0) {
                            mbar_arrive_expect_tx(landed, (uint32_t)nc * 32u);
                            bulk_g2s(smem_u32(dst), ra.cpos + src, (uint32_t)nc * 16u, landed);
                            bulk_g2s(smem_u32(dst + RF_CELL_BYTES / 2), ra.cw + src, (uint32_t)nc * 16u, landed);
                        } else {
                            mbar_arrive(landed);
                        }
                    }
                    __syncwarp();
                    ++i;
                    if (++cs == RF_CELL_SLOTS) {
                        cs = 0;
                        par ^= 1u;
                    }
                    if (i - jp > RF_PROJ_LAG && !finalize_next()) {
                        ok = false;
                        break;
                    }
                }
            }
        }
        while (ok && jp < i)
            if (!finalize_next()) ok = false;
        if (!ok && lane == 0) {
            s_abort = 1;
            atomicExch(g.err, 1);
        }
        // copies in flight land before the CTA exits (bounded): those issued
        // and not yet finalised (none, unless the block aborted)
        if (lane == 0)
            for (int64_t k = (jp > i - RF_CELL_SLOTS ? jp : i - RF_CELL_SLOTS); k < i; ++k)
                mbar_wait_drain(&bar_raw_full[(int)(k % RF_CELL_SLOTS)], (uint32_t)((k / RF_CELL_SLOTS) & 1));
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer: one accumulator pair (D0, D1)
            const uint32_t idesc = idesc_f16_f32(TC_BM, TC_BN);
            int s = 0;
            uint32_t sph = 0;
            uint32_t c = 0;                 // chunk sequence number
            bool ok = true;
            for (int it = it_begin; it < it_end && ok; ++it) {
                const GemmItem item = g.items[it];
                for (int k0 = item.kb0; k0 < item.kb1 && ok; k0 += g.kcb, ++c) {
                    // the drain of chunk c - 1 has read the accumulator
                    if (!mbar_wait(&bar_acc_empty, (c & 1u) ^ 1u, g.limit_ns, &s_abort)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const int k1 = min(item.kb1, k0 + g.kcb);
                    bool first = true;
                    for (int kb = k0; kb < k1; ++kb) {
                        if (!mbar_wait(&bar_full[s], sph, g.limit_ns, &s_abort)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const uint32_t st = sbase + (uint32_t)s * TC_STAGE_BYTES;
                        const uint64_t ah0 = sw128_desc(st), al0 = sw128_desc(st + TC_BLOCK_BYTES);
                        const uint64_t bh0 = sw128_desc(st + 2 * TC_BLOCK_BYTES);
                        const uint64_t bl0 = sw128_desc(st + 3 * TC_BLOCK_BYTES);
#pragma unroll
                        for (int k16 = 0; k16 < 4; ++k16) {
                            tc_mma3_f16<1>(taddr, taddr + 128u, ah0 + 2 * k16, al0 + 2 * k16, bh0 + 2 * k16,
                                           bl0 + 2 * k16, idesc, first ? 0u : 1u);
                            first = false;
                        }
                        tc_commit(&bar_empty[s]);
                        if (++s == STG) {
                            s = 0;
                            sph ^= 1u;
                        }
                    }
                    if (!ok) break;
                    tc_commit(&bar_acc_full);
                }
            }
            if (!ok) {
                s_abort = 1;
                atomicExch(g.err, 2);
            }
            tc_commit(&bar_final);
            mbar_wait_drain(&bar_final, 0);
        }
    } else if (warp < 2 + RF_GEN_WARPS) {
        // ---------------- generating warps: the operand stages
        const int t = threadIdx.x - 64;
        const int q4 = t & 15;                      // cells 4 q4 .. + 3 of each k-block
        const int r = t >> 4;                       // B nodes r, r + 32; A node r / 2
        const int h = r & 1;                        // A cells 4 q4 + 2h, + 1
        const float2 zero2 = make_float2(0.f, 0.f);
        // this thread's nodes times 4 (phases in quarter turns; exact)
        auto x4 = [](float2 v) { return make_float2(4.0f * v.x, 4.0f * v.y); };
        const float2 qb0 = r < ra.nzg ? x4(ra.qz[r]) : zero2;
        const float2 qb1 = r + 32 < ra.nzg ? x4(ra.qz[r + 32]) : zero2;
        int s = 0;
        uint32_t epar = 1u;                         // parity of the stage's previous "empty" phase
        int cs = 0;
        uint32_t cpar = 0u;                         // parity of the cell slot's next "full" phase
        bool ok = true;
        for (int it = it_begin; it < it_end && ok; ++it) {
            const GemmItem item = g.items[it];
            // the coarse node of this thread's A rows in the item's A tile
            const int a_node = 16 * item.mt + (r >> 1);
            const float2 qa = a_node < ra.nyg ? x4(ra.qy[a_node]) : zero2;
            for (int kb = item.kb0; kb < item.kb1; ++kb) {
                // this k-block's cells
                if (!warp_wait(&bar_cell_full[cs], cpar, g.limit_ns, &s_abort)) {
                    ok = false;
                    break;
                }
                // the slot as the loader warp laid it out: u of cells 4 q4 .. + 3,
                // scaled weights of cells 4 q4 + 2h (even) and + 1 (odd)
                const uint8_t* cl = cells + cs * RF_CELL_BYTES;
                const float4 uh4 = *reinterpret_cast<const float4*>(cl + 16 * q4);
                const float4 ul4 = *reinterpret_cast<const float4*>(cl + 256 + 16 * q4);
                const float4 w0 = *reinterpret_cast<const float4*>(cl + RF_CELL_BYTES / 2 + 16 * (2 * q4 + h));
                const float4 w1 = *reinterpret_cast<const float4*>(cl + RF_CELL_BYTES / 2 + 512 + 16 * (2 * q4 + h));
                // the slot's next contents arrive by bulk copy (async proxy):
                // order these generic reads before it, then release the slot
                fence_proxy_async_smem();
                mbar_arrive(&bar_cell_empty[cs]);
                if (++cs == RF_CELL_SLOTS) {
                    cs = 0;
                    cpar ^= 1u;
                }
                const float uh[4] = {uh4.x, uh4.y, uh4.z, uh4.w};
                const float ul[4] = {ul4.x, ul4.y, ul4.z, ul4.w};
                // the stage, once the MMAs have read its previous contents
                if (!warp_wait(&bar_empty[s], epar, g.limit_ns, &s_abort)) {
                    ok = false;
                    break;
                }
                ray_gen_block(sgen + s * TC_STAGE_BYTES, uh, ul, w0, w1, q4, r, qb0, qb1, qa);
                fence_proxy_async_smem();
                mbar_arrive(&bar_full[s]);
                if (++s == STG) {
                    s = 0;
                    epar ^= 1u;
                }
            }
        }
        if (!ok && lane == 0) {
            s_abort = 1;
            atomicExch(g.err, 3);
        }
    } else {
        // ---------------- drain warps: one per TMEM lane quadrant, all 128
        // columns: each chunk into the running sums, each item's sums out
        const int quad = warp & 3;
        const uint32_t tb = taddr + ((uint32_t)(quad * 32) << 16);
        uint32_t c = 0;                             // chunk sequence number
        bool ok = true;
        for (int it = it_begin; it < it_end && ok; ++it) {
            const GemmItem item = g.items[it];
            bool any = false;
            for (int k0 = item.kb0, ci = 0; k0 < item.kb1; k0 += g.kcb, ++ci, ++c) {
                int okw = 0;
                if (lane == 0) okw = mbar_wait(&bar_acc_full, c & 1u, g.limit_ns, &s_abort) ? 1 : 0;
                okw = __shfl_sync(0xffffffffu, okw, 0);
                if (!okw) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                ray_drain_chunk(tb, ci == 0, TC_RENORM <= 1 || (ci + 1) % TC_RENORM == 0);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&bar_acc_empty);
                any = true;
            }
            if (!ok) {
                if (lane == 0) {
                    s_abort = 1;
                    atomicExch(g.err, 3);
                }
                break;
            }
            const int row = quad * 32 + lane;       // this lane's accumulator row (of A tile item.mt)
            if (item.slot < 0) {
                // an output of one piece: its amplitudes, rounded to FP32, go
                // straight into F (FbView layout).  Rays mirror no axis, so
                // lane p = 0 of each (cos, sin) row pair writes
                // F = (cc - ss) - i (cs + sc), its partner lane holding sc, ss.
                // This form's schedule sends outputs of several pieces through
                // partial slots.
                if (item.two) {
                    if (lane == 0) atomicExch(g.err, 4);
                    continue;
                }
                const AxisMap& ax = g.ax;
                const int mg = item.mt * TC_BM + row;
                const int p = mg & 1, qi = mg >> 1;
                const int ag = qi / g.nch, ch = qi & (g.nch - 1);
                const int64_t mrows = (int64_t)g.nch * ax.ny;
                float2* Fo = reinterpret_cast<float2*>(g.F) + (int64_t)(-1 - item.slot) * (ax.nz - ax.zs0) * mrows +
                             ch + (int64_t)g.nch * (ax.hy + ag);
                const bool act = p == 0 && ag < ax.nyg;
                const float sc = g.scale[ch & 3];
                for (int cb = 0; cb < 16; ++cb) {
                    float xh[8], xl[8];
                    if (any) {
                        tmem_ld8(tb + 256 + 8 * cb, xh);
                        tmem_ld8(tb + 384 + 8 * cb, xl);
                        tmem_wait_ld();
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; ++i) xh[i] = xl[i] = 0.f;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const uint64_t x = f2_add(f2_pack(xh[2 * u], xh[2 * u + 1]), f2_pack(xl[2 * u], xl[2 * u + 1]));
                        const uint64_t y = __shfl_xor_sync(0xffffffffu, x, 1);
                        const int bg = 4 * cb + u;
                        if (act && bg < ax.nzg) {
                            const float cc = f2_lane0(x), cs = f2_lane1(x), scs = f2_lane0(y), ss = f2_lane1(y);
                            Fo[(int64_t)(ax.hz + bg - ax.zs0) * mrows] = make_float2(sc * (cc - ss), -sc * (cs + scs));
                        }
                    }
                }
                continue;
            }
            // the item's tile, unscaled, to its partial slot P[slot]
            // (k_gemm_reduce combines them), 8 columns at a time from TMEM
            float4* out = reinterpret_cast<float4*>(g.P) + (int64_t)item.slot * (TC_BM * TC_BN / 2) + row;
            for (int cb = 0; cb < 16; ++cb) {
                float xh[8], xl[8];
                if (any) {
                    tmem_ld8(tb + 256 + 8 * cb, xh);
                    tmem_ld8(tb + 384 + 8 * cb, xl);
                    tmem_wait_ld();
                } else {
#pragma unroll
                    for (int i = 0; i < 8; ++i) xh[i] = xl[i] = 0.f;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    out[(4 * cb + u) * TC_BM] = make_float4(xh[2 * u], xl[2 * u], xh[2 * u + 1], xl[2 * u + 1]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) tc_dealloc<1>(taddr, 512);
}

// Reduction of item tiles (two-float elements) into per-output amplitudes
// (two-float complex; stored by an output's first piece, added by later ones).
// Thread (output r, GEMM q_z index b, pair qi = nch a + c) sums the splits of
// the tile rows 2 qi (cos q_y Y: cc, cs) and 2 qi + 1 (sin q_y Y: sc, ss) at
// column pair j = b mod 64 of B tile b / 64, then writes the amplitudes of
// every sign combination of the symmetric axes whose q_z row is stored
// (s_z = +1 only when both axes are symmetric, FbView):
//   F[out][b_out - zs0][nch a_out + c] (+)= scale_{c mod 4} ((cc - s_y s_z ss) - i (s_z cs + s_y sc)).
// Threads run over qi fastest, so the tile reads and the F writes are
// contiguous.
struct RedDesc {
    int32_t slot_base;
    int32_t splits;
    int32_t out;
    int32_t store;        // bit 0: first piece of its output (store, else add); bit 1: several pieces (two-float)
};

struct Scale4 {
    float v[4];
};

__global__ void k_gemm_reduce(const double* __restrict__ P, const RedDesc* __restrict__ reds, int n_red, AxisMap ax,
                              int ntiles, int nch, Scale4 scale, double* __restrict__ F, int64_t lo_off)
{
    const int64_t qrows = (int64_t)nch * ax.nyg;
    const int64_t per_red = qrows * ax.nzg;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_red * per_red) return;
    const int r = (int)(idx / per_red);
    const int64_t rem = idx % per_red;
    const int bg = (int)(rem / qrows);
    const int qi = (int)(rem % qrows);
    const int ag = qi / nch, c = qi & (nch - 1);
    const int mg = 2 * qi;
    const int mt = mg >> 7, row = mg & 127, nt = bg >> 6, j = bg & 63;
    const RedDesc d = reds[r];
    const int64_t base = (int64_t)d.slot_base + (int64_t)(mt * ntiles + nt) * d.splits;
    const float4* P4 = reinterpret_cast<const float4*>(P);
    // two-float sums in FP32 (FP64 is slow on GB300); the scale is a power
    // of two, exact in FP32
    float4 a0 = make_float4(0.f, 0.f, 0.f, 0.f), a1 = a0;
    for (int s = 0; s < d.splits; ++s) {
        const float4* t = P4 + (base + s) * (TC_BM * TC_BN / 2) + (int64_t)j * TC_BM + row;
        a0 = tf_add4(a0, t[0]);
        a1 = tf_add4(a1, t[1]);
    }
    const float2 cc = make_float2(a0.x, a0.y), cs = make_float2(a0.z, a0.w);
    const float2 sc = make_float2(a1.x, a1.y), ss = make_float2(a1.z, a1.w);
    const float f = scale.v[c & 3];
    const int64_t mrows = (int64_t)nch * ax.ny;
    float2* Fo = reinterpret_cast<float2*>(F) + (int64_t)d.out * (ax.nz - ax.zs0) * mrows + c;
    const int zlast = (ax.mz && ax.zs0 == 0) ? 1 : 0;   // -q_z only where those rows are stored
    for (int ys = 0; ys <= ax.my; ++ys) {
        const int a_out = ys ? ax.ny - 1 - ax.hy - ag : ax.hy + ag;
        if (ys && a_out == ax.hy + ag) continue;        // q_y = 0 is its own mirror
        for (int zs = 0; zs <= zlast; ++zs) {
            const int b_out = zs ? ax.nz - 1 - ax.hz - bg : ax.hz + bg;
            if (zs && b_out == ax.hz + bg) continue;
            float4 v = combine_tf(cc, cs, sc, ss, ys ? -1.f : 1.f, zs ? -1.f : 1.f);
            v = make_float4(f * v.x, f * v.y, f * v.z, f * v.w);
            float2* oh = Fo + (int64_t)(b_out - ax.zs0) * mrows + (int64_t)nch * a_out;
            if (d.store & 2) {
                float2* ol = oh + lo_off;
                if (!(d.store & 1)) {
                    const float2 h = *oh, l = *ol;
                    v = tf_add4(v, make_float4(h.x, l.x, h.y, l.y));
                }
                *oh = make_float2(v.x, v.z);
                *ol = make_float2(v.y, v.w);
            } else {
                *oh = make_float2(v.x + v.y, v.z + v.w);   // the output's only piece, rounded to FP32
            }
        }
    }
}

// ------------------------------------------------------------------ self-test
// A bounded wait that runs out: one thread waits on an mbarrier nothing
// arrives on, with the same wait the GEMM uses; after limit_ns it records
// code 7 in err and returns.  Nothing is in flight, so the context stays
// usable.
__global__ void k_selftest_wait(uint64_t limit_ns, int32_t* err)
{
    __shared__ __align__(8) uint64_t bar;
    __shared__ volatile int abort_flag;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait(&bar, 0, limit_ns, &abort_flag)) atomicExch(err, 7);
}

cudaError_t launch_selftest_wait(uint64_t limit_ns, int32_t* err, cudaStream_t s)
{
    k_selftest_wait<<<1, 32, 0, s>>>(limit_ns, err);
    return cudaGetLastError();
}

// Self-test of sincos_node: for each t, sin and cos of 2 pi t by
// sincos_node (node 1, coordinate t: out[4i], out[4i + 1]) and by sincospif
// (out[4i + 2], + 3).
__global__ void k_selftest_sincos(const float* __restrict__ t, int64_t n, float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s, c, s2, c2;
    sincos_node(make_float2(4.0f, 0.0f), t[i], 0.0f, s, c);
    sincospif(2.0f * t[i], &s2, &c2);
    out[4 * i] = s;
    out[4 * i + 1] = c;
    out[4 * i + 2] = s2;
    out[4 * i + 3] = c2;
}

cudaError_t launch_selftest_sincos(const float* t, int64_t n, float* out, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_selftest_sincos<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(t, n, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ launchers
cudaError_t tc_launch_tables(const float4* cpos, const float4* cw, int64_t wstride, int nch, const int64_t* kb_cell0,
                             const int32_t* kb_ncell, int64_t nkb, const float2* qy, int nyg, const float2* qz, int nzg,
                             int mtiles, int ntiles, const float wscale[4], void* tab, cudaStream_t s)
{
    uint8_t* A_hi = (uint8_t*)tab;
    uint8_t* A_lo = A_hi + (size_t)mtiles * nkb * TC_BLOCK_BYTES;
    uint8_t* B_hi = A_lo + (size_t)mtiles * nkb * TC_BLOCK_BYTES;
    uint8_t* B_lo = B_hi + (size_t)ntiles * nkb * TC_BLOCK_BYTES;
    if (nkb <= 0) return cudaSuccess;
    k_tables<<<(unsigned)std::min<int64_t>(nkb, 0x7fffffff), TAB_THREADS, 0, s>>>(
        cpos, cw, wstride, nch, kb_cell0, kb_ncell, qy, nyg, qz, nzg,
        make_float4(wscale[0], wscale[1], wscale[2], wscale[3]), nkb, mtiles, ntiles, A_hi, A_lo, B_hi, B_lo);
    return cudaGetLastError();
}

// Two 2D maps over `rows` table rows of 128 bytes (64 x 16-bit) at tab:
// boxes of 128 rows (an A block) and of 64 rows (half a B block).  The data
// is already in the MMA's swizzled layout, so the copies do not swizzle.
static cudaError_t encode_row_maps(const void* tab, int64_t rows, CUtensorMap* tm)
{
    typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                    const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                    CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
    static EncodeTiled encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return e != cudaSuccess ? e : cudaErrorNotSupported;
        encode = (EncodeTiled)fn;
    }
    const cuuint64_t dim[2] = {64, (cuuint64_t)rows};
    const cuuint64_t stride[1] = {128};
    const cuuint32_t estr[2] = {1, 1};
    const cuuint32_t boxA[2] = {64, 128}, boxB[2] = {64, 64};
    CUresult r = encode(&tm[0], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(tab), dim, stride, boxA, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r == CUDA_SUCCESS)
        r = encode(&tm[1], CU_TENSOR_MAP_DATA_TYPE_UINT16, 2, const_cast<void*>(tab), dim, stride, boxB, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t tc_launch_gemm(const void* tab, int64_t nkb, int mtiles, int ntiles, const void* items,
                           const int32_t* unit_item0, int grid, int kcb, double* P, double* F, int64_t lo_off,
                           const AxisMap& ax, int nch, const double scale[4], int32_t* err, uint64_t limit_ns, int mode,
                           cudaStream_t s)
{
    static_assert(GemmCfg<0>::STAGES * GemmCfg<0>::STAGE_BYTES == GemmCfg<2>::STAGES * GemmCfg<2>::STAGE_BYTES,
                  "one dynamic shared-memory size for every mode");
    static bool attr = false;
    const int smem = GemmCfg<0>::STAGES * GemmCfg<0>::STAGE_BYTES + 1024;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_f16x3<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_gemm_f16x3<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if ((mode != 0 && mode != 2) || (mode == 2 && ((grid & 1) || (mtiles & 1)))) return cudaErrorInvalidValue;
    // MODE 2: tensor maps over the chunk's tables as rows of 128 bytes
    const int64_t rows = (int64_t)(2 * mtiles + 2 * ntiles) * nkb * (TC_BLOCK_BYTES / 128);
    CUtensorMap tm[2];
    memset(tm, 0, sizeof(tm));
    if (mode == 2) {
        if (rows > 0x7fffffffll) return cudaErrorInvalidValue;   // row coordinates are 32-bit
        const cudaError_t e = encode_row_maps(tab, rows, tm);
        if (e != cudaSuccess) return e;
    }
    GemmArgs ga;
    ga.A_hi = (const uint8_t*)tab;
    ga.A_lo = ga.A_hi + (size_t)mtiles * nkb * TC_BLOCK_BYTES;
    ga.B_hi = ga.A_lo + (size_t)mtiles * nkb * TC_BLOCK_BYTES;
    ga.B_lo = ga.B_hi + (size_t)ntiles * nkb * TC_BLOCK_BYTES;
    ga.nkb = nkb;
    ga.items = (const GemmItem*)items;
    ga.unit_item0 = unit_item0;
    ga.kcb = kcb;
    ga.P = P;
    ga.F = F;
    ga.lo_off = lo_off;
    ga.ax = ax;
    ga.nch = nch;
    for (int c = 0; c < 4; ++c) ga.scale[c] = (float)scale[c];
    ga.err = err;
    ga.limit_ns = limit_ns;
    ga.mtiles = mtiles;
    ga.ntiles = ntiles;
    if (mode == 0) {
        k_gemm_f16x3<0><<<grid, TC_THREADS, smem, s>>>(ga, tm[0], tm[1]);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(TC_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_gemm_f16x3<2>, ga, tm[0], tm[1]);
}

cudaError_t tc_launch_gemm_rays(const float4* cpos, const float4* cw, const int64_t* kb_cell0, const int32_t* kb_ncell,
                                const RayProjection& pr, const float2* qy, int nyg, const float2* qz, int nzg,
                                const float wscale[4], const void* items, const int32_t* unit_item0, int grid, int kcb,
                                double* P, double* F, int64_t lo_off, const AxisMap& ax, int nch,
                                const double scale[4], int32_t* err, uint64_t limit_ns, cudaStream_t s)
{
    if (nyg < 0 || nyg > RF_MAX_COARSE || nzg < 0 || nzg > 64 || nch != 4 || kcb < 1) return cudaErrorInvalidValue;
    if (pr.ray_sc && (pr.n_rl < 1 || pr.n_rl > RF_MAX_SLOTS || pr.n_rays < 1 || pr.n_cells < 1))
        return cudaErrorInvalidValue;
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(k_gemm_ray_fused, cudaFuncAttributeMaxDynamicSharedMemorySize, RF_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    GemmArgs ga;
    memset(&ga, 0, sizeof(ga));
    ga.items = (const GemmItem*)items;
    ga.unit_item0 = unit_item0;
    ga.kcb = kcb;
    ga.P = P;
    ga.F = F;
    ga.lo_off = lo_off;
    ga.ax = ax;
    ga.nch = nch;
    for (int c = 0; c < 4; ++c) ga.scale[c] = (float)scale[c];
    ga.err = err;
    ga.limit_ns = limit_ns;
    ga.mtiles = 1;
    ga.ntiles = 1;
    RayFusedArgs ra;
    memset(&ra, 0, sizeof(ra));
    ra.cpos = cpos;
    ra.cw = cw;
    ra.kb_cell0 = kb_cell0;
    ra.kb_ncell = kb_ncell;
    ra.project = pr.ray_sc ? 1 : 0;
    ra.ray_sc = pr.ray_sc;
    ra.n_cells = pr.n_cells;
    ra.slot0 = pr.slot0;
    ra.n_rays = pr.n_rays;
    ra.n_rl = pr.n_rl;
    ra.wscale = make_float4(wscale[0], wscale[1], wscale[2], wscale[3]);
    ra.nyg = nyg;
    ra.nzg = nzg;
    for (int a = 0; a < nyg; ++a) ra.qy[a] = qy[a];
    for (int b = 0; b < nzg; ++b) ra.qz[b] = qz[b];
    if (grid <= 0) return cudaSuccess;
    k_gemm_ray_fused<<<grid, RF_THREADS, RF_SMEM, s>>>(ga, ra);
    return cudaGetLastError();
}

cudaError_t tc_launch_reduce(const double* P, const void* reds, int n_red, const AxisMap& ax, int ntiles, int nch,
                             const double scale[4], double* F, int64_t lo_off, cudaStream_t s)
{
    Scale4 sc;
    for (int c = 0; c < 4; ++c) sc.v[c] = (float)scale[c];
    const int64_t n = (int64_t)n_red * nch * ax.nyg * ax.nzg;
    if (n == 0) return cudaSuccess;   // every item of the chunk wrote its output directly
    k_gemm_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(P, (const RedDesc*)reds, n_red, ax, ntiles, nch, sc, F,
                                                              lo_off);
    return cudaGetLastError();
}

size_t tc_item_bytes() { return sizeof(GemmItem); }
size_t tc_red_bytes() { return sizeof(RedDesc); }
size_t tc_block_bytes() { return TC_BLOCK_BYTES; }
int tc_block_cells() { return TC_BK; }
float tc_operand_scale() { return TC_SCALE; }

}  // namespace nms
