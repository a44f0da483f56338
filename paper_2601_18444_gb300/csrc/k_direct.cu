// Rotation/weights preparation and the FP32 direct Fourier sum.
//
// Paper, Sec. "Real-space input data": X, Y, Z = R (x^{kl} + r^k); Sec.
// "Summation approach": nu^R = +sum nu cos(Psi), nu^I = -sum nu sin(Psi) with
// Psi = q_y Y + q_z Z (the phase function at q_y = q sin t, q_z = q cos t).
//
// GB300 design: the direct sum is bound by the FP32 and MUFU pipes.  Each
// thread owns PPT pixels, cells are staged through shared memory, and the
// phase is carried in *turns* (t = Psi / 2 pi) as a two-float product so that
// the reduction t - rint(t) is exact; sincospif() then evaluates the reduced
// angle.  Accumulation runs in FP32 over groups of 8 cells and is folded into
// two-float (hi, lo) running sums, which keeps the summation error at the
// 1e-7 level even for coherent pixels and millions of cells.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "nms_internal.h"

namespace nms {

// ------------------------------------------------------------------ prep
__device__ __forceinline__ float4 split2(double y, double z)
{
    float yh = (float)y;
    float yl = (float)(y - (double)yh);
    float zh = (float)z;
    float zl = (float)(z - (double)zh);
    return make_float4(yh, yl, zh, zl);
}

__global__ void k_prep(int64_t n, const double* __restrict__ pos, const double* __restrict__ vol,
                       const double* __restrict__ nuc, const double* __restrict__ mag,
                       const double* __restrict__ cen_cell, double r0, double r1, double r2, double r3,
                       double r4, double r5, double r6, double r7, double r8, float4* __restrict__ cpos,
                       float4* __restrict__ cposl, float4* __restrict__ cw, double* __restrict__ yz,
                       double* __restrict__ yzl, double* __restrict__ w64)
{
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2];
    // local rotated coordinates (rows 2 and 3 of R x)
    double Yl = r3 * x + r4 * y + r5 * z;
    double Zl = r6 * x + r7 * y + r8 * z;
    double Yg = Yl, Zg = Zl;
    if (cen_cell) {
        double cx = cen_cell[3 * j], cy = cen_cell[3 * j + 1], cz = cen_cell[3 * j + 2];
        double gx = x + cx, gy = y + cy, gz = z + cz;
        Yg = r3 * gx + r4 * gy + r5 * gz;
        Zg = r6 * gx + r7 * gy + r8 * gz;
    }
    cpos[j] = split2(Yg, Zg);
    if (cposl) cposl[j] = split2(Yl, Zl);
    double v = vol ? vol[j] : 1.0;
    double wn = nuc ? v * nuc[j] : 0.0;
    double wx = 0.0, wy = 0.0, wz = 0.0;
    if (mag) {
        double mx = mag[3 * j], my = mag[3 * j + 1], mz = mag[3 * j + 2];
        wx = v * (r0 * mx + r1 * my + r2 * mz);
        wy = v * (r3 * mx + r4 * my + r5 * mz);
        wz = v * (r6 * mx + r7 * my + r8 * mz);
    }
    cw[j] = make_float4((float)wn, (float)wx, (float)wy, (float)wz);
    if (yz) {
        yz[j] = Yg;
        yz[n + j] = Zg;
    }
    if (yzl) {
        yzl[j] = Yl;
        yzl[n + j] = Zl;
    }
    if (w64) {
        w64[j] = wn;
        w64[n + j] = wx;
        w64[2 * n + j] = wy;
        w64[3 * n + j] = wz;
    }
}

// max over cells and weight sets of V_j |N_j| and V_j |M_j| (the operand
// scales of the tensor path).  Non-negative doubles order like their bit
// patterns, so the maxima are integer atomics on those patterns.
__global__ void k_weight_max(int64_t n, int n_sets, const double* __restrict__ vol, const double* __restrict__ nuc,
                             const double* __restrict__ mag, unsigned long long* __restrict__ out)
{
    double wn = 0.0, wm = 0.0;
    for (int64_t js = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; js < (int64_t)n_sets * n;
         js += (int64_t)gridDim.x * blockDim.x) {
        const double v = vol ? fabs(vol[js % n]) : 1.0;
        if (nuc) wn = fmax(wn, v * fabs(nuc[js]));
        if (mag) {
            const double mx = mag[3 * js], my = mag[3 * js + 1], mz = mag[3 * js + 2];
            wm = fmax(wm, v * sqrt(mx * mx + my * my + mz * mz));
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        wn = fmax(wn, __shfl_xor_sync(0xffffffffu, wn, o));
        wm = fmax(wm, __shfl_xor_sync(0xffffffffu, wm, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&out[0], (unsigned long long)__double_as_longlong(wn));
        atomicMax(&out[1], (unsigned long long)__double_as_longlong(wm));
    }
}

cudaError_t launch_weight_max(const Plan& p, double wmax[2], cudaStream_t s)
{
    unsigned long long* d = nullptr;
    cudaError_t e = cudaMallocAsync((void**)&d, 2 * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    unsigned long long h[2] = {0, 0};
    e = cudaMemsetAsync(d, 0, sizeof(h), s);
    const int64_t total = (int64_t)p.n_sets * p.n_cells;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 8 * device_sm_count()));
    if (e == cudaSuccess) {
        k_weight_max<<<blocks, 256, 0, s>>>(p.n_cells, p.n_sets, p.d_vol, p.d_nuc, p.d_mag, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    wmax[0] = __builtin_bit_cast(double, h[0]);
    wmax[1] = __builtin_bit_cast(double, h[1]);
    return cudaSuccess;
}

cudaError_t launch_prep(Plan& p, const double* R, cudaStream_t s, int set)
{
    int64_t n = p.n_cells;
    int th = 256;
    int64_t bl = (n + th - 1) / th;
    // weight set `set` of nuc [S][n] and mag [S][n][3]
    const double* nuc = p.d_nuc ? p.d_nuc + (size_t)set * n : nullptr;
    const double* mag = p.d_mag ? p.d_mag + (size_t)set * 3 * n : nullptr;
    k_prep<<<(unsigned)bl, th, 0, s>>>(n, p.d_pos, p.d_vol, nuc, mag, p.d_cen_cell, R[0], R[1], R[2],
                                       R[3], R[4], R[5], R[6], R[7], R[8], p.d_cpos,
                                       p.d_cposl != p.d_cpos ? p.d_cposl : nullptr, p.d_cw, p.d_yz,
                                       p.d_yzl != p.d_yz ? p.d_yzl : nullptr, p.d_w64);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ direct sum
constexpr int DIRECT_THREADS = 256;
constexpr int DIRECT_PPT = 2;       // pixels per thread
constexpr int DIRECT_TILE = 512;    // cells per shared-memory tile
constexpr int DIRECT_GROUP = 8;     // cells per FP32 partial before the two-float fold

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x)
{
    float s = hi + x;
    float bb = s - hi;
    float e = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo += e;
}

template <bool COMP>
__device__ __forceinline__ void phase_sincos(const float4 q, const float4 c, float& sn, float& cs)
{
    float t;
    if (COMP) {
        // two-float products (q_y' Y) and (q_z' Z) in turns, exact reduction
        float py = q.x * c.x;
        float ey = fmaf(q.x, c.x, -py) + fmaf(q.x, c.y, q.y * c.x);
        float pz = q.z * c.z;
        float ez = fmaf(q.z, c.z, -pz) + fmaf(q.z, c.w, q.w * c.z);
        float s = py + pz;
        float bb = s - py;
        float es = (py - (s - bb)) + (pz - bb);
        float n = rintf(s);
        t = (s - n) + (es + ey + ez);
    } else {
        t = fmaf(q.x, c.x, q.z * c.z);
    }
    sincospif(2.0f * t, &sn, &cs);
}

template <bool COMP>
__global__ void __launch_bounds__(DIRECT_THREADS)
k_direct(const float4* __restrict__ cpos, const float4* __restrict__ cw, int64_t c0, int64_t c1,
         const float4* __restrict__ qturn, int64_t npix, double* __restrict__ part)
{
    __shared__ float4 s_pos[DIRECT_TILE];
    __shared__ float4 s_w[DIRECT_TILE];
    const int splits = gridDim.y;
    const int64_t ncell = c1 - c0;
    const int64_t per = (ncell + splits - 1) / splits;
    const int64_t b0 = c0 + (int64_t)blockIdx.y * per;
    const int64_t b1 = min(c1, b0 + per);

    int64_t pix[DIRECT_PPT];
    float4 q[DIRECT_PPT];
    float hi[DIRECT_PPT][8], lo[DIRECT_PPT][8];
#pragma unroll
    for (int k = 0; k < DIRECT_PPT; ++k) {
        pix[k] = (int64_t)blockIdx.x * DIRECT_THREADS * DIRECT_PPT + k * DIRECT_THREADS + threadIdx.x;
        q[k] = pix[k] < npix ? qturn[pix[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int a = 0; a < 8; ++a) { hi[k][a] = 0.f; lo[k][a] = 0.f; }
    }

    for (int64_t t0 = b0; t0 < b1; t0 += DIRECT_TILE) {
        const int nt = (int)min((int64_t)DIRECT_TILE, b1 - t0);
        __syncthreads();
        for (int i = threadIdx.x; i < nt; i += DIRECT_THREADS) {
            s_pos[i] = cpos[t0 + i];
            s_w[i] = cw[t0 + i];
        }
        // zero-weight padding up to a whole group keeps the inner loop branch-free
        for (int i = nt + threadIdx.x; i < ((nt + DIRECT_GROUP - 1) / DIRECT_GROUP) * DIRECT_GROUP;
             i += DIRECT_THREADS) {
            s_pos[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            s_w[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const int ng = (nt + DIRECT_GROUP - 1) / DIRECT_GROUP;
        for (int g = 0; g < ng; ++g) {
            float acc[DIRECT_PPT][8];
#pragma unroll
            for (int k = 0; k < DIRECT_PPT; ++k)
#pragma unroll
                for (int a = 0; a < 8; ++a) acc[k][a] = 0.f;
#pragma unroll 4
            for (int u = 0; u < DIRECT_GROUP; ++u) {
                const float4 c = s_pos[g * DIRECT_GROUP + u];
                const float4 w = s_w[g * DIRECT_GROUP + u];
#pragma unroll
                for (int k = 0; k < DIRECT_PPT; ++k) {
                    float sn, cs;
                    phase_sincos<COMP>(q[k], c, sn, cs);
                    acc[k][0] = fmaf(w.x, cs, acc[k][0]);
                    acc[k][1] = fmaf(-w.x, sn, acc[k][1]);
                    acc[k][2] = fmaf(w.y, cs, acc[k][2]);
                    acc[k][3] = fmaf(-w.y, sn, acc[k][3]);
                    acc[k][4] = fmaf(w.z, cs, acc[k][4]);
                    acc[k][5] = fmaf(-w.z, sn, acc[k][5]);
                    acc[k][6] = fmaf(w.w, cs, acc[k][6]);
                    acc[k][7] = fmaf(-w.w, sn, acc[k][7]);
                }
            }
#pragma unroll
            for (int k = 0; k < DIRECT_PPT; ++k)
#pragma unroll
                for (int a = 0; a < 8; ++a) two_sum_acc(hi[k][a], lo[k][a], acc[k][a]);
        }
    }
    // partial layout [split][4][npix][2]
    double* out = part + (int64_t)blockIdx.y * 8 * npix;
#pragma unroll
    for (int k = 0; k < DIRECT_PPT; ++k) {
        if (pix[k] >= npix) continue;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double re = (double)hi[k][2 * c] + (double)lo[k][2 * c];
            double im = (double)hi[k][2 * c + 1] + (double)lo[k][2 * c + 1];
            reinterpret_cast<double2*>(out)[(int64_t)c * npix + pix[k]] = make_double2(re, im);
        }
    }
}

cudaError_t launch_direct(const Plan& p, const float4* cpos, int64_t c0, int64_t c1, bool comp, int splits,
                          cudaStream_t s)
{
    const int64_t per_block = (int64_t)DIRECT_THREADS * DIRECT_PPT;
    dim3 grid((unsigned)((p.npix + per_block - 1) / per_block), (unsigned)splits);
    if (comp)
        k_direct<true><<<grid, DIRECT_THREADS, 0, s>>>(cpos, p.d_cw, c0, c1, p.d_qturn, p.npix, p.d_Fpart);
    else
        k_direct<false><<<grid, DIRECT_THREADS, 0, s>>>(cpos, p.d_cw, c0, c1, p.d_qturn, p.npix, p.d_Fpart);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ split reduction
__global__ void k_reduce_splits(const double* __restrict__ part, int splits, int64_t m, double* __restrict__ out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double acc = 0.0;
    for (int sp = 0; sp < splits; ++sp) acc += part[(int64_t)sp * m + i];
    out[i] = acc;
}

cudaError_t launch_reduce_splits(const Plan& p, int splits, double* out, cudaStream_t s)
{
    int64_t m = 8 * p.npix;
    k_reduce_splits<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(p.d_Fpart, splits, m, out);
    return cudaGetLastError();
}

}  // namespace nms
