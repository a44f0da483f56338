// Batch kernels of the tensor path: per-rotation preparation into stacked
// arrays, and the accumulation of many amplitudes F_o (objects and/or
// rotations) into the Hermitian products G and the total amplitude.
//
// Paper, Sec. "Summation approach", interparticle decomposition:
//   |sum_k F_k e^{-iq.r^k}|^2 = sum_k |F_k|^2 + cross terms;
// the dilute part is G_dil = sum_k F_k F_k^dagger, the total amplitude is
// F_tot = sum_k F_k exp(-i q.(R r^k)) (object k moved to its rotated centre),
// and orientation averages add G over rotations.
//
// GB300: FP64 is slow on this part, so the products are formed in FP32 from
// the FP64 amplitudes and accumulated in two-float (hi, lo) registers; the
// FP64 arrays in HBM are touched once per batch.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "nms_internal.h"

namespace nms {

__device__ __forceinline__ float4 split_pos(double y, double z)
{
    const float yh = (float)y, zh = (float)z;
    return make_float4(yh, (float)(y - (double)yh), zh, (float)(z - (double)zh));
}

// Rotated positions (global R(x + r^k) or local R x) and rotated weights of
// one rotation, written at the given offset of the stacked arrays; weights
// of weight set s (nuc [S][n], mag [S][n][3]) go to cw[s * wstride + j].
__global__ void k_prep_rot(int64_t n, int n_sets, int64_t wstride, const double* __restrict__ pos,
                           const double* __restrict__ vol, const double* __restrict__ nuc,
                           const double* __restrict__ mag, const double* __restrict__ cen_cell, RotMat R,
                           float4* __restrict__ cpos, float4* __restrict__ cw)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2];
    if (cen_cell) {
        x += cen_cell[3 * j];
        y += cen_cell[3 * j + 1];
        z += cen_cell[3 * j + 2];
    }
    const double* r = R.m;
    cpos[j] = split_pos(r[3] * x + r[4] * y + r[5] * z, r[6] * x + r[7] * y + r[8] * z);
    const double v = vol ? vol[j] : 1.0;
    for (int st = 0; st < n_sets; ++st) {
        const int64_t js = (int64_t)st * n + j;
        const double wn = nuc ? v * nuc[js] : 0.0;
        double wx = 0.0, wy = 0.0, wz = 0.0;
        if (mag) {
            const double mx = mag[3 * js], my = mag[3 * js + 1], mz = mag[3 * js + 2];
            wx = v * (r[0] * mx + r[1] * my + r[2] * mz);
            wy = v * (r[3] * mx + r[4] * my + r[5] * mz);
            wz = v * (r[6] * mx + r[7] * my + r[8] * mz);
        }
        cw[(int64_t)st * wstride + j] = make_float4((float)wn, (float)wx, (float)wy, (float)wz);
    }
}

cudaError_t launch_prep_rot(const Plan& p, const RotMat& R, bool global, float4* cpos, float4* cw, int64_t wstride,
                            cudaStream_t s)
{
    const int64_t n = p.n_cells;
    k_prep_rot<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, p.n_sets, wstride, p.d_pos, p.d_vol, p.d_nuc, p.d_mag,
                                                           global ? p.d_cen_cell : nullptr, R, cpos, cw);
    return cudaGetLastError();
}

// Rotated centre of each output: (Y, Z) rows of R_rot r^obj, as two-float.
__global__ void k_centres(int n_out, const int32_t* __restrict__ out_obj, const int32_t* __restrict__ out_rot,
                          int rot0, const double* __restrict__ rot, const double* __restrict__ cen,
                          float4* __restrict__ cyz)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_out) return;
    const double* r = rot + 9 * (int64_t)(rot0 + out_rot[o]);
    const double* c = cen + 3 * (int64_t)out_obj[o];
    cyz[o] = split_pos(r[3] * c[0] + r[4] * c[1] + r[5] * c[2], r[6] * c[0] + r[7] * c[1] + r[8] * c[2]);
}

cudaError_t launch_centres(int n_out, const int32_t* out_obj, const int32_t* out_rot, int rot0, const double* rot,
                           const double* cen, float4* cyz, cudaStream_t s)
{
    k_centres<<<(n_out + 127) / 128, 128, 0, s>>>(n_out, out_obj, out_rot, rot0, rot, cen, cyz);
    return cudaGetLastError();
}

__device__ __forceinline__ void ts_acc(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

__device__ __forceinline__ int pair_idx(int a, int b)  // a < b
{
    return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}

// Complex value idx of an amplitude array as FP32: two-float
// (re hi, re lo, im hi, im lo) when TF, else FP64 (re, im).
template <bool TF>
__device__ __forceinline__ float2 load_c(const void* __restrict__ F, int64_t idx)
{
    if constexpr (TF) {
        const float4 v = reinterpret_cast<const float4*>(F)[idx];
        return make_float2(v.x + v.y, v.z + v.w);
    } else {
        const double2 v = reinterpret_cast<const double2*>(F)[idx];
        return make_float2((float)v.x, (float)v.y);
    }
}

// G[16][npix] += sum_o F_o F_o^dagger (F_o: [4][npix] complex at F + o *
// ostride2 complex values; two-float GEMM outputs or FP64 totals).
template <bool TF>
__global__ void k_gacc_batch(const void* __restrict__ F, int n_out, int64_t ostride2, int64_t npix,
                             double* __restrict__ G)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    float hi[16], lo[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) { hi[k] = 0.f; lo[k] = 0.f; }
    for (int o = 0; o < n_out; ++o) {
        float2 f[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) f[c] = load_c<TF>(F, (int64_t)o * ostride2 + (int64_t)c * npix + p);
#pragma unroll
        for (int a = 0; a < 4; ++a) ts_acc(hi[a], lo[a], fmaf(f[a].x, f[a].x, f[a].y * f[a].y));
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = a + 1; b < 4; ++b) {
                const int k = pair_idx(a, b);
                ts_acc(hi[4 + 2 * k], lo[4 + 2 * k], fmaf(f[a].x, f[b].x, f[a].y * f[b].y));
                ts_acc(hi[5 + 2 * k], lo[5 + 2 * k], fmaf(f[a].y, f[b].x, -f[a].x * f[b].y));
            }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) G[(int64_t)k * npix + p] += (double)hi[k] + (double)lo[k];
}

cudaError_t launch_gacc_batch(const double* F, int n_out, int64_t ostride, int64_t npix, double* G, bool two_float,
                              cudaStream_t s)
{
    if (n_out <= 0) return cudaSuccess;
    const unsigned blocks = (unsigned)((npix + 127) / 128);
    if (two_float) k_gacc_batch<true><<<blocks, 128, 0, s>>>(F, n_out, ostride / 2, npix, G);
    else k_gacc_batch<false><<<blocks, 128, 0, s>>>(F, n_out, ostride / 2, npix, G);
    return cudaGetLastError();
}

// FP64 amplitudes from two-float ones: (re hi + re lo, im hi + im lo)
__global__ void k_tf_to_f64(const float4* __restrict__ src, double2* __restrict__ dst, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4 v = src[i];
    dst[i] = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
}

cudaError_t launch_tf_to_f64(const double* src, double* dst, int64_t n_complex, cudaStream_t s)
{
    k_tf_to_f64<<<(unsigned)((n_complex + 255) / 256), 256, 0, s>>>(reinterpret_cast<const float4*>(src),
                                                                    reinterpret_cast<double2*>(dst), n_complex);
    return cudaGetLastError();
}

// One pass over a batch of object amplitudes F_o (two-float [n_out][4][npix]):
//   G_dil[16][p]              += F_o F_o^dagger                  (dilute part)
//   Ftot[out_rot[o]][c][p]    += F_o[c][p] exp(-i (q_y cy_o + q_z cz_o))
// The shift phase is a two-float product in turns reduced exactly (as in the
// direct sum).  Outputs are ordered by rotation, so each thread flushes its
// two-float shifted sums to FP64 once per rotation.  The next output's
// amplitudes are loaded while the current one is processed, so each thread
// keeps two outputs' loads in flight.
__device__ __forceinline__ void load_f(const float4* __restrict__ F, int64_t o, int64_t ostride2, int64_t npix,
                                       int64_t p, float4* v)
{
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = F[o * ostride2 + (int64_t)c * npix + p];
}

__global__ void __launch_bounds__(128)
k_dilute_shift_batch(const float4* __restrict__ F, int n_out, int64_t ostride2, const float4* __restrict__ cyz,
                     const int32_t* __restrict__ out_rot, const float4* __restrict__ qturn, int64_t npix,
                     double* __restrict__ Gdil, double2* __restrict__ Ftot, int64_t tstride2)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix || n_out <= 0) return;
    const float4 q = qturn[p];
    float gh[16], gl[16], th[8], tl[8];
#pragma unroll
    for (int k = 0; k < 16; ++k) { gh[k] = 0.f; gl[k] = 0.f; }
#pragma unroll
    for (int k = 0; k < 8; ++k) { th[k] = 0.f; tl[k] = 0.f; }
    float4 nxt[4];
    load_f(F, 0, ostride2, npix, p, nxt);
    int cur = out_rot[0];
    for (int o = 0; o < n_out; ++o) {
        float2 f[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) f[c] = make_float2(nxt[c].x + nxt[c].y, nxt[c].z + nxt[c].w);
        if (o + 1 < n_out) load_f(F, o + 1, ostride2, npix, p, nxt);
        const int r = out_rot[o];
        if (r != cur) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                double2* t = Ftot + (int64_t)cur * tstride2 + (int64_t)c * npix + p;
                double2 v = *t;
                v.x += (double)th[2 * c] + (double)tl[2 * c];
                v.y += (double)th[2 * c + 1] + (double)tl[2 * c + 1];
                *t = v;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) { th[k] = 0.f; tl[k] = 0.f; }
            cur = r;
        }
        // dilute: F_o F_o^dagger
#pragma unroll
        for (int a = 0; a < 4; ++a) ts_acc(gh[a], gl[a], fmaf(f[a].x, f[a].x, f[a].y * f[a].y));
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = a + 1; b < 4; ++b) {
                const int k = pair_idx(a, b);
                ts_acc(gh[4 + 2 * k], gl[4 + 2 * k], fmaf(f[a].x, f[b].x, f[a].y * f[b].y));
                ts_acc(gh[5 + 2 * k], gl[5 + 2 * k], fmaf(f[a].y, f[b].x, -f[a].x * f[b].y));
            }
        // total: F_o moved to its rotated centre
        const float4 cc = cyz[o];
        const float py = q.x * cc.x;
        const float ey = fmaf(q.x, cc.x, -py) + fmaf(q.x, cc.y, q.y * cc.x);
        const float pz = q.z * cc.z;
        const float ez = fmaf(q.z, cc.z, -pz) + fmaf(q.z, cc.w, q.w * cc.z);
        const float sm = py + pz;
        const float bb = sm - py;
        const float es = (py - (sm - bb)) + (pz - bb);
        const float t = (sm - rintf(sm)) + (es + ey + ez);
        float sn, cs;
        sincospif(2.0f * t, &sn, &cs);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            ts_acc(th[2 * c], tl[2 * c], fmaf(f[c].x, cs, f[c].y * sn));
            ts_acc(th[2 * c + 1], tl[2 * c + 1], fmaf(f[c].y, cs, -f[c].x * sn));
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double2* t = Ftot + (int64_t)cur * tstride2 + (int64_t)c * npix + p;
        double2 v = *t;
        v.x += (double)th[2 * c] + (double)tl[2 * c];
        v.y += (double)th[2 * c + 1] + (double)tl[2 * c + 1];
        *t = v;
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) Gdil[(int64_t)k * npix + p] += (double)gh[k] + (double)gl[k];
}

cudaError_t launch_dilute_shift_batch(const double* F, int n_out, int64_t ostride, const float4* cyz,
                                      const int32_t* out_rot, const float4* qturn, int64_t npix, double* Gdil,
                                      double* Ftot, int64_t tstride, cudaStream_t s)
{
    if (n_out <= 0) return cudaSuccess;
    k_dilute_shift_batch<<<(unsigned)((npix + 127) / 128), 128, 0, s>>>(
        reinterpret_cast<const float4*>(F), n_out, ostride / 2, cyz, out_rot, qturn, npix, Gdil,
        reinterpret_cast<double2*>(Ftot), tstride / 2);
    return cudaGetLastError();
}

}  // namespace nms

namespace nms {

// Per-object azimuthal binning of one response evaluated from a batch of
// amplitudes: Iobj[obj[o]][bin(p)] += resp(F_o, p) over the pixels of each
// bin (Eq. iqazi on the ring bins of the detector).  The response is formed
// in FP32 from the two-float amplitudes:
//   N  = s |F_N|^2,  M = s b^2 (|F_M|^2 - |qhat.F_M|^2)   (|Q|^2, Eq. HJdef)
//   P  = s b^2 |u.F_M|^2, u = P - qhat (qhat.P)            (Eq. PSANSdef)
//   SF = M - P,  UNPOL = N + M.
__global__ void k_obj_bin(const float4* __restrict__ F, int n_out, const int32_t* __restrict__ out_obj,
                          const double* __restrict__ hy, const double* __restrict__ hz,
                          const int32_t* __restrict__ bin_of, int64_t npix, int nbins, int id, float s, float b,
                          float Px, float Py, float Pz, double* __restrict__ Iobj)
{
    extern __shared__ float s_bins[];
    const int o = blockIdx.y;
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) s_bins[k] = 0.f;
    __syncthreads();
    const float4* Fo = F + (int64_t)o * 4 * npix;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const int bin = bin_of[p];
        if (bin < 0) continue;
        float2 f[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const float4 v = Fo[(int64_t)c * npix + p];
            f[c] = make_float2(v.x + v.y, v.z + v.w);
        }
        const float y = (float)hy[p], z = (float)hz[p];
        const float nn = f[0].x * f[0].x + f[0].y * f[0].y;
        const float mm = f[1].x * f[1].x + f[1].y * f[1].y + f[2].x * f[2].x + f[2].y * f[2].y + f[3].x * f[3].x +
                         f[3].y * f[3].y;
        const float pr = y * f[2].x + z * f[3].x, pi = y * f[2].y + z * f[3].y;
        const float vM = s * b * b * (mm - (pr * pr + pi * pi));
        float v;
        if (id == NMS_RESP_N) {
            v = s * nn;
        } else if (id == NMS_RESP_M) {
            v = vM;
        } else if (id == NMS_RESP_UNPOL) {
            v = s * nn + vM;
        } else {
            const float qp = y * Py + z * Pz;
            const float ux = Px, uy = Py - y * qp, uz = Pz - z * qp;
            const float ur = ux * f[1].x + uy * f[2].x + uz * f[3].x, ui = ux * f[1].y + uy * f[2].y + uz * f[3].y;
            const float vP = s * b * b * (ur * ur + ui * ui);
            v = id == NMS_RESP_P ? vP : vM - vP;
        }
        atomicAdd(&s_bins[bin], v);
    }
    __syncthreads();
    double* dst = Iobj + (int64_t)out_obj[o] * nbins;
    for (int k = threadIdx.x; k < nbins; k += blockDim.x)
        if (s_bins[k] != 0.f) atomicAdd(&dst[k], (double)s_bins[k]);
}

cudaError_t launch_obj_bin(const double* F, int n_out, const int32_t* out_obj, const Plan& p, const int32_t* bin_of,
                           int nbins, int id, double* Iobj, cudaStream_t s)
{
    if (n_out <= 0) return cudaSuccess;
    const int64_t pix_blocks = std::min<int64_t>((p.npix + 1023) / 1024, 64);
    dim3 grid((unsigned)pix_blocks, (unsigned)n_out);
    k_obj_bin<<<grid, 256, nbins * sizeof(float), s>>>(reinterpret_cast<const float4*>(F), n_out, out_obj, p.d_hy,
                                                       p.d_hz, bin_of, p.npix, nbins, id, (float)(1.0 / p.V),
                                                       (float)p.bH, (float)p.P[0], (float)p.P[1], (float)p.P[2], Iobj);
    return cudaGetLastError();
}

}  // namespace nms
