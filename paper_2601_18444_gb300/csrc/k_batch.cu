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
#include "tc_ptx.cuh"

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

// The same for nrl rotations in one launch: rotation rot0 + y of the device
// array rot [n_rot][9] (row-major) into the slot at y * n of the stacked arrays.
__global__ void k_prep_rot_batch(int64_t n, int n_sets, int64_t wstride, const double* __restrict__ pos,
                                 const double* __restrict__ vol, const double* __restrict__ nuc,
                                 const double* __restrict__ mag, const double* __restrict__ cen_cell,
                                 const double* __restrict__ rot, int rot0, float4* __restrict__ cpos,
                                 float4* __restrict__ cw)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int rl = blockIdx.y;
    const double* r = rot + 9 * (int64_t)(rot0 + rl);
    double x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2];
    if (cen_cell) {
        x += cen_cell[3 * j];
        y += cen_cell[3 * j + 1];
        z += cen_cell[3 * j + 2];
    }
    const int64_t o = (int64_t)rl * n + j;
    cpos[o] = split_pos(r[3] * x + r[4] * y + r[5] * z, r[6] * x + r[7] * y + r[8] * z);
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
        cw[(int64_t)st * wstride + o] = make_float4((float)wn, (float)wx, (float)wy, (float)wz);
    }
}

cudaError_t launch_prep_rot_batch(const Plan& p, const double* d_rot, int rot0, int nrl, bool global, float4* cpos,
                                  float4* cw, int64_t wstride, cudaStream_t s)
{
    const int64_t n = p.n_cells;
    if (n <= 0 || nrl <= 0) return cudaSuccess;
    k_prep_rot_batch<<<dim3((unsigned)((n + 255) / 256), (unsigned)nrl), 256, 0, s>>>(
        n, p.n_sets, wstride, p.d_pos, p.d_vol, p.d_nuc, p.d_mag, global ? p.d_cen_cell : nullptr, d_rot, rot0, cpos,
        cw);
    return cudaGetLastError();
}

// Polar detector on the tensor path (rays).  On the ray at angle theta the
// pixel q = |q| (sin theta, cos theta) (the POLAR grid's q_y, q_z) has the
// phase q.r = |q| u with u = Y sin theta + Z cos theta, so every ray is a
// one-dimensional sum over the projections u.  Slot s = slot0 + blockIdx.y
// (rotation s / n_rays, ray s mod n_rays) gets the projection of each rotated
// position in both coordinates, (u, u), and the rotated weights as in
// k_prep_rot_batch (the weights do not depend on the ray); with cen_cell
// (plans without per-object parts) the object centres are added first.
__global__ void k_prep_ray_batch(int64_t n, int n_sets, int64_t wstride, const double* __restrict__ pos,
                                 const double* __restrict__ vol, const double* __restrict__ nuc,
                                 const double* __restrict__ mag, const double* __restrict__ cen_cell,
                                 const double* __restrict__ rot, const double2* __restrict__ ray_sc, int n_rays,
                                 int slot0, float4* __restrict__ cpos, float4* __restrict__ cw)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int rl = blockIdx.y;
    const int slot = slot0 + rl;
    const double* r = rot + 9 * (int64_t)(slot / n_rays);
    const double2 sc = ray_sc[slot % n_rays];   // (sin theta, cos theta)
    double x = pos[3 * j], y = pos[3 * j + 1], z = pos[3 * j + 2];
    if (cen_cell) {
        x += cen_cell[3 * j];
        y += cen_cell[3 * j + 1];
        z += cen_cell[3 * j + 2];
    }
    const double u = sc.x * (r[3] * x + r[4] * y + r[5] * z) + sc.y * (r[6] * x + r[7] * y + r[8] * z);
    const int64_t o = (int64_t)rl * n + j;
    cpos[o] = split_pos(u, u);
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
        cw[(int64_t)st * wstride + o] = make_float4((float)wn, (float)wx, (float)wy, (float)wz);
    }
}

// The same slots from inputs rotated once per rotation: rpos [n_rot][n]
// holds the rotated (Y, Z) of every cell as two-float and rw
// [set][n_rot][n] its weights (k_prep_rot_batch over all rotations).  The
// projection u = Y sin theta + Z cos theta is formed in two-float FP32
// arithmetic (products made exact by FMA, sums by TwoSum; relative error
// about 2^-44 of |Y| + |Z|, far below what the phase tables resolve), so the
// per-ray work has no FP64; the weights are copied.
__device__ __forceinline__ void ray_two_prod(float a_h, float a_l, float b_h, float b_l, float& p, float& e)
{
    p = a_h * b_h;
    e = fmaf(a_h, b_h, -p) + fmaf(a_h, b_l, a_l * b_h);
}

__global__ void k_prep_ray_from_rot(int64_t n, int n_sets, int64_t wstride, int64_t rwstride,
                                    const float4* __restrict__ rpos, const float4* __restrict__ rw,
                                    const float4* __restrict__ ray_sc_tf, int n_rays, int slot0,
                                    float4* __restrict__ cpos, float4* __restrict__ cw)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int rl = blockIdx.y;
    const int slot = slot0 + rl;
    const int64_t src = (int64_t)(slot / n_rays) * n + j;
    const float4 sc = ray_sc_tf[slot % n_rays];   // sin theta (hi, lo), cos theta (hi, lo)
    const float4 yz = rpos[src];                  // Y (hi, lo), Z (hi, lo)
    float p1, e1, p2, e2;
    ray_two_prod(sc.x, sc.y, yz.x, yz.y, p1, e1);
    ray_two_prod(sc.z, sc.w, yz.z, yz.w, p2, e2);
    const float s = p1 + p2;
    const float bb = s - p1;
    const float e = ((p1 - (s - bb)) + (p2 - bb)) + (e1 + e2);
    const float uh = s + e;
    const float ul = e - (uh - s);
    const int64_t o = (int64_t)rl * n + j;
    cpos[o] = make_float4(uh, ul, uh, ul);
    for (int st = 0; st < n_sets; ++st) cw[(int64_t)st * wstride + o] = rw[(int64_t)st * rwstride + src];
}

cudaError_t launch_prep_ray_from_rot(const Plan& p, const float4* rpos, const float4* rw, int64_t rwstride,
                                     const float4* ray_sc_tf, int n_rays, int slot0, int nrl, float4* cpos, float4* cw,
                                     int64_t wstride, cudaStream_t s)
{
    const int64_t n = p.n_cells;
    if (n <= 0 || nrl <= 0) return cudaSuccess;
    k_prep_ray_from_rot<<<dim3((unsigned)((n + 255) / 256), (unsigned)nrl), 256, 0, s>>>(
        n, p.n_sets, wstride, rwstride, rpos, rw, ray_sc_tf, n_rays, slot0, cpos, cw);
    return cudaGetLastError();
}

cudaError_t launch_prep_ray_batch(const Plan& p, const double* d_rot, const double2* ray_sc, int n_rays, int slot0,
                                  int nrl, bool global, float4* cpos, float4* cw, int64_t wstride, cudaStream_t s)
{
    const int64_t n = p.n_cells;
    if (n <= 0 || nrl <= 0) return cudaSuccess;
    k_prep_ray_batch<<<dim3((unsigned)((n + 255) / 256), (unsigned)nrl), 256, 0, s>>>(
        n, p.n_sets, wstride, p.d_pos, p.d_vol, p.d_nuc, p.d_mag, global ? p.d_cen_cell : nullptr, d_rot, ray_sc,
        n_rays, slot0, cpos, cw);
    return cudaGetLastError();
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

// Rays: the projection v = Cy sin theta + Cz cos theta of each output's
// rotated centre on its ray (slot slot0 + out_rot[o]: rotation slot / n_rays,
// ray slot mod n_rays), as two-float in both coordinates, so that the shift
// factor e^{-i |q| v} separates over the ray GEMM's two axes like
// e^{-i (q_y cy + q_z cz)} on a Cartesian detector.
__global__ void k_ray_centres(int n_out, const int32_t* __restrict__ out_obj, const int32_t* __restrict__ out_rot,
                              int slot0, const double* __restrict__ rot, const double2* __restrict__ ray_sc,
                              int n_rays, const double* __restrict__ cen, float4* __restrict__ cyz)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_out) return;
    const int slot = slot0 + out_rot[o];
    const double* r = rot + 9 * (int64_t)(slot / n_rays);
    const double2 sc = ray_sc[slot % n_rays];
    const double* c = cen + 3 * (int64_t)out_obj[o];
    const double v = sc.x * (r[3] * c[0] + r[4] * c[1] + r[5] * c[2]) + sc.y * (r[6] * c[0] + r[7] * c[1] + r[8] * c[2]);
    cyz[o] = split_pos(v, v);
}

cudaError_t launch_ray_centres(int n_out, const int32_t* out_obj, const int32_t* out_rot, int slot0, const double* rot,
                               const double2* ray_sc, int n_rays, const double* cen, float4* cyz, cudaStream_t s)
{
    if (n_out <= 0) return cudaSuccess;
    k_ray_centres<<<(n_out + 127) / 128, 128, 0, s>>>(n_out, out_obj, out_rot, slot0, rot, ray_sc, n_rays, cen, cyz);
    return cudaGetLastError();
}

cudaError_t launch_centres(int n_out, const int32_t* out_obj, const int32_t* out_rot, int rot0, const double* rot,
                           const double* cen, float4* cyz, cudaStream_t s)
{
    k_centres<<<(n_out + 127) / 128, 128, 0, s>>>(n_out, out_obj, out_rot, rot0, rot, cen, cyz);
    return cudaGetLastError();
}

// Shift factors of each output along each detector axis:
//   eyz[o][a]      = (cos, sin)(2 pi q'_y,a cy_o)   a < ny
//   eyz[o][ny + b] = (cos, sin)(2 pi q'_z,b cz_o)   b < nz
// (q' in turns, two-float; the product is reduced exactly to [-1/2, 1/2]).
// The phase of pixel (a, b) is the sum of the two (the detector-plane
// phase separates), so the per-pixel work is one complex product.
__global__ void k_shift_factors(int n_out, const float4* __restrict__ cyz, const float2* __restrict__ qy, int ny,
                                const float2* __restrict__ qz, int nz, float2* __restrict__ eyz)
{
    const int o = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_out || i >= ny + nz) return;
    const float4 c = cyz[o];
    const bool y = i < ny;
    const float2 q = y ? qy[i] : qz[i - ny];
    const float ch = y ? c.x : c.z, cl = y ? c.y : c.w;
    const float p = q.x * ch;
    const float e = fmaf(q.x, ch, -p) + fmaf(q.x, cl, q.y * ch);
    const float t = (p - rintf(p)) + e;
    float sn, cs;
    sincospif(2.0f * t, &sn, &cs);
    eyz[(int64_t)o * (ny + nz) + i] = make_float2(cs, sn);
}

cudaError_t launch_shift_factors(int n_out, const float4* cyz, const float2* qy, int ny, const float2* qz, int nz,
                                 float2* eyz, cudaStream_t s)
{
    if (n_out <= 0) return cudaSuccess;
    k_shift_factors<<<dim3((unsigned)((ny + nz + 127) / 128), (unsigned)n_out), 128, 0, s>>>(n_out, cyz, qy, ny, qz, nz,
                                                                                          eyz);
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

// A Hermitian product set G of one pixel holds |F_c|^2 at k = c < 4 and
// Re, Im of F_i conj(F_j) at k = 4 + 2 m, 5 + 2 m for the pair m =
// pair_idx(i, j).  Its conjugate (the set at the mirror pixel -q) changes
// the sign of the imaginary parts.
__device__ __forceinline__ double g_conj_sign(int k) { return (k >= 5 && (k & 1)) ? -1.0 : 1.0; }

// G[16][npix] += sum_o F_o F_o^dagger.  GEMM outputs (F_b, FbView layout;
// threads over the stored pixels, q_y fastest, so a warp reads contiguous
// channel rows; a pixel whose point mirror is not stored also adds the
// conjugate products there) or FP64 totals ([4][npix] complex per output at
// ostride2 complex values, threads over pixels).
template <bool TF>
__global__ void k_gacc_batch(FbView V, const double2* __restrict__ T, int n_out, int64_t ostride2, int64_t npix,
                             double* __restrict__ G)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (TF ? V.stored_pixels() : npix)) return;
    int64_t p = t;
    int a = 0, b = 0;
    if constexpr (TF) {
        a = (int)(t % V.ny);
        b = V.zs0 + (int)(t / V.ny);
        p = (int64_t)a * V.nz + b;
    }
    float hi[16], lo[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) { hi[k] = 0.f; lo[k] = 0.f; }
    for (int o = 0; o < n_out; ++o) {
        float2 f[4];
        if constexpr (TF) {
#pragma unroll
            for (int c = 0; c < 4; ++c) f[c] = V.load(o, a, b, c);
        } else {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const double2 v = T[(int64_t)o * ostride2 + (int64_t)c * npix + p];
                f[c] = make_float2((float)v.x, (float)v.y);
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) ts_acc(hi[i], lo[i], fmaf(f[i].x, f[i].x, f[i].y * f[i].y));
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = i + 1; j < 4; ++j) {
                const int k = pair_idx(i, j);
                ts_acc(hi[4 + 2 * k], lo[4 + 2 * k], fmaf(f[i].x, f[j].x, f[i].y * f[j].y));
                ts_acc(hi[5 + 2 * k], lo[5 + 2 * k], fmaf(f[i].y, f[j].x, -f[i].x * f[j].y));
            }
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) G[(int64_t)k * npix + p] += (double)hi[k] + (double)lo[k];
    if (TF && V.mirror_unstored(b)) {
        const int64_t pm = (int64_t)(V.ny - 1 - a) * V.nz + (V.nz - 1 - b);
#pragma unroll
        for (int k = 0; k < 16; ++k) G[(int64_t)k * npix + pm] += g_conj_sign(k) * ((double)hi[k] + (double)lo[k]);
    }
}

cudaError_t launch_gacc_batch(const FbView& V, int n_out, double* G, cudaStream_t s)
{
    if (n_out <= 0) return cudaSuccess;
    const int64_t npix = (int64_t)V.ny * V.nz;
    const int64_t nt = V.stored_pixels();
    k_gacc_batch<true><<<(unsigned)((nt + 127) / 128), 128, 0, s>>>(V, nullptr, n_out, 0, npix, G);
    return cudaGetLastError();
}

cudaError_t launch_gacc_totals(const double* T, int n_out, int64_t ostride, int64_t npix, double* G, cudaStream_t s)
{
    if (n_out <= 0) return cudaSuccess;
    FbView none{};
    k_gacc_batch<false><<<(unsigned)((npix + 127) / 128), 128, 0, s>>>(
        none, reinterpret_cast<const double2*>(T), n_out, ostride / 2, npix, G);
    return cudaGetLastError();
}

// Rays (polar detector, see k_prep_ray_batch): the outputs of a batch are
// the slots slot0 .. slot0 + n_out - 1 (rotation slot / n_rays, ray slot mod
// n_rays); output o holds its ray's amplitudes at |q|_i, i = k2 i1 + i2, in
// GEMM cell (a = i1, b = i2).  One thread per (ray, |q| node) adds F F^dagger
// of every output of the batch on that ray (one rotation after another, so
// no two threads update one value) into G at the POLAR pixel i n1 + ray and,
// when n1 is even (mirror), the conjugate products at the ray theta + pi,
// pixel i n1 + ray + n1 / 2: there q is negated and F(-q) = conj F(q) for
// real weights.  The amplitudes of rotation last_rot also go to F (FP64).
// G is accumulated in FP64 from the two-float amplitudes (a few values per
// pixel and rotation).
__global__ void k_ray_gacc(FbView V, int n_out, int slot0, int n_rays, int mirror, int n0, int n1, int k2,
                           int last_rot, double* __restrict__ G, double* __restrict__ Gd, double2* __restrict__ F)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_rays * n0) return;
    const int ray = (int)(t % n_rays), i = (int)(t / n_rays);
    const int a = i / k2, b = i % k2;
    const int64_t npix = (int64_t)n0 * n1;
    const int64_t p = (int64_t)i * n1 + ray;
    const int64_t pm = p + n1 / 2;
    double g[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) g[k] = 0.0;
    bool any = false;
    for (int o = (ray - slot0 % n_rays + n_rays) % n_rays; o < n_out; o += n_rays) {
        double2 f[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) f[c] = V.load_f64(o, a, b, c);
#pragma unroll
        for (int c = 0; c < 4; ++c) g[c] += f[c].x * f[c].x + f[c].y * f[c].y;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int d = c + 1; d < 4; ++d) {
                const int k = pair_idx(c, d);
                g[4 + 2 * k] += f[c].x * f[d].x + f[c].y * f[d].y;
                g[5 + 2 * k] += f[c].y * f[d].x - f[c].x * f[d].y;
            }
        if ((slot0 + o) / n_rays == last_rot)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                F[(int64_t)c * npix + p] = f[c];
                if (mirror) F[(int64_t)c * npix + pm] = make_double2(f[c].x, -f[c].y);
            }
        any = true;
    }
    if (!any) return;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        G[(int64_t)k * npix + p] += g[k];
        if (mirror) G[(int64_t)k * npix + pm] += g_conj_sign(k) * g[k];
        if (Gd) {
            Gd[(int64_t)k * npix + p] += g[k];
            if (mirror) Gd[(int64_t)k * npix + pm] += g_conj_sign(k) * g[k];
        }
    }
}

cudaError_t launch_ray_gacc(const FbView& V, int n_out, int slot0, int n_rays, int mirror, int n0, int n1, int k2,
                            int last_rot, double* G, double* Gd, double* F, cudaStream_t s)
{
    if (n_out <= 0) return cudaSuccess;
    const int64_t nt = (int64_t)n_rays * n0;
    k_ray_gacc<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(V, n_out, slot0, n_rays, mirror, n0, n1, k2, last_rot, G,
                                                            Gd, reinterpret_cast<double2*>(F));
    return cudaGetLastError();
}

// Rays with objects: after the dilute pass of a batch of nrl slots, slot
// rl holds the dilute products Gdil_b[rl] [16][npr] and the shifted total
// Ftot_b[rl] [4][npr] (complex) on its ray grid, node i = k2 i1 + i2 at
// ray-grid pixel i.  One thread per (ray, |q| node) adds, for every slot of
// the batch on that ray (rotation after rotation), the dilute products into
// G_dil and F_tot F_tot^dagger into G_tot at the POLAR pixel i n1 + ray (and
// the conjugates at the ray theta + pi when mirror), and writes F_tot of
// rotation last_rot into Ftot (FP64).
__global__ void k_ray_totals(int nrl, int slot0, int n_rays, int mirror, int n0, int n1, int64_t npr,
                             const double2* __restrict__ Ftot_b, int64_t fstride2, const double* __restrict__ Gdil_b,
                             int64_t gstride, int last_rot, double* __restrict__ Gtot, double* __restrict__ Gdil,
                             double2* __restrict__ Ftot)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n_rays * n0) return;
    const int ray = (int)(t % n_rays), i = (int)(t / n_rays);
    const int64_t npix = (int64_t)n0 * n1;
    const int64_t p = (int64_t)i * n1 + ray;
    const int64_t pm = p + n1 / 2;
    double gt[16], gd[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) { gt[k] = 0.0; gd[k] = 0.0; }
    bool any = false;
    for (int rl = (ray - slot0 % n_rays + n_rays) % n_rays; rl < nrl; rl += n_rays) {
        double2 f[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) f[c] = Ftot_b[(int64_t)rl * fstride2 + (int64_t)c * npr + i];
#pragma unroll
        for (int c = 0; c < 4; ++c) gt[c] += f[c].x * f[c].x + f[c].y * f[c].y;
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int d = c + 1; d < 4; ++d) {
                const int k = pair_idx(c, d);
                gt[4 + 2 * k] += f[c].x * f[d].x + f[c].y * f[d].y;
                gt[5 + 2 * k] += f[c].y * f[d].x - f[c].x * f[d].y;
            }
#pragma unroll
        for (int k = 0; k < 16; ++k) gd[k] += Gdil_b[(int64_t)rl * gstride + (int64_t)k * npr + i];
        if ((slot0 + rl) / n_rays == last_rot)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                Ftot[(int64_t)c * npix + p] = f[c];
                if (mirror) Ftot[(int64_t)c * npix + pm] = make_double2(f[c].x, -f[c].y);
            }
        any = true;
    }
    if (!any) return;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        Gtot[(int64_t)k * npix + p] += gt[k];
        Gdil[(int64_t)k * npix + p] += gd[k];
        if (mirror) {
            Gtot[(int64_t)k * npix + pm] += g_conj_sign(k) * gt[k];
            Gdil[(int64_t)k * npix + pm] += g_conj_sign(k) * gd[k];
        }
    }
}

cudaError_t launch_ray_totals(int nrl, int slot0, int n_rays, int mirror, int n0, int n1, int64_t npr,
                              const double* Ftot_b, int64_t fstride, const double* Gdil_b, int64_t gstride,
                              int last_rot, double* Gtot, double* Gdil, double* Ftot, cudaStream_t s)
{
    if (nrl <= 0) return cudaSuccess;
    const int64_t nt = (int64_t)n_rays * n0;
    k_ray_totals<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(
        nrl, slot0, n_rays, mirror, n0, n1, npr, reinterpret_cast<const double2*>(Ftot_b), fstride / 2, Gdil_b,
        gstride, last_rot, Gtot, Gdil, reinterpret_cast<double2*>(Ftot));
    return cudaGetLastError();
}

// FP64 amplitudes [4][npix] of one output from its F_b value (high word
// plus, for outputs of several pieces, the low word)
__global__ void k_tf_to_f64(FbView V, int64_t o, double2* __restrict__ dst)
{
    const int64_t npix = (int64_t)V.ny * V.nz;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 4 * npix) return;
    const int c = (int)(i / npix);
    const int64_t p = i % npix;
    const int a = (int)(p / V.nz), b = (int)(p % V.nz);
    dst[i] = V.load_f64(o, a, b, c);
}

cudaError_t launch_tf_to_f64(const FbView& V, int64_t o, double* dst, cudaStream_t s)
{
    const int64_t n = 4 * (int64_t)V.ny * V.nz;
    k_tf_to_f64<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(V, o, reinterpret_cast<double2*>(dst));
    return cudaGetLastError();
}

// One pass over a batch of object amplitudes F_o (FbView layout):
//   G_dil[16][p]              += F_o F_o^dagger                  (dilute part)
//   Ftot[out_rot[o]][c][p]    += F_o[c][p] exp(-i (q_y cy_o + q_z cz_o))
// The shift factor of pixel (a, b) is the product of the output's factors
// along q_y and q_z (k_shift_factors).  One thread per stored pixel; q_y
// runs fastest, so a warp reads contiguous channel rows of F_b.  When only
// the q_z >= 0 half is stored (FbView.zs0 > 0) each thread also adds the
// conjugates of its two sums at the mirror pixel -q: the product set and the
// shifted sum of -q are the conjugates of those at q.
//
// Each thread stages its own inputs of the next DS_DEPTH - 1 outputs (32 B of
// F, 16 B of shift factors) in shared memory with cp.async, so the loads in
// flight hold no registers and no thread waits on another.  The terms of
// DS_RUN consecutive outputs are accumulated by FMA into FP32 partial sums,
// which are then added into the two-float (hi, lo) totals: one TwoSum per
// run instead of one per output.  A run's FP32 sum of n terms errs by at most
// (n - 1) 2^-24 times the sum of their magnitudes.  Outputs are ordered by
// rotation; the shifted sums are flushed to FP64 at each change of rotation.
constexpr int DS_DEPTH = 6;   // outputs staged per thread (ring slots)
constexpr int DS_RUN = 8;     // outputs per FP32 partial sum

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
                 "l"(src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait()
{
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Output slices.  A batch's outputs are split into gridDim.y contiguous
// slices, one per blockIdx.y, so that a detector with few stored pixels
// still keeps enough threads in flight.  Slice 0 adds its sums into G_dil
// and Ftot; slice s >= 1 stores its G_dil sums into a scratch plane, and
// its shifted sums into G_dil's rotation-by-rotation totals directly for
// every rotation but its first, whose outputs may continue those of slice
// s - 1: that one goes to a scratch plane too.  Only one slice writes a
// rotation directly, so no two blocks update one value, and
// k_dilute_combine then adds the scratch planes in slice order (the result
// does not depend on timing).
struct DiluteOut {
    double* Gdil;         // [16][npix]
    double2* Ftot;        // [rotation][4][npix] at tstride2 complex values per rotation
    int64_t tstride2;
    double* Gscr;         // [slices - 1][16][npix]
    double2* Fscr;        // [slices - 1][4][npix]
};

__device__ __forceinline__ void dil_put_f(const DiluteOut& D, int slice, int rot, int rot_first, int64_t npix,
                                          int64_t p, int64_t pm, bool mir, int c, double re, double im)
{
    if (slice > 0 && rot == rot_first) {
        double2* t = D.Fscr + ((int64_t)(slice - 1) * 4 + c) * npix;
        t[p] = make_double2(re, im);
        if (mir) t[pm] = make_double2(re, -im);
    } else {
        double2* t = D.Ftot + (int64_t)rot * D.tstride2 + (int64_t)c * npix;
        double2 v = t[p];
        v.x += re;
        v.y += im;
        t[p] = v;
        if (mir) {
            v = t[pm];
            v.x += re;
            v.y -= im;
            t[pm] = v;
        }
    }
}

__device__ __forceinline__ void dil_put_g(const DiluteOut& D, int slice, int64_t npix, int64_t p, int64_t pm,
                                          bool mir, int k, double g)
{
    if (slice > 0) {
        double* t = D.Gscr + ((int64_t)(slice - 1) * 16 + k) * npix;
        t[p] = g;
        if (mir) t[pm] = g_conj_sign(k) * g;
    } else {
        double* t = D.Gdil + (int64_t)k * npix;
        t[p] += g;
        if (mir) t[pm] += g_conj_sign(k) * g;
    }
}

__global__ void k_dilute_combine(DiluteOut D, int n_out, int slices, const int32_t* __restrict__ out_rot, int64_t npix)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    for (int sl = 1; sl < slices; ++sl) {
        const int rot = out_rot[(int64_t)n_out * sl / slices];
#pragma unroll
        for (int k = 0; k < 16; ++k) D.Gdil[(int64_t)k * npix + p] += D.Gscr[((int64_t)(sl - 1) * 16 + k) * npix + p];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const double2 a = D.Fscr[((int64_t)(sl - 1) * 4 + c) * npix + p];
            double2* t = D.Ftot + (int64_t)rot * D.tstride2 + (int64_t)c * npix + p;
            double2 v = *t;
            v.x += a.x;
            v.y += a.y;
            *t = v;
        }
    }
}

__global__ void __launch_bounds__(128, 4)   // 4 blocks per SM: one wave for a 256 x 256 detector
k_dilute_shift_batch(FbView V, int n_out, const float2* __restrict__ eyz, const int32_t* __restrict__ out_rot,
                     DiluteOut D)
{
    __shared__ float4 ring[DS_DEPTH][3][128];   // per slot: channels 0-1, channels 2-3, (e_y, e_z)
    const int64_t npix = (int64_t)V.ny * V.nz;
    const int64_t nst = V.stored_pixels();
    if (nst <= 0 || n_out <= 0) return;
    // threads past the last stored pixel compute on the last one and store
    // nothing, so every lane of a warp takes part in the shuffles below
    const int64_t tid0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = tid0 < nst;
    const int64_t tid = act ? tid0 : nst - 1;
    const int lt = threadIdx.x;
    const int qa = (int)(tid % V.ny), qb = V.zs0 + (int)(tid / V.ny);
    const int64_t p = (int64_t)qa * V.nz + qb;
    // the point mirror -q, written here when it is not stored (conjugates)
    const bool mir = act && V.mirror_unstored(qb);
    const int64_t pm = (int64_t)(V.ny - 1 - qa) * V.nz + (V.nz - 1 - qb);
    const int ne = V.ny + V.nz;
    // this block's slice of the outputs; o below counts within it
    const int slice = blockIdx.y;
    const int o_lo = (int)((int64_t)n_out * slice / gridDim.y);
    n_out = (int)((int64_t)n_out * (slice + 1) / gridDim.y) - o_lo;
    out_rot += o_lo;
    const int rot_first = out_rot[0];
    // 16-byte aligned: channel groups of 4 complex FP32
    const float2* fsrc = V.hi + V.idx(0, qa, qb) + (int64_t)o_lo * V.ostride2;
    const float2* eysrc = eyz + (int64_t)o_lo * ne + qa;
    const float2* ezsrc = eyz + (int64_t)o_lo * ne + V.ny + qb;
    auto stage = [&](int o) {
        if (o < n_out) {
            const int sl = o % DS_DEPTH;
            const float2* f = fsrc + (int64_t)o * V.ostride2;
            cp_async16(&ring[sl][0][lt], f);
            cp_async16(&ring[sl][1][lt], f + 2);
            float2* e = reinterpret_cast<float2*>(&ring[sl][2][lt]);
            cp_async8(e, eysrc + (int64_t)o * ne);
            cp_async8(e + 1, ezsrc + (int64_t)o * ne);
        }
        cp_async_commit();   // one group per output, empty past the end
    };
#pragma unroll
    for (int o = 0; o < DS_DEPTH - 1; ++o) stage(o);

    float gh[16], gl[16], th[8], tl[8], rg[16], rt[8];
#pragma unroll
    for (int k = 0; k < 16; ++k) { gh[k] = 0.f; gl[k] = 0.f; rg[k] = 0.f; }
#pragma unroll
    for (int k = 0; k < 8; ++k) { th[k] = 0.f; tl[k] = 0.f; rt[k] = 0.f; }
    auto fold_t = [&]() {
#pragma unroll
        for (int k = 0; k < 8; ++k) { ts_acc(th[k], tl[k], rt[k]); rt[k] = 0.f; }
    };
    auto flush = [&](int rot) {
        fold_t();
        if (act)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                dil_put_f(D, slice, rot, rot_first, npix, p, pm, mir, c, (double)th[2 * c] + (double)tl[2 * c],
                          (double)th[2 * c + 1] + (double)tl[2 * c + 1]);
#pragma unroll
        for (int k = 0; k < 8; ++k) { th[k] = 0.f; tl[k] = 0.f; }
    };
    // rotation of the outputs, 32 at a time: lane l holds out_rot[o32 + l], and
    // bit l of chg says that output o32 + l starts a new rotation
    const int lane = lt & 31;
    int cur = out_rot[0];
    int rw = 0;
    unsigned chg = 0;
    int run = 0;
    for (int o = 0; o < n_out; ++o) {
        if ((o & 31) == 0) {
            rw = out_rot[min(o + lane, n_out - 1)];
            const int prev = __shfl_up_sync(0xffffffffu, rw, 1);
            chg = __ballot_sync(0xffffffffu, lane == 0 ? rw != cur : rw != prev);
        }
        stage(o + DS_DEPTH - 1);
        cp_async_wait<DS_DEPTH - 1>();   // this thread's copies of output o have landed
        const int sl = o % DS_DEPTH;
        const float4 c01 = ring[sl][0][lt], c23 = ring[sl][1][lt], e = ring[sl][2][lt];
        const float2 f[4] = {make_float2(c01.x, c01.y), make_float2(c01.z, c01.w), make_float2(c23.x, c23.y),
                             make_float2(c23.z, c23.w)};
        if ((chg >> (o & 31)) & 1u) {
            flush(cur);
            cur = __shfl_sync(0xffffffffu, rw, o & 31);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) rg[i] = fmaf(f[i].x, f[i].x, fmaf(f[i].y, f[i].y, rg[i]));
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = i + 1; j < 4; ++j) {
                const int k = pair_idx(i, j);
                rg[4 + 2 * k] = fmaf(f[i].x, f[j].x, fmaf(f[i].y, f[j].y, rg[4 + 2 * k]));
                rg[5 + 2 * k] = fmaf(f[i].y, f[j].x, fmaf(-f[i].x, f[j].y, rg[5 + 2 * k]));
            }
        const float cs = fmaf(e.x, e.z, -e.y * e.w);   // e_y e_z, complex
        const float sn = fmaf(e.y, e.z, e.x * e.w);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            rt[2 * c] = fmaf(f[c].x, cs, fmaf(f[c].y, sn, rt[2 * c]));
            rt[2 * c + 1] = fmaf(f[c].y, cs, fmaf(-f[c].x, sn, rt[2 * c + 1]));
        }
        if (++run == DS_RUN) {
            run = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k) { ts_acc(gh[k], gl[k], rg[k]); rg[k] = 0.f; }
            fold_t();
        }
    }
    cp_async_wait<0>();
    flush(cur);
    if (act)
#pragma unroll
        for (int k = 0; k < 16; ++k)
            dil_put_g(D, slice, npix, p, pm, mir, k, ((double)gh[k] + (double)gl[k]) + (double)rg[k]);
}

// The same pass for detectors whose q_y rows are whole multiples of 128
// pixels and plans of one weight set (4 channels): the 128 pixels of a block
// then share q_z, and their 4 channels of output o are one contiguous 4 KB
// run of F_b.  One thread copies that run into a ring slot with a bulk copy
// (cp.async.bulk, completion counted on the slot's "full" mbarrier), so no
// thread spends load instructions on F; each thread loads its own shift
// factors (L2-resident) two outputs ahead.  Each warp releases a slot on its
// "empty" mbarrier after reading it; the copying thread refills the slot of
// output c with output c + DB_DEPTH once every warp has released c, which it
// checks DB_LAG outputs later so that it does not wait on slower warps.
// Every wait is bounded by limit_ns; on expiry the block sets err, stops, and
// the copying thread waits (bounded) for the copies it has in flight.
constexpr int DB_DEPTH = 10;
constexpr int DB_LAG = 2;
constexpr int DB_SLOT = 128 * 32;   // F bytes per slot

__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__global__ void __launch_bounds__(128, 4)
k_dilute_shift_bulk(FbView V, int n_out, const float2* __restrict__ eyz, const int32_t* __restrict__ out_rot,
                    DiluteOut D, int32_t* err, uint64_t limit_ns)
{
    __shared__ __align__(128) unsigned char ring[DB_DEPTH][DB_SLOT];
    __shared__ __align__(8) uint64_t full[DB_DEPTH], empty[DB_DEPTH];
    __shared__ volatile int abort_flag;
    const int64_t npix = (int64_t)V.ny * V.nz;
    const int lt = threadIdx.x, lane = lt & 31;
    const int64_t t0 = (int64_t)blockIdx.x * 128;   // stored pixels, q_y fastest
    const int qa = (int)(t0 % V.ny) + lt, qb = V.zs0 + (int)(t0 / V.ny);   // one q_z row per block
    const int64_t p = (int64_t)qa * V.nz + qb;
    // the point mirror -q, written here when it is not stored (conjugates)
    const bool mir = V.mirror_unstored(qb);
    const int64_t pm = (int64_t)(V.ny - 1 - qa) * V.nz + (V.nz - 1 - qb);
    const int ne = V.ny + V.nz;
    // this block's slice of the outputs; o below counts within it
    const int slice = blockIdx.y;
    const int o_lo = (int)((int64_t)n_out * slice / gridDim.y);
    n_out = (int)((int64_t)n_out * (slice + 1) / gridDim.y) - o_lo;
    out_rot += o_lo;
    const int rot_first = out_rot[0];
    const float2* fsrc = V.hi + V.idx(0, qa - lt, qb) + (int64_t)o_lo * V.ostride2;
    const float2* eysrc = eyz + (int64_t)o_lo * ne + qa;
    const float2* ezsrc = eyz + (int64_t)o_lo * ne + V.ny + qb;
    if (lt == 0) {
        abort_flag = 0;
        for (int s = 0; s < DB_DEPTH; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 4);
        }
        fence_proxy_async_smem();
    }
    __syncthreads();
    auto issue = [&](int o) {   // thread 0: output o into slot o % DB_DEPTH
        const int sl = o % DB_DEPTH;
        mbar_arrive_expect_tx(&full[sl], DB_SLOT);
        bulk_copy(smem_u32(ring[sl]), fsrc + (int64_t)o * V.ostride2, DB_SLOT, &full[sl]);
    };
    // shift factors (L2-resident) are loaded two outputs ahead into registers
    auto load_e = [&](int o) {
        const int64_t off = (int64_t)min(o, n_out - 1) * ne;
        const float2 y = __ldg(eysrc + off), z = __ldg(ezsrc + off);
        return make_float4(y.x, y.y, z.x, z.y);
    };
    float4 e0 = load_e(0), e1 = load_e(1);
    int issued = 0;   // thread 0: outputs [0, issued) have been copied or are in flight
    if (lt == 0)
        for (; issued < min(DB_DEPTH, n_out); ++issued) issue(issued);

    float gh[16], gl[16], th[8], tl[8], rg[16], rt[8];
#pragma unroll
    for (int k = 0; k < 16; ++k) { gh[k] = 0.f; gl[k] = 0.f; rg[k] = 0.f; }
#pragma unroll
    for (int k = 0; k < 8; ++k) { th[k] = 0.f; tl[k] = 0.f; rt[k] = 0.f; }
    auto fold_t = [&]() {
#pragma unroll
        for (int k = 0; k < 8; ++k) { ts_acc(th[k], tl[k], rt[k]); rt[k] = 0.f; }
    };
    auto flush = [&](int rot) {
        fold_t();
#pragma unroll
        for (int c = 0; c < 4; ++c)
            dil_put_f(D, slice, rot, rot_first, npix, p, pm, mir, c, (double)th[2 * c] + (double)tl[2 * c],
                      (double)th[2 * c + 1] + (double)tl[2 * c + 1]);
#pragma unroll
        for (int k = 0; k < 8; ++k) { th[k] = 0.f; tl[k] = 0.f; }
    };
    int cur = out_rot[0];
    int rw = 0;
    unsigned chg = 0;
    int run = 0;
    int o = 0;
    bool fail = false;
    for (; o < n_out; ++o) {
        if ((o & 31) == 0) {
            rw = out_rot[min(o + lane, n_out - 1)];
            const int prev = __shfl_up_sync(0xffffffffu, rw, 1);
            chg = __ballot_sync(0xffffffffu, lane == 0 ? rw != cur : rw != prev);
        }
        const int sl = o % DB_DEPTH;
        const bool got = mbar_wait(&full[sl], (uint32_t)(o / DB_DEPTH) & 1u, limit_ns, &abort_flag);
        if (!__all_sync(0xffffffffu, got)) {   // a warp leaves the loop as a whole
            fail = true;
            break;
        }
        const unsigned char* slot = ring[sl];
        const float4 c01 = reinterpret_cast<const float4*>(slot)[2 * lt];
        const float4 c23 = reinterpret_cast<const float4*>(slot)[2 * lt + 1];
        const float4 e = e0;
        e0 = e1;
        e1 = load_e(o + 2);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[sl]);
        const float2 f[4] = {make_float2(c01.x, c01.y), make_float2(c01.z, c01.w), make_float2(c23.x, c23.y),
                             make_float2(c23.z, c23.w)};
        if ((chg >> (o & 31)) & 1u) {
            flush(cur);
            cur = __shfl_sync(0xffffffffu, rw, o & 31);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) rg[i] = fmaf(f[i].x, f[i].x, fmaf(f[i].y, f[i].y, rg[i]));
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = i + 1; j < 4; ++j) {
                const int k = pair_idx(i, j);
                rg[4 + 2 * k] = fmaf(f[i].x, f[j].x, fmaf(f[i].y, f[j].y, rg[4 + 2 * k]));
                rg[5 + 2 * k] = fmaf(f[i].y, f[j].x, fmaf(-f[i].x, f[j].y, rg[5 + 2 * k]));
            }
        const float cs = fmaf(e.x, e.z, -e.y * e.w);
        const float sn = fmaf(e.y, e.z, e.x * e.w);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            rt[2 * c] = fmaf(f[c].x, cs, fmaf(f[c].y, sn, rt[2 * c]));
            rt[2 * c + 1] = fmaf(f[c].y, cs, fmaf(-f[c].x, sn, rt[2 * c + 1]));
        }
        if (++run == DS_RUN) {
            run = 0;
#pragma unroll
            for (int k = 0; k < 16; ++k) { ts_acc(gh[k], gl[k], rg[k]); rg[k] = 0.f; }
            fold_t();
        }
        bool stalled = false;
        if (lt == 0) {   // refill the slot of output o - DB_LAG once every warp has released it
            const int c = o - DB_LAG;
            if (c >= 0 && c + DB_DEPTH < n_out) {
                if (mbar_wait(&empty[c % DB_DEPTH], (uint32_t)(c / DB_DEPTH) & 1u, limit_ns, &abort_flag))
                    issue(issued++);
                else
                    stalled = true;
            }
        }
        if (__any_sync(0xffffffffu, stalled)) {
            fail = true;
            ++o;   // output o was read
            break;
        }
    }
    if (fail) {
        abort_flag = 1;
        atomicExch(err, 8);
        if (lt == 0) {   // let this block's copies land before its shared memory is released
            volatile int never = 0;
            for (int x = o; x < issued; ++x)
                mbar_wait(&full[x % DB_DEPTH], (uint32_t)(x / DB_DEPTH) & 1u, 1000000000ull, &never);
        }
        return;
    }
    flush(cur);
#pragma unroll
    for (int k = 0; k < 16; ++k) dil_put_g(D, slice, npix, p, pm, mir, k, ((double)gh[k] + (double)gl[k]) + (double)rg[k]);
}

// Output slices of one dilute pass: as many as keep every block resident
// at once (four per SM; a second, partial wave would double the pass), at
// most 8 (the scratch planes are sized by this count).
int dilute_slices(int64_t stored_pixels)
{
    const int64_t bx = std::max<int64_t>(1, (stored_pixels + 127) / 128);
    const int64_t fit = 4 * (int64_t)device_sm_count() / bx;
    return (int)std::max<int64_t>(1, std::min<int64_t>(8, fit));
}

// scratch: (dilute_slices(V.stored_pixels()) - 1) x 24 x npix doubles, or
// null when that count is 1
cudaError_t launch_dilute_shift_batch(const FbView& V, int n_out, const float2* eyz, const int32_t* out_rot,
                                      double* Gdil, double* Ftot, int64_t tstride, double* scratch, int32_t* err,
                                      uint64_t limit_ns, cudaStream_t s)
{
    if (n_out <= 0) return cudaSuccess;
    const int64_t npix = (int64_t)V.ny * V.nz;
    const int64_t nst = V.stored_pixels();
    const int max_slices = scratch ? dilute_slices(nst) : 1;
    const int slices = std::min(max_slices, n_out);
    DiluteOut D;
    D.Gdil = Gdil;
    D.Ftot = reinterpret_cast<double2*>(Ftot);
    D.tstride2 = tstride / 2;
    D.Gscr = scratch;
    D.Fscr = scratch ? reinterpret_cast<double2*>(scratch + (int64_t)(max_slices - 1) * 16 * npix) : nullptr;
    const bool bulk = V.nch == 4 && V.ny % 128 == 0 && (reinterpret_cast<uintptr_t>(V.hi) & 15) == 0;
    if (bulk)
        k_dilute_shift_bulk<<<dim3((unsigned)(nst / 128), (unsigned)slices), 128, 0, s>>>(V, n_out, eyz, out_rot, D,
                                                                                          err, limit_ns);
    else
        k_dilute_shift_batch<<<dim3((unsigned)((nst + 127) / 128), (unsigned)slices), 128, 0, s>>>(V, n_out, eyz,
                                                                                                  out_rot, D);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || slices == 1) return e;
    k_dilute_combine<<<(unsigned)((npix + 255) / 256), 256, 0, s>>>(D, n_out, slices, out_rot, npix);
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
__global__ void k_obj_bin(FbView V, int n_out, const int32_t* __restrict__ out_obj,
                          const double* __restrict__ hy, const double* __restrict__ hz,
                          const int32_t* __restrict__ bin_of, int64_t npix, int nbins, int id, float s, float b,
                          float Px, float Py, float Pz, double* __restrict__ Iobj)
{
    extern __shared__ float s_bins[];
    const int o = blockIdx.y;
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) s_bins[k] = 0.f;
    __syncthreads();
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < npix; t += (int64_t)gridDim.x * blockDim.x) {
        // q_y fastest: a warp reads contiguous channel rows of F_b
        const int qa = (int)(t % V.ny), qb = (int)(t / V.ny);
        const int64_t p = (int64_t)qa * V.nz + qb;
        const int bin = bin_of[p];
        if (bin < 0) continue;
        float2 f[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) f[c] = V.load(o, qa, qb, c);
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

cudaError_t launch_obj_bin(const FbView& F, int n_out, const int32_t* out_obj, const Plan& p, const int32_t* bin_of,
                           int nbins, int id, double* Iobj, cudaStream_t s)
{
    if (n_out <= 0) return cudaSuccess;
    const int64_t pix_blocks = std::min<int64_t>((p.npix + 1023) / 1024, 64);
    dim3 grid((unsigned)pix_blocks, (unsigned)n_out);
    k_obj_bin<<<grid, 256, nbins * sizeof(float), s>>>(F, n_out, out_obj, p.d_hy,
                                                       p.d_hz, bin_of, p.npix, nbins, id, (float)(1.0 / p.V),
                                                       (float)p.bH, (float)p.P[0], (float)p.P[1], (float)p.P[2], Iobj);
    return cudaGetLastError();
}

}  // namespace nms
