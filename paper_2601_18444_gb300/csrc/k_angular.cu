// Angular spectrum of a 2D cross section (paper, Eq. CosineSinceIntensities),
// its modal amplitudes (Eq. ModalAmplitudes), and the 2D correlation
// function (Eq. crav2d).
//
// The modal intensities are HBM-bound reductions of the detector image: each
// pixel is read once.  On the polar grid a block owns one q row, keeps the row
// and a table of cos/sin(2 pi m / n_theta) in shared memory, and one warp per
// harmonic k sums f_j T[(k j) mod n_theta] (the periodic trapezoid).  On ring
// bins the pixels are counting-sorted by bin and one block per bin sums
// f cos(k theta), f sin(k theta) (angle-addition recurrence from
// qhat = (0, sin theta, cos theta)) in registers.
//
// The 2D correlation is a dense sum over pixels for every output point
// rho_vec = rho (0, sin alpha, cos alpha):
//   C(rho, alpha) = sum_p W_p f_p exp(+i q_p . rho_vec),
// with W_p the trapezoid weights of the grid (q dq dtheta on the polar grid,
// dq_y dq_z on the Cartesian grid).  It is bound by the FP32 pipes like the
// direct Fourier sum and uses the same numerics: the phase in turns as a
// two-float product with exact reduction, sincospif, FP32 partials over
// groups of 8 pixels folded into two-float sums, K split over blocks.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <vector>

#include "nms_internal.h"

namespace nms {

// ------------------------------------------------------------ polar grid
constexpr int ANG_THREADS = 256;
constexpr size_t ANG_POLAR_MAX_SMEM = 200u << 10;   // row + cos/sin tables: n_theta <= 8533

// Ic/Is[k][i] = (2 - delta_k0)/n_theta * sum_j f(q_i, theta_j) {cos, sin}(k theta_j)
__global__ void __launch_bounds__(ANG_THREADS)
k_angspec_polar(const double* __restrict__ img, int n_q, int n_theta, int kmax, double* __restrict__ Ic,
                double* __restrict__ Is)
{
    extern __shared__ double s_ang[];
    double* row = s_ang;                 // [n_theta]
    double* tc = s_ang + n_theta;        // cos(2 pi m / n_theta)
    double* ts = s_ang + 2 * n_theta;    // sin(2 pi m / n_theta)
    const int i = blockIdx.x;
    for (int j = threadIdx.x; j < n_theta; j += blockDim.x) {
        row[j] = img[(int64_t)i * n_theta + j];
        double sn, cs;
        sincospi(2.0 * (double)j / (double)n_theta, &sn, &cs);
        tc[j] = cs;
        ts[j] = sn;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int k = warp; k <= kmax; k += blockDim.x >> 5) {
        double c = 0.0, s = 0.0;
        for (int j = lane; j < n_theta; j += 32) {
            const int m = (int)(((int64_t)k * j) % n_theta);
            c = fma(row[j], tc[m], c);
            s = fma(row[j], ts[m], s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c += __shfl_xor_sync(0xffffffffu, c, o);
            s += __shfl_xor_sync(0xffffffffu, s, o);
        }
        if (lane == 0) {
            const double pref = (k == 0 ? 1.0 : 2.0) / (double)n_theta;
            Ic[(int64_t)k * n_q + i] = pref * c;
            Is[(int64_t)k * n_q + i] = pref * s;
        }
    }
}

cudaError_t launch_angspec_polar(const Plan& p, const double* img, int kmax, double* Ic, double* Is, cudaStream_t s)
{
    const int n_theta = p.grid.n1;
    const size_t smem = (size_t)3 * n_theta * sizeof(double);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_angspec_polar, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)ANG_POLAR_MAX_SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (smem > ANG_POLAR_MAX_SMEM) return cudaErrorInvalidValue;
    k_angspec_polar<<<p.grid.n0, ANG_THREADS, smem, s>>>(img, p.grid.n0, n_theta, kmax, Ic, Is);
    return cudaGetLastError();
}

// ------------------------------------------------------------ ring bins
// The pixels are counting-sorted by ring bin (bin of every pixel, bin sizes,
// offsets, scatter).  Each bin is cut into parts of at most ANG_PART pixels;
// one block per part sums f cos(k theta) and f sin(k theta) for a chunk of
// harmonics in registers and writes the part's sums, and a last pass adds
// the parts of each bin in order: no atomics on the sums, the same result
// for any pixel order within a part's block reduction.
constexpr int ANG_KC = 16;          // harmonics per register chunk
constexpr int ANG_RED_THREADS = 128;
constexpr int ANG_PART = 256;       // pixels per part

__global__ void k_ang_bins(const double* __restrict__ qa, int64_t npix, const double* __restrict__ edges, int nbins,
                           int32_t* __restrict__ bin_of, int32_t* __restrict__ count)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const int b = find_bin(edges, nbins, qa[p]);
        bin_of[p] = b;
        if (b >= 0) atomicAdd(&count[b], 1);
    }
}

// exclusive prefixes (one block): start[b] of the pixels, cursor[b] = start[b],
// pstart[b] of the parts (pstart[nbins] = number of parts)
__global__ void k_ang_offsets(const int32_t* __restrict__ count, int nbins, int32_t* __restrict__ start,
                              int32_t* __restrict__ cursor, int32_t* __restrict__ pstart)
{
    __shared__ int32_t s_pix[1024];
    __shared__ int32_t s_prt[1024];
    const int per = (nbins + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per, b1 = min(nbins, b0 + per);
    int32_t sp = 0, sq = 0;
    for (int b = b0; b < b1; ++b) {
        sp += count[b];
        sq += (count[b] + ANG_PART - 1) / ANG_PART;
    }
    s_pix[threadIdx.x] = sp;
    s_prt[threadIdx.x] = sq;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t rp = 0, rq = 0;
        for (int t = 0; t < (int)blockDim.x; ++t) {
            const int32_t vp = s_pix[t], vq = s_prt[t];
            s_pix[t] = rp;
            s_prt[t] = rq;
            rp += vp;
            rq += vq;
        }
        pstart[nbins] = rq;
    }
    __syncthreads();
    int32_t rp = s_pix[threadIdx.x], rq = s_prt[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        start[b] = rp;
        cursor[b] = rp;
        pstart[b] = rq;
        rp += count[b];
        rq += (count[b] + ANG_PART - 1) / ANG_PART;
    }
}

__global__ void k_ang_scatter(const int32_t* __restrict__ bin_of, int64_t npix, int32_t* __restrict__ cursor,
                              int32_t* __restrict__ perm)
{
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
        const int b = bin_of[p];
        if (b >= 0) perm[atomicAdd(&cursor[b], 1)] = (int32_t)p;
    }
}

// one block per part: psum[part][r], r < K cos sums, K <= r < 2K sin sums,
// r = 2K the |q| sum
__global__ void __launch_bounds__(ANG_RED_THREADS)
k_ang_parts(const double* __restrict__ img, const double* __restrict__ hy, const double* __restrict__ hz,
            const double* __restrict__ qa, const int32_t* __restrict__ perm, const int32_t* __restrict__ start,
            const int32_t* __restrict__ count, const int32_t* __restrict__ pstart, int nbins, int kmax,
            double* __restrict__ psum)
{
    __shared__ double s_red[2 * ANG_KC + 1][ANG_RED_THREADS / 32];
    const int part = blockIdx.x;
    if (part >= pstart[nbins]) return;
    // bin of this part: last b with pstart[b] <= part
    int lo = 0, hi = nbins;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pstart[mid] <= part) lo = mid;
        else hi = mid;
    }
    const int b = lo;
    const int i0 = (part - pstart[b]) * ANG_PART;
    const int n = min(ANG_PART, count[b] - i0);
    const int32_t* idx = perm + start[b] + i0;
    const int K = kmax + 1;
    const int R = 2 * K + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nw = ANG_RED_THREADS / 32;
    for (int k0 = 0; k0 < K; k0 += ANG_KC) {
        double ac[ANG_KC], as[ANG_KC], aq = 0.0;
#pragma unroll
        for (int u = 0; u < ANG_KC; ++u) { ac[u] = 0.0; as[u] = 0.0; }
        for (int i = threadIdx.x; i < n; i += ANG_RED_THREADS) {
            const int p = idx[i];
            const double f = img[p];
            const double c1 = hz[p], s1 = hy[p];   // cos(theta), sin(theta)
            // (cos, sin)(k0 theta) by binary powering of exp(i theta)
            double ck = 1.0, sk = 0.0, bc = c1, bs = s1;
            for (int e = k0; e; e >>= 1) {
                if (e & 1) {
                    const double t = ck * bc - sk * bs;
                    sk = sk * bc + ck * bs;
                    ck = t;
                }
                const double t = bc * bc - bs * bs;
                bs = 2.0 * bc * bs;
                bc = t;
            }
            const int nk = min(ANG_KC, K - k0);
#pragma unroll
            for (int u = 0; u < ANG_KC; ++u) {
                if (u < nk) {
                    ac[u] = fma(f, ck, ac[u]);
                    as[u] = fma(f, sk, as[u]);
                    const double t = ck * c1 - sk * s1;
                    sk = sk * c1 + ck * s1;
                    ck = t;
                }
            }
            if (k0 == 0) aq += qa[p];
        }
#pragma unroll
        for (int u = 0; u < ANG_KC; ++u) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                ac[u] += __shfl_xor_sync(0xffffffffu, ac[u], o);
                as[u] += __shfl_xor_sync(0xffffffffu, as[u], o);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) aq += __shfl_xor_sync(0xffffffffu, aq, o);
        __syncthreads();
        if (lane == 0) {
#pragma unroll
            for (int u = 0; u < ANG_KC; ++u) {
                s_red[u][warp] = ac[u];
                s_red[ANG_KC + u][warp] = as[u];
            }
            s_red[2 * ANG_KC][warp] = aq;
        }
        __syncthreads();
        if (threadIdx.x < 2 * ANG_KC + 1) {
            double v = 0.0;
            for (int w = 0; w < nw; ++w) v += s_red[threadIdx.x][w];
            const int r = threadIdx.x;
            double* out = psum + (int64_t)part * R;
            if (r < 2 * ANG_KC) {
                const int k = k0 + (r % ANG_KC);
                if (k < K) out[r < ANG_KC ? k : K + k] = v;
            } else if (k0 == 0) {
                out[2 * K] = v;
            }
        }
    }
}

// Ic/Is[k][b] = (2 - delta_k0) * (sum of the bin's parts, in order) / count;
// counts, qmean; NaN for empty bins
__global__ void k_ang_finish(const double* __restrict__ psum, const int32_t* __restrict__ count,
                             const int32_t* __restrict__ pstart, int nbins, int kmax, double* __restrict__ Ic,
                             double* __restrict__ Is, int64_t* __restrict__ counts, double* __restrict__ qmean)
{
    const int K = kmax + 1;
    const int R = 2 * K + 1;
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)R * nbins) return;
    const int r = (int)(t / nbins), b = (int)(t % nbins);
    const int n = count[b];
    double v = 0.0;
    for (int q = pstart[b]; q < pstart[b + 1]; ++q) v += psum[(int64_t)q * R + r];
    if (r < 2 * K) {
        const int k = r < K ? r : r - K;
        const double out = n ? (k == 0 ? 1.0 : 2.0) * v / (double)n : nan("");
        if (r < K) Ic[(int64_t)k * nbins + b] = out;
        else Is[(int64_t)k * nbins + b] = out;
    } else {
        counts[b] = n;
        qmean[b] = n ? v / (double)n : nan("");
    }
}

static int64_t ang_max_parts(int64_t npix, int nbins) { return (npix + ANG_PART - 1) / ANG_PART + nbins; }

cudaError_t launch_angspec_rings(const Plan& p, const double* img, const double* d_edges, int nbins, int kmax,
                                 void* work, double* Ic, double* Is, int64_t* counts, double* qmean, cudaStream_t s)
{
    // work: part sums [max parts][2K+1] (FP64), then bin_of, perm [npix],
    // count, start, cursor [nbins], pstart [nbins+1] (int32)
    const int K = kmax + 1;
    const int64_t mp = ang_max_parts(p.npix, nbins);
    double* psum = (double*)work;
    int32_t* bin_of = (int32_t*)(psum + mp * (2 * K + 1));
    int32_t* perm = bin_of + p.npix;
    int32_t* count = perm + p.npix;
    int32_t* start = count + nbins;
    int32_t* cursor = start + nbins;
    int32_t* pstart = cursor + nbins;
    cudaError_t e = cudaMemsetAsync(count, 0, (size_t)nbins * sizeof(int32_t), s);
    if (e != cudaSuccess) return e;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((p.npix + 255) / 256, 8 * device_sm_count()));
    k_ang_bins<<<blocks, 256, 0, s>>>(p.d_qa, p.npix, d_edges, nbins, bin_of, count);
    k_ang_offsets<<<1, 1024, 0, s>>>(count, nbins, start, cursor, pstart);
    k_ang_scatter<<<blocks, 256, 0, s>>>(bin_of, p.npix, cursor, perm);
    k_ang_parts<<<(unsigned)mp, ANG_RED_THREADS, 0, s>>>(img, p.d_hy, p.d_hz, p.d_qa, perm, start, count, pstart,
                                                        nbins, kmax, psum);
    const int64_t nf = (int64_t)(2 * K + 1) * nbins;
    k_ang_finish<<<(unsigned)((nf + 255) / 256), 256, 0, s>>>(psum, count, pstart, nbins, kmax, Ic, Is, counts, qmean);
    return cudaGetLastError();
}

size_t angspec_rings_work_bytes(int64_t npix, int nbins, int kmax)
{
    const int64_t mp = ang_max_parts(npix, nbins);
    return (size_t)mp * (2 * (kmax + 1) + 1) * sizeof(double) + (size_t)(2 * npix + 4 * (int64_t)nbins + 1) * 4;
}

// ------------------------------------------------------------ modal amplitudes
// a_k = sum over finite nodes of I_k; A_k = a_k / sum_j sqrt(a_j^s^2 + a_j^c^2)
__global__ void k_modal_amplitudes(const double* __restrict__ Ic, const double* __restrict__ Is, int nb, int kmax,
                                   double* __restrict__ Ac, double* __restrict__ As)
{
    extern __shared__ double s_mod[];
    const int K = kmax + 1;
    double* ac = s_mod;
    double* as = s_mod + K;
    double* nrm = s_mod + 2 * K;
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        double c = 0.0, s = 0.0;
        for (int b = 0; b < nb; ++b) {
            const double x = Ic[(int64_t)k * nb + b], y = Is[(int64_t)k * nb + b];
            if (isfinite(x)) c += x;
            if (isfinite(y)) s += y;
        }
        ac[k] = c;
        as[k] = s;
        nrm[k] = sqrt(c * c + s * s);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double d = 0.0;
        for (int k = 0; k < K; ++k) d += nrm[k];
        nrm[K] = d;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += blockDim.x) {
        Ac[k] = ac[k] / nrm[K];
        As[k] = as[k] / nrm[K];
    }
}

cudaError_t launch_modal_amplitudes(const double* Ic, const double* Is, int nb, int kmax, double* Ac, double* As,
                                    cudaStream_t s)
{
    const size_t smem = (size_t)(3 * (kmax + 1) + 1) * sizeof(double);
    k_modal_amplitudes<<<1, 256, smem, s>>>(Ic, Is, nb, kmax, Ac, As);
    return cudaGetLastError();
}

// ------------------------------------------------------------ 2D correlation
constexpr int C2_THREADS = 256;
constexpr int C2_OPT = 2;          // output points per thread
constexpr int C2_TILE = 1024;      // pixels per shared-memory tile
constexpr int C2_GROUP = 8;        // pixels per FP32 partial before the two-float fold

// per pixel: (qy/2pi, qz/2pi) as two-float (from the plan) and the weight W_p f_p
__device__ __forceinline__ double trap_weight(int i, int n, double lo, double hi)
{
    if (n < 2) return 0.0;
    const double h = (hi - lo) / (double)(n - 1);
    return (i == 0 || i == n - 1) ? 0.5 * h : h;
}

__global__ void k_corr2d_weights(const double* __restrict__ img, int kind, int n0, int n1, double lo0, double hi0,
                                 double lo1, double hi1, float* __restrict__ w, double* __restrict__ wabs)
{
    const int64_t npix = (int64_t)n0 * n1;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (p < npix) {
        const int a = (int)(p / n1), b = (int)(p % n1);
        double W;
        if (kind == NMS_QGRID_POLAR) {
            const double q = n0 == 1 ? lo0 : lo0 + ((hi0 - lo0) * a) / (double)(n0 - 1);
            W = trap_weight(a, n0, lo0, hi0) * q * (2.0 * M_PI / (double)n1);
        } else {
            W = trap_weight(a, n0, lo0, hi0) * trap_weight(b, n1, lo1, hi1);
        }
        v = W * img[p];
        w[p] = (float)v;
    }
    // block sum of |W f| (the scale of the result, reported with it)
    __shared__ double red[256];
    red[threadIdx.x] = fabs(v);
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(wabs, red[0]);
}

__device__ __forceinline__ void c2_two_sum(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

// part[split][out] = (re, im) of sum over this split's pixels
__global__ void __launch_bounds__(C2_THREADS)
k_corr2d(const float4* __restrict__ qturn, const float* __restrict__ w, int64_t npix,
         const float4* __restrict__ rho_t, int n_out, double2* __restrict__ part)
{
    __shared__ float4 s_q[C2_TILE];
    __shared__ float s_w[C2_TILE];
    const int splits = gridDim.y;
    const int64_t per = (npix + splits - 1) / splits;
    const int64_t p0 = (int64_t)blockIdx.y * per;
    const int64_t p1 = min(npix, p0 + per);
    int o[C2_OPT];
    float4 r[C2_OPT];
    float hr[C2_OPT], lr[C2_OPT], hi[C2_OPT], li[C2_OPT];
#pragma unroll
    for (int k = 0; k < C2_OPT; ++k) {
        o[k] = blockIdx.x * C2_THREADS * C2_OPT + k * C2_THREADS + threadIdx.x;
        r[k] = o[k] < n_out ? rho_t[o[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
        hr[k] = lr[k] = hi[k] = li[k] = 0.f;
    }
    for (int64_t t0 = p0; t0 < p1; t0 += C2_TILE) {
        const int nt = (int)min((int64_t)C2_TILE, p1 - t0);
        const int ntg = ((nt + C2_GROUP - 1) / C2_GROUP) * C2_GROUP;
        __syncthreads();
        for (int i = threadIdx.x; i < ntg; i += C2_THREADS) {
            s_q[i] = i < nt ? qturn[t0 + i] : make_float4(0.f, 0.f, 0.f, 0.f);
            s_w[i] = i < nt ? w[t0 + i] : 0.f;
        }
        __syncthreads();
        for (int g = 0; g < ntg; g += C2_GROUP) {
            float ar[C2_OPT], ai[C2_OPT];
#pragma unroll
            for (int k = 0; k < C2_OPT; ++k) ar[k] = ai[k] = 0.f;
#pragma unroll 4
            for (int u = 0; u < C2_GROUP; ++u) {
                const float4 q = s_q[g + u];
                const float wv = s_w[g + u];
#pragma unroll
                for (int k = 0; k < C2_OPT; ++k) {
                    // two-float (q_y' rho_y + q_z' rho_z) in turns, exact reduction
                    const float py = q.x * r[k].x;
                    const float ey = fmaf(q.x, r[k].x, -py) + fmaf(q.x, r[k].y, q.y * r[k].x);
                    const float pz = q.z * r[k].z;
                    const float ez = fmaf(q.z, r[k].z, -pz) + fmaf(q.z, r[k].w, q.w * r[k].z);
                    const float sm = py + pz;
                    const float bb = sm - py;
                    const float es = (py - (sm - bb)) + (pz - bb);
                    const float tt = (sm - rintf(sm)) + (es + ey + ez);
                    float sn, cs;
                    sincospif(2.0f * tt, &sn, &cs);
                    ar[k] = fmaf(wv, cs, ar[k]);
                    ai[k] = fmaf(wv, sn, ai[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < C2_OPT; ++k) {
                c2_two_sum(hr[k], lr[k], ar[k]);
                c2_two_sum(hi[k], li[k], ai[k]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < C2_OPT; ++k)
        if (o[k] < n_out)
            part[(int64_t)blockIdx.y * n_out + o[k]] =
                make_double2((double)hr[k] + (double)lr[k], (double)hi[k] + (double)li[k]);
}

__global__ void k_corr2d_reduce(const double2* __restrict__ part, int splits, int n_out, double2* __restrict__ C)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_out) return;
    double re = 0.0, im = 0.0;
    for (int s = 0; s < splits; ++s) {
        const double2 v = part[(int64_t)s * n_out + o];
        re += v.x;
        im += v.y;
    }
    C[o] = make_double2(re, im);
}

// rho_vec = rho (0, sin alpha, cos alpha) as two-float; with q/2 pi per
// pixel the product is the phase in turns
__global__ void k_corr2d_points(const double* __restrict__ rho, int n_rho, const double* __restrict__ alpha,
                                int n_alpha, float4* __restrict__ pts)
{
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_rho * n_alpha) return;
    const double rr = rho[o / n_alpha], al = alpha[o % n_alpha];
    double sa, ca;
    sincos(al, &sa, &ca);
    const double y = rr * sa, z = rr * ca;
    const float yh = (float)y, zh = (float)z;
    pts[o] = make_float4(yh, (float)(y - (double)yh), zh, (float)(z - (double)zh));
}

cudaError_t launch_corr2d(const Plan& p, const double* img, const double* d_rho, int n_rho, const double* d_alpha,
                          int n_alpha, float* d_w, double* d_wabs, float4* d_pts, double2* d_part, int splits,
                          double2* d_C, cudaStream_t s)
{
    const int64_t np = p.npix;
    k_corr2d_weights<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(img, p.grid.kind, p.grid.n0, p.grid.n1, p.grid.lo0,
                                                                  p.grid.hi0, p.grid.lo1, p.grid.hi1, d_w, d_wabs);
    const int n_out = n_rho * n_alpha;
    k_corr2d_points<<<(n_out + 127) / 128, 128, 0, s>>>(d_rho, n_rho, d_alpha, n_alpha, d_pts);
    const int ob = (n_out + C2_THREADS * C2_OPT - 1) / (C2_THREADS * C2_OPT);
    k_corr2d<<<dim3((unsigned)ob, (unsigned)splits), C2_THREADS, 0, s>>>(p.d_qturn, d_w, np, d_pts, n_out, d_part);
    k_corr2d_reduce<<<(n_out + 127) / 128, 128, 0, s>>>(d_part, splits, n_out, d_C);
    return cudaGetLastError();
}

int corr2d_splits(int64_t npix, int n_out)
{
    const int ob = (n_out + C2_THREADS * C2_OPT - 1) / (C2_THREADS * C2_OPT);
    const int want = std::max(1, 4 * device_sm_count() / std::max(1, ob));
    const int64_t cap = std::max<int64_t>(1, npix / (2 * C2_TILE));   // at least two tiles per split
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
}

}  // namespace nms
