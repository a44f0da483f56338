// Azimuthal average on the polar grid (paper, Eq. iqazi) and correlation
// functions (Eqs. crrad, prrad).  Both are small, HBM-bound reductions over
// the detector image; the kernels read each pixel once.  (Ring-binned
// averages on Cartesian and list grids are the k = 0 mode of the angular
// spectrum kernels.)
#include <cuda_runtime.h>
#include <math.h>

#include "nms_internal.h"

namespace nms {

// ------------------------------------------------------------ polar grid
// Periodic trapezoid over theta_j = 2 pi j / n_theta equals the mean over j.
__global__ void k_azimuthal_polar(const double* __restrict__ img, int n0, int n1, double* __restrict__ Iq)
{
    __shared__ double red[256];
    int i = blockIdx.x;
    double acc = 0.0;
    for (int j = threadIdx.x; j < n1; j += blockDim.x) acc += img[(int64_t)i * n1 + j];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) Iq[i] = red[0] / (double)n1;
}

cudaError_t launch_azimuthal_polar(const Plan& p, const double* img, double* Iq, cudaStream_t s)
{
    k_azimuthal_polar<<<p.grid.n0, 256, 0, s>>>(img, p.grid.n0, p.grid.n1, Iq);
    return cudaGetLastError();
}

// Per-pixel q-grid quantities in FP64 (Sec. "Summation approach": the
// detector plane q = (0, q_y, q_z)): q_y, q_z, the unit vector (h_y, h_z) =
// q/|q| (0, 1 at q = 0), |q|, and q/(2 pi) as two-float turns.  Cartesian:
// pixel i = a n1 + b, q_y = node(a; n0, lo0, hi0), q_z = node(b; n1, lo1,
// hi1); polar: |q| = node(a; n0, lo0, hi0), theta = 2 pi b / n1, q_y =
// |q| sin theta, q_z = |q| cos theta, h = (sin, cos); list: (q_y, q_z) pairs.
// node(a; n, lo, hi) = lo + ((hi - lo) a)/(n - 1), without contraction.
__device__ __forceinline__ double grid_node(int64_t a, int64_t n, double lo, double hi)
{
    if (n == 1) return lo;
    return __dadd_rn(lo, __ddiv_rn(__dmul_rn(__dadd_rn(hi, -lo), (double)a), (double)(n - 1)));
}

__global__ void k_grid(int kind, int64_t np, int n0, int n1, double lo0, double hi0, double lo1, double hi1,
                       const double* __restrict__ qlist, double* __restrict__ qy, double* __restrict__ qz,
                       double* __restrict__ hy, double* __restrict__ hz, double* __restrict__ qa,
                       float4* __restrict__ qturn)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const double two_pi = 6.283185307179586;
    double y, z, h1, h2, a;
    if (kind == NMS_QGRID_POLAR) {
        const double qm = grid_node(i / n1, n0, lo0, hi0);
        const double th = __ddiv_rn(__dmul_rn(two_pi, (double)(i % n1)), (double)n1);
        double st, ct;
        sincos(th, &st, &ct);
        y = __dmul_rn(qm, st);
        z = __dmul_rn(qm, ct);
        h1 = st;
        h2 = ct;
        a = qm;
    } else {
        if (kind == NMS_QGRID_CARTESIAN) {
            y = grid_node(i / n1, n0, lo0, hi0);
            z = grid_node(i % n1, n1, lo1, hi1);
        } else {
            y = qlist[2 * i];
            z = qlist[2 * i + 1];
        }
        a = hypot(y, z);
        if (a > 0.0) {
            h1 = __ddiv_rn(y, a);
            h2 = __ddiv_rn(z, a);
        } else {
            h1 = 0.0;
            h2 = 1.0;
        }
    }
    qy[i] = y;
    qz[i] = z;
    hy[i] = h1;
    hz[i] = h2;
    qa[i] = a;
    const double ty = __ddiv_rn(y, two_pi), tz = __ddiv_rn(z, two_pi);
    const float tyh = (float)ty, tzh = (float)tz;
    qturn[i] = make_float4(tyh, (float)(ty - (double)tyh), tzh, (float)(tz - (double)tzh));
}

cudaError_t launch_grid(const nms_qgrid& g, int64_t np, const double* d_qlist, double* qy, double* qz, double* hy,
                        double* hz, double* qa, float4* qturn, cudaStream_t s)
{
    k_grid<<<(unsigned)((np + 255) / 256), 256, 0, s>>>((int)g.kind, np, g.n0, g.n1, g.lo0, g.hi0, g.lo1, g.hi1, d_qlist,
                                                        qy, qz, hy, hz, qa, qturn);
    return cudaGetLastError();
}

// Nodes of the polar grid as bins: counts[i] = n_theta, qmean[i] = q_i
// (linear nodes lo + ((hi - lo) i)/(n - 1), as the grid defines them).
__global__ void k_polar_nodes(int n0, int n1, double lo, double hi, int64_t* __restrict__ counts,
                              double* __restrict__ qmean)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n0) return;
    if (counts) counts[i] = n1;
    if (qmean) qmean[i] = n0 == 1 ? lo : lo + ((hi - lo) * i) / (double)(n0 - 1);
}

cudaError_t launch_polar_nodes(const Plan& p, int64_t* counts, double* qmean, cudaStream_t s)
{
    k_polar_nodes<<<(p.grid.n0 + 127) / 128, 128, 0, s>>>(p.grid.n0, p.grid.n1, p.grid.lo0, p.grid.hi0, counts,
                                                          qmean);
    return cudaGetLastError();
}

// ------------------------------------------------------------ correlation
// Compaction of the finite nodes (one block, order preserving), then one
// block per r_m sums the trapezoids I j0(q r) q^2.
__global__ void k_corr_compact(int nq, const double* __restrict__ q, const double* __restrict__ I,
                               double* __restrict__ qo, double* __restrict__ Io, int* __restrict__ nout)
{
    __shared__ int s_base;
    __shared__ int s_scan[1024];
    if (threadIdx.x == 0) s_base = 0;
    __syncthreads();
    for (int start = 0; start < nq; start += blockDim.x) {
        int i = start + threadIdx.x;
        int ok = (i < nq) && isfinite(q[i]) && isfinite(I[i]);
        s_scan[threadIdx.x] = ok;
        __syncthreads();
        // inclusive Hillis-Steele scan
        for (int off = 1; off < blockDim.x; off <<= 1) {
            int v = (threadIdx.x >= off) ? s_scan[threadIdx.x - off] : 0;
            __syncthreads();
            s_scan[threadIdx.x] += v;
            __syncthreads();
        }
        if (ok) {
            int dst = s_base + s_scan[threadIdx.x] - 1;
            qo[dst] = q[i];
            Io[dst] = I[i];
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_base += s_scan[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *nout = s_base;
}

__device__ __forceinline__ double j0_sph(double x)
{
    return x == 0.0 ? 1.0 : sin(x) / x;
}

__global__ void k_corr(const double* __restrict__ q, const double* __restrict__ I, const int* __restrict__ nvalid,
                       const double* __restrict__ r, double pref, double* __restrict__ c, double* __restrict__ pr)
{
    __shared__ double red[256];
    const int m = blockIdx.x;
    const int n = *nvalid;
    const double rm = r[m];
    double acc = 0.0;
    for (int i = threadIdx.x; i + 1 < n; i += blockDim.x) {
        double q0 = q[i], q1 = q[i + 1];
        double f0 = I[i] * j0_sph(q0 * rm) * q0 * q0;
        double f1 = I[i + 1] * j0_sph(q1 * rm) * q1 * q1;
        acc += 0.5 * (f0 + f1) * (q1 - q0);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double v = pref * red[0];
        if (c) c[m] = v;
        if (pr) pr[m] = rm * rm * v;
    }
}

cudaError_t launch_correlation(int nq, const double* q, const double* Iq, int nr, const double* r, double pref,
                               double* c, double* pr, double* sq, double* sf, int* sn, cudaStream_t s)
{
    k_corr_compact<<<1, 1024, 0, s>>>(nq, q, Iq, sq, sf, sn);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (nr > 0) k_corr<<<nr, 256, 0, s>>>(sq, sf, sn, r, pref, c, pr);
    return cudaGetLastError();
}

}  // namespace nms
