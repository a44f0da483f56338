// Hermitian products, Halpern-Johnson projection and the response functions.
//
// Every cross section of the paper is a Hermitian form in the four
// amplitudes F = (F_N, F_Mx, F_My, F_Mz).  The library therefore accumulates
// G = F F^dagger (16 reals per pixel) -- summed over objects for the dilute
// part and over rotations for orientation averages -- and evaluates any
// response from G afterwards, in FP64:
//   Q = qhat x (qhat x F_M) = -Pi F_M,  Pi = I - qhat qhat^T     (Eq. HJdef)
//   Q_a Q_b^* = (Pi G_M Pi)_ab, u = Pi P, P.Q = -u . F_M
//   N  = G_NN / V                                                (Eq. NuclearSANS)
//   M  = b^2 tr(Pi G_M Pi) / V                                   (Eq. MagneticSANS)
//   P  = b^2 u^T G_M u / V                                       (Eq. PSANSdef)
//   NM = -2 b sum_a u_a Re G_{N a} / V                           (Eq. NMdef)
//   CHI = 2 b^2 [P_z Im A_xy - P_y Im A_xz + P_x Im A_yz] / V, A = Pi G_M Pi
//                                                                (Eq. ChiralSANS)
//   and the POLARIS, SANSPOL and unpolarized combinations.
// G layout: [16][npix]; 0..3 = G_aa (a = N, x, y, z); then for the pairs
// (N,x) (N,y) (N,z) (x,y) (x,z) (y,z): Re G_ab, Im G_ab with G_ab = F_a F_b^*.
#include <cuda_runtime.h>

#include "nms_internal.h"

namespace nms {

__device__ __forceinline__ int pair_index(int a, int b)  // a < b, channels 0..3
{
    // (0,1)=0 (0,2)=1 (0,3)=2 (1,2)=3 (1,3)=4 (2,3)=5
    return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}

__global__ void k_gacc(const double2* __restrict__ F, int64_t npix, double* __restrict__ G)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    double2 f[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) f[c] = F[(int64_t)c * npix + p];
#pragma unroll
    for (int a = 0; a < 4; ++a) G[(int64_t)a * npix + p] += f[a].x * f[a].x + f[a].y * f[a].y;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a + 1; b < 4; ++b) {
            // F_a F_b^* = (ar + i ai)(br - i bi)
            double re = f[a].x * f[b].x + f[a].y * f[b].y;
            double im = f[a].y * f[b].x - f[a].x * f[b].y;
            int k = pair_index(a, b);
            G[(int64_t)(4 + 2 * k) * npix + p] += re;
            G[(int64_t)(5 + 2 * k) * npix + p] += im;
        }
}

cudaError_t launch_gacc(const Plan& p, const double* F, double* G, cudaStream_t s)
{
    k_gacc<<<(unsigned)((p.npix + 255) / 256), 256, 0, s>>>(reinterpret_cast<const double2*>(F), p.npix, G);
    return cudaGetLastError();
}

// Ftot += Fk exp(-i (q_y cy + q_z cz)): object k moved to its rotated centre.
__global__ void k_shift_add(const double2* __restrict__ Fk, const double* __restrict__ qy,
                            const double* __restrict__ qz, double cy, double cz, int64_t npix,
                            double2* __restrict__ Ftot)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    double ph = qy[p] * cy + qz[p] * cz;
    double sn, cs;
    sincos(ph, &sn, &cs);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        double2 f = Fk[(int64_t)c * npix + p];
        double2 t = Ftot[(int64_t)c * npix + p];
        // (fr + i fi)(cs - i sn)
        t.x += f.x * cs + f.y * sn;
        t.y += f.y * cs - f.x * sn;
        Ftot[(int64_t)c * npix + p] = t;
    }
}

cudaError_t launch_shift_add(const Plan& p, const double* Fk, double cy, double cz, double* Ftot, cudaStream_t s)
{
    k_shift_add<<<(unsigned)((p.npix + 255) / 256), 256, 0, s>>>(reinterpret_cast<const double2*>(Fk), p.d_qy,
                                                                 p.d_qz, cy, cz, p.npix,
                                                                 reinterpret_cast<double2*>(Ftot));
    return cudaGetLastError();
}

struct RespConst {
    double s, b, P[3];
};

__device__ __forceinline__ void load_G(const double* __restrict__ G, int64_t npix, int64_t p, double g[16])
{
#pragma unroll
    for (int k = 0; k < 16; ++k) g[k] = G[(int64_t)k * npix + p];
}

// complex G_ab (a, b in 0..3) from the packed 16 reals
__device__ __forceinline__ void gab(const double g[16], int a, int b, double& re, double& im)
{
    if (a == b) { re = g[a]; im = 0.0; return; }
    if (a < b) {
        int k = pair_index(a, b);
        re = g[4 + 2 * k]; im = g[5 + 2 * k];
    } else {
        int k = pair_index(b, a);
        re = g[4 + 2 * k]; im = -g[5 + 2 * k];
    }
}

__global__ void k_response(int id, const double* __restrict__ Ga, const double* __restrict__ Gb, double norm,
                           const double* __restrict__ hy, const double* __restrict__ hz, int64_t npix,
                           RespConst rc, double* __restrict__ out)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    double g[16];
    load_G(Ga, npix, p, g);
    if (Gb) {
        // INTERFERENCE = TOTAL - DILUTE is linear in G
#pragma unroll
        for (int k = 0; k < 16; ++k) g[k] -= Gb[(int64_t)k * npix + p];
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) g[k] *= norm;
    const double y = hy[p], z = hz[p];
    // Pi = I - qhat qhat^T, qhat = (0, y, z)
    const double Pi[3][3] = {{1.0, 0.0, 0.0}, {0.0, 1.0 - y * y, -y * z}, {0.0, -y * z, 1.0 - z * z}};
    double Gr[3][3], Gi[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) gab(g, a + 1, b + 1, Gr[a][b], Gi[a][b]);
    // A = Pi G_M Pi (real and imaginary parts separately; Pi is real symmetric)
    double Tr[3][3], Ti[3][3], Ar[3][3], Ai[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double sr = 0.0, si = 0.0;
            for (int k = 0; k < 3; ++k) { sr += Pi[a][k] * Gr[k][b]; si += Pi[a][k] * Gi[k][b]; }
            Tr[a][b] = sr; Ti[a][b] = si;
        }
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double sr = 0.0, si = 0.0;
            for (int k = 0; k < 3; ++k) { sr += Tr[a][k] * Pi[k][b]; si += Ti[a][k] * Pi[k][b]; }
            Ar[a][b] = sr; Ai[a][b] = si;
        }
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = Pi[a][0] * rc.P[0] + Pi[a][1] * rc.P[1] + Pi[a][2] * rc.P[2];
    const double s = rc.s, b = rc.b, b2 = rc.b * rc.b;
    double vN = s * g[0];
    double vM = s * b2 * (Ar[0][0] + Ar[1][1] + Ar[2][2]);
    double uGu = 0.0;
    for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) uGu += u[a] * u[c] * Gr[a][c];
    double vP = s * b2 * uGu;
    double nm = 0.0;
    for (int a = 0; a < 3; ++a) {
        double re, im;
        gab(g, 0, a + 1, re, im);
        nm += u[a] * re;
    }
    double vNM = -2.0 * s * b * nm;
    double vCHI = 2.0 * s * b2 * (rc.P[2] * Ai[0][1] - rc.P[1] * Ai[0][2] + rc.P[0] * Ai[1][2]);
    double vSF = vM - vP;
    double r = 0.0;
    switch (id) {
        case NMS_RESP_N: r = vN; break;
        case NMS_RESP_M: r = vM; break;
        case NMS_RESP_P: r = vP; break;
        case NMS_RESP_NM: r = vNM; break;
        case NMS_RESP_CHI: r = vCHI; break;
        case NMS_RESP_SF: r = vSF; break;
        case NMS_RESP_PM: r = vSF + vCHI; break;
        case NMS_RESP_MP: r = vSF - vCHI; break;
        case NMS_RESP_PP: r = vN + vNM + vP; break;
        case NMS_RESP_MM: r = vN - vNM + vP; break;
        case NMS_RESP_SANSPOL_P: r = (vN + vNM + vP) + (vSF + vCHI); break;
        case NMS_RESP_SANSPOL_M: r = (vN - vNM + vP) + (vSF - vCHI); break;
        case NMS_RESP_UNPOL: r = vN + vM; break;
        case NMS_RESP_QX2: r = s * Ar[0][0]; break;
        case NMS_RESP_QY2: r = s * Ar[1][1]; break;
        case NMS_RESP_QZ2: r = s * Ar[2][2]; break;
        default: {
            int k = id - NMS_RESP_G_XX_RE;       // 0..17: (a, b, re/im)
            int a = k / 6, bb = (k / 2) % 3;
            double re, im;
            gab(g, a + 1, bb + 1, re, im);
            r = s * ((k & 1) ? im : re);
        }
    }
    out[p] = r;
}

cudaError_t launch_response(const Plan& p, int id, const double* Ga, const double* Gb, double norm, double* out,
                            cudaStream_t s)
{
    RespConst rc;
    rc.s = 1.0 / p.V;
    rc.b = p.bH;
    rc.P[0] = p.P[0]; rc.P[1] = p.P[1]; rc.P[2] = p.P[2];
    k_response<<<(unsigned)((p.npix + 127) / 128), 128, 0, s>>>(id, Ga, Gb, norm, p.d_hy, p.d_hz, p.npix, rc, out);
    return cudaGetLastError();
}

}  // namespace nms
