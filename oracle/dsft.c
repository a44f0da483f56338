/*
 * FP64 CPU oracle: the discrete Fourier sums of the nuclear density and the
 * magnetization, written out as their definition.  TEST INFRASTRUCTURE ONLY:
 * tests, the package's smoke check and the benchmark's CPU-baseline leg may
 * call this; the library never does.
 *
 * Paper, Sec. "Summation approach" (DSFT of n_j and m_j), with the detector
 * geometry q = (0, q_y, q_z) of Sec. "Basic SANS cross sections and
 * conventions" (Eq. qdef):
 *
 *   F_c(q) = sum_j w_cj exp(-i (q_y Y_j + q_z Z_j)),   c in {N, Mx, My, Mz}
 *
 * split into cos and sin as in the paper's real/imaginary sums:
 *   Re F_c = + sum_j w_cj cos(Psi_j),  Im F_c = - sum_j w_cj sin(Psi_j),
 *   Psi_j = q_y Y_j + q_z Z_j   (the phase function of Sec. "Real-space input
 *   data", evaluated at q_y = q sin(theta), q_z = q cos(theta)).
 *
 * No normalisation factor is applied (the caller owns scaling).  Plain FP64
 * recursive summation in index order j = 0..n-1; libm sin/cos.  OpenMP over
 * the q points only.
 */
#include <math.h>
#include <stdint.h>
#ifdef _OPENMP
#include <omp.h>
#endif

void oracle_dsft(int64_t n_cells, const double* Y, const double* Z,
                 const double* w,                      /* [4][n_cells] */
                 int64_t n_q, const double* qy, const double* qz,
                 double* F_re, double* F_im)           /* [4][n_q] each */
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n_q; ++i) {
        double re[4] = {0.0, 0.0, 0.0, 0.0};
        double im[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t j = 0; j < n_cells; ++j) {
            double psi = qy[i] * Y[j] + qz[i] * Z[j];
            double c = cos(psi);
            double s = sin(psi);
            for (int ch = 0; ch < 4; ++ch) {
                double wj = w[(int64_t)ch * n_cells + j];
                re[ch] += wj * c;
                im[ch] -= wj * s;
            }
        }
        for (int ch = 0; ch < 4; ++ch) {
            F_re[(int64_t)ch * n_q + i] = re[ch];
            F_im[(int64_t)ch * n_q + i] = im[ch];
        }
    }
}

/* Number of OpenMP threads the oracle uses (reported with CPU timings). */
int oracle_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
