/*
 * nms.h -- C ABI of the GB300 SANS Fourier-sum library (libnms.so).
 *
 * The library evaluates, on one NVIDIA GB300 (sm_103a), the hot path of the
 * NuMagSANS method: the discrete Fourier sums of the nuclear scattering-length
 * density and of the magnetization over every (rotated) cell, on a 2D
 * detector q-grid, the Halpern-Johnson projection, the nuclear, magnetic,
 * interference, polarised and unpolarized cross sections, their azimuthal
 * average and the Fourier-Bessel correlation functions.
 *
 * Conventions used by every entry point:
 *  - Lengths in the caller's unit (nm in the examples), q in the inverse
 *    unit.  The scattering geometry is fixed as in the paper: beam along x,
 *    detector in the y-z plane, q = (0, q_y, q_z), qhat = (0, sin t, cos t).
 *  - Amplitudes are RAW sums F_c(q) = sum_j w_cj exp(-i q.r'_j) with
 *    w_cj = V_j (N_j, M'_xj, M'_yj, M'_zj): the (2 pi)^{-3/2} of the DSFT and
 *    the 8 pi^3 of the cross sections cancel, so every cross section is the
 *    raw quadratic form times 1/V (and b_H, b_H^2 for magnetic terms).
 *  - Row-major arrays.  "host or device" pointers are told apart by the
 *    *_is_device flag next to them; nothing is inferred.
 *  - Status codes only: no exception or abort crosses the ABI.  On failure
 *    nms_last_error() returns a thread-local message.  Failed creates leave
 *    *out == NULL.
 *  - Thread safety: one plan per host thread (a plan owns one CUDA stream).
 *  - Memory: the plan deep-copies its inputs to the device at create time and
 *    owns all device memory it allocates until nms_plan_destroy().  Caller
 *    buffers are never retained after a call returns.
 *  - No CPU fallback: without a usable sm_103a device every call that would
 *    compute returns NMS_ERR_CUDA.
 */
#ifndef NMS_H
#define NMS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nms_plan_s* nms_plan_t;

typedef enum {
    NMS_OK = 0,
    NMS_ERR_INVALID_ARG = 1,   /* a size, pointer, id or option is out of range   */
    NMS_ERR_OUT_OF_MEMORY = 2, /* a device or host allocation failed              */
    NMS_ERR_CUDA = 3,          /* a CUDA call failed (no device, launch failure)  */
    NMS_ERR_UNSUPPORTED = 4,   /* valid request the chosen path cannot serve      */
    NMS_ERR_TIMEOUT = 5,       /* a bounded device wait gave up (kernel returned) */
    NMS_ERR_BAD_STATE = 6      /* call out of order (e.g. response before sums)   */
} nms_status;

/* Detector grids (paper, Sec. "Configuration file" and Eq. qdef).
 *  CARTESIAN: q_y[a] = lo0 + (hi0-lo0) a/(n0-1), a < n0 (n0 == 1 gives lo0),
 *             q_z[b] likewise with (n1, lo1, hi1); pixel p = a*n1 + b.
 *             Separable: served by the tensor-core path.
 *  POLAR:     q_i = lo0 + (hi0-lo0) i/(n0-1), theta_j = 2 pi j/n1,
 *             q_y = q sin theta, q_z = q cos theta; pixel p = i*n1 + j.
 *             This is the paper's (q, theta) grid; served by the direct sum.
 *  LIST:      n0 arbitrary points, qlist[2p] = q_y, qlist[2p+1] = q_z (host).
 *             Served by the direct sum.
 * qhat = q/|q|; where |q| == 0 qhat = e_z (CARTESIAN, LIST) or uses theta_j
 * (POLAR). */
typedef enum { NMS_QGRID_CARTESIAN = 0, NMS_QGRID_POLAR = 1, NMS_QGRID_LIST = 2 } nms_qgrid_kind;

typedef struct {
    int32_t kind;            /* nms_qgrid_kind */
    int32_t n0, n1;          /* CARTESIAN: n_y, n_z; POLAR: n_q, n_theta; LIST: n, ignored */
    double lo0, hi0;         /* CARTESIAN: q_y range; POLAR: |q| range */
    double lo1, hi1;         /* CARTESIAN: q_z range; unused otherwise */
    const double* qlist;     /* LIST only: host [n0][2] */
} nms_qgrid;

/* How the Fourier sums are evaluated. */
typedef enum {
    NMS_PREC_AUTO = 0,          /* TC_F16X3 on CARTESIAN and POLAR grids,
                                   FP32_DIRECT on LIST grids                      */
    NMS_PREC_TC_F16X3 = 1,      /* split-FP16 (hi/lo, 3 products) tcgen05 GEMM, FP32
                                   TMEM accumulation promoted to two-float every
                                   kc_cells cells; CARTESIAN grids, and POLAR grids
                                   as one GEMM per ray (the phase |q| u with u the
                                   cell's projection on the ray splits over two
                                   axes |q| = lo + 64 i1 dq + i2 dq; the ray at
                                   theta + pi is the conjugate; no per-object
                                   averages).  It takes
                                   the place of TF32x3 (same ~2^-22 per-product
                                   error, but TF32 runs at half the FP16 rate on
                                   tcgen05), BF16x3 (2^-17: misses 1e-6) and
                                   BF16x6 (twice the MMAs for no gain over this) */
    NMS_PREC_FP32_DIRECT = 2,   /* compensated FP32 direct sum (two-float phase in
                                   turns, exact reduction, sincospif)                  */
    NMS_PREC_FP32_NAIVE = 3     /* plain FP32 phase + sincosf: fast, inaccurate at
                                   large |q.r|; reported for comparison only           */
} nms_precision;

typedef struct {
    int32_t precision;       /* nms_precision */
    int32_t want_dilute;     /* 1: also accumulate sum_k G_k over objects (form
                                factors without interparticle interference)     */
    double volume_V;         /* scattering volume V of the 1/V prefactor; 0 -> 1 */
    double b_H;              /* magnetic scattering length b_H; 0 -> 1           */
    double P[3];             /* polarisation unit vector; all 0 -> e_z           */
    int32_t kc_cells;        /* tensor path: cells per FP32 TMEM chunk, rounded
                                down to a multiple of 64 (at least 64); 0 -> 192.
                                Larger chunks drain less often and run faster,
                                but the error at fully coherent pixels grows
                                about linearly with the chunk: at most 8.9e-7
                                of sum |w| at 192, 5.2e-7 at 128, 1.1e-6 at 256 */
    int32_t split_k;         /* tensor path: work items per SM of a GEMM launch
                                (how finely the cells of each output are split
                                over CTAs); 0 -> 8, or the autotuned value      */
    int64_t max_spin;        /* bounded device waits: microseconds (%globaltimer)
                                a wait lasts before the kernel gives up with
                                NMS_ERR_TIMEOUT; 0 -> 4,000,000 (4 s)          */
    int64_t workspace_bytes; /* cap on the tensor-path phase-table workspace
                                (cells beyond it are processed in chunks);
                                0 -> min(free / 3, 8 GiB)                      */
    int32_t timing;          /* 1: record CUDA events around each stage (see
                                nms_plan_stage_ms)                               */
    int32_t autotune;        /* tensor path: 1 = time candidate GEMM forms
                                (one CTA per tile, two-SM MMA),
                                kc and work-list granularities on a probe of
                                the cells at plan creation and keep the
                                fastest whose amplitude error (vs the
                                compensated direct sum) is <= 3e-7 of sum|w|;
                                cached per shape and device (file
                                $NMS_AUTOTUNE_CACHE if set)                    */
    int32_t n_sets;          /* weight sets S (loop mode: e.g. one magnetization
                                state per applied field) over the same cells,
                                objects and orientations; nuc and mag then hold
                                S sets ([S][n], [S][n][3]).  0 -> 1.  Tensor
                                path: S <= 32, stacked along the GEMM rows so
                                every q_z table block serves all sets; results
                                per set via nms_select_set.                    */
    int32_t reserved[5];
} nms_options;

/* Fill *opt with the defaults above. */
nms_status nms_options_default(nms_options* opt);

/* Create a plan: validate inputs, copy them to the device (H2D), build the
 * q-grid.  Paper: Sec. "Real-space input data" (cells x^{kl}, objects k with
 * centres r^k, indexing W = sum N_k), Sec. "Configuration file" (rotation
 * R = R_z(beta) R_y(alpha), generalised here to any R), Sec. "Summation
 * approach".
 *   n_cells         W >= 1 total cells.
 *   pos             host [n_cells][3] local cell coordinates x^{kl}.
 *   cell_vol        host [n_cells] cell volumes V_j, or NULL for all 1.
 *   nuc             host [n_cells] nuclear density N_j, or NULL (channel off);
 *                   [S][n_cells] with opt->n_sets = S > 1.
 *   mag             host [n_cells][3] magnetization M_j, or NULL (off);
 *                   [S][n_cells][3] with S weight sets.
 *   n_objects       K >= 1.
 *   object_offsets  host [K+1], 0 = off_0 <= ... <= off_K = n_cells (empty
 *                   objects allowed), or NULL when K == 1.
 *   object_centers  host [K][3] centres r^k, or NULL (all 0: dilute system).
 *   n_rot           >= 1 sample orientations; results are averaged over them.
 *   rot             host [n_rot][9] row-major rotation matrices, or NULL for
 *                   the identity (n_rot must then be 1).  Positions AND
 *                   magnetizations are rotated: r' = R (x + r^k), M' = R M.
 *   grid            detector grid (copied).
 *   opt             options (copied), or NULL for defaults.
 *   cuda_stream     cudaStream_t every launch of this plan goes to (NULL: the
 *                   legacy default stream).
 * Errors: INVALID_ARG (sizes, offsets not monotone, TC precision on a LIST
 * grid), OUT_OF_MEMORY, CUDA. */
nms_status nms_plan_create(nms_plan_t* out, int64_t n_cells, const double* pos,
                           const double* cell_vol, const double* nuc, const double* mag,
                           int64_t n_objects, const int64_t* object_offsets,
                           const double* object_centers, int32_t n_rot, const double* rot,
                           const nms_qgrid* grid, const nms_options* opt, void* cuda_stream);

/* Evaluate the Fourier sums for every rotation and accumulate the Hermitian
 * products G = F F^dagger (16 reals per pixel) that every response is a
 * linear function of: G_total from the full amplitude sum_k F_k e^{-iq.r^k}
 * and, with want_dilute, G_dilute = sum_k F_k F_k^dagger (paper, Sec.
 * "Summation approach": interparticle decomposition).  Both are averaged over
 * the rotations.  Asynchronous on the plan's stream; errors from the device
 * (e.g. TIMEOUT) surface here or at the next synchronising call. */
nms_status nms_amplitudes(nms_plan_t plan);

/* Copy the total amplitudes of the LAST rotation evaluated:
 * out[c][p][2] = (Re, Im) F_c(q_p), c = N, Mx, My, Mz (rotated frame),
 * n_pixels = n0*n1 (n0 for LIST).  out is host or device memory of
 * 8*n_pixels doubles.  Synchronises the plan's stream. */
nms_status nms_get_amplitudes(nms_plan_t plan, double* out, int32_t out_is_device);

/* Response ids (paper, Sec. "SANS observables"):
 *  N   = |F_N|^2 / V                                    Eq. NuclearSANS
 *  M   = b^2 |Q|^2 / V, Q = qhat x (qhat x F_M)          Eqs. MagneticSANS, HJdef
 *  P   = b^2 |P.Q|^2 / V                                 Eq. PSANSdef
 *  NM  = b (F_N (P.Q)^* + F_N^* P.Q) / V                 Eq. NMdef
 *  CHI = -i b^2 P.(Q x Q^*) / V                          Eq. ChiralSANS
 *  SF  = M - P                                           Eq. sfdef
 *  PM, MP = SF +- CHI  (+-, -+)      PP, MM = N +- NM + P  (++, --)
 *  SANSPOL_P = PP + PM,  SANSPOL_M = MM + MP             SANSPOL section
 *  UNPOL = (PP + MM + PM + MP)/2 = N + M                 unpolarized section
 *  G_ab_RE/IM = Re/Im F_Ma F_Mb^* / V (a, b in x, y, z)  Fourier cross spectra
 *  QX2, QY2, QZ2 = |Q_x|^2/V, |Q_y|^2/V, |Q_z|^2/V */
enum {
    NMS_RESP_N = 0, NMS_RESP_M, NMS_RESP_P, NMS_RESP_NM, NMS_RESP_CHI, NMS_RESP_SF,
    NMS_RESP_PM, NMS_RESP_MP, NMS_RESP_PP, NMS_RESP_MM, NMS_RESP_SANSPOL_P,
    NMS_RESP_SANSPOL_M, NMS_RESP_UNPOL,
    NMS_RESP_G_XX_RE, NMS_RESP_G_XX_IM, NMS_RESP_G_XY_RE, NMS_RESP_G_XY_IM,
    NMS_RESP_G_XZ_RE, NMS_RESP_G_XZ_IM, NMS_RESP_G_YX_RE, NMS_RESP_G_YX_IM,
    NMS_RESP_G_YY_RE, NMS_RESP_G_YY_IM, NMS_RESP_G_YZ_RE, NMS_RESP_G_YZ_IM,
    NMS_RESP_G_ZX_RE, NMS_RESP_G_ZX_IM, NMS_RESP_G_ZY_RE, NMS_RESP_G_ZY_IM,
    NMS_RESP_G_ZZ_RE, NMS_RESP_G_ZZ_IM,
    NMS_RESP_QX2, NMS_RESP_QY2, NMS_RESP_QZ2,
    NMS_RESP_COUNT
};

/* Which part of the object decomposition a response is taken from. */
enum { NMS_PART_TOTAL = 0, NMS_PART_DILUTE = 1, NMS_PART_INTERFERENCE = 2 };

/* Evaluate one response on every pixel from the accumulated G (FP64).
 * out: host or device [n_pixels] doubles, layout as the grid.  DILUTE and
 * INTERFERENCE (= TOTAL - DILUTE) need want_dilute.  Errors: INVALID_ARG
 * (id, part), BAD_STATE (no nms_amplitudes yet), UNSUPPORTED (dilute part
 * without want_dilute). */
nms_status nms_response(nms_plan_t plan, int32_t response_id, int32_t part,
                        double* out, int32_t out_is_device);

/* Azimuthal average of a per-pixel image of this plan's grid (paper,
 * Eq. iqazi, trapezoidal rule).
 *  POLAR grid:  nbins must equal n0 and bin_edges may be NULL; Iq[i] is the
 *               mean over theta_j (the periodic trapezoid), counts[i] = n1,
 *               qmean[i] = q_i.
 *  CARTESIAN/LIST: bin b collects pixels with edges[b] <= |q| < edges[b+1]
 *               (bin_edges host [nbins+1], increasing); Iq[b] = their mean,
 *               counts[b] = their number, qmean[b] = their mean |q|; empty
 *               bins give NaN in Iq and qmean.
 * img: [n_pixels] doubles, host or device per img_is_device.  Iq, counts,
 * qmean (qmean may be NULL): host or device per out_is_device.  Synchronous. */
nms_status nms_azimuthal_average(nms_plan_t plan, const double* img, int32_t img_is_device,
                                 int32_t nbins, const double* bin_edges,
                                 double* Iq, int64_t* counts, double* qmean,
                                 int32_t out_is_device);

/* Angular spectrum of a per-pixel image of this plan's grid (paper, Eq.
 * CosineSinceIntensities, trapezoidal rule) and its modal amplitudes (Eq.
 * ModalAmplitudes).
 *  POLAR grid:  nbins must equal n0 (bin_edges may be NULL) and n1 <= 8533;
 *               Ic[k][i] = (2 - delta_k0)/n1 sum_j f(q_i, theta_j) cos(k theta_j),
 *               Is likewise with sin (the periodic trapezoid); counts[i] = n1,
 *               qmean[i] = q_i.
 *  CARTESIAN/LIST: ring bins as in nms_azimuthal_average; Ic[k][b] =
 *               (2 - delta_k0) x the mean over the bin's pixels of
 *               f cos(k theta), Is with sin, theta = atan2(q_y, q_z) (0 at
 *               q = 0); NaN for empty bins.
 * Ac[k], As[k] = a_k / sum_j sqrt(a_j^s^2 + a_j^c^2), a_k = sum of I_k over
 * the finite nodes.  0 <= kmax <= 1023.  Ic, Is: [kmax+1][nbins]; counts,
 * qmean: [nbins]; Ac, As: [kmax+1]; counts, qmean, Ac, As may be NULL.
 * img host or device per img_is_device, outputs per out_is_device.
 * Synchronous. */
nms_status nms_angular_spectrum(nms_plan_t plan, const double* img, int32_t img_is_device, int32_t kmax,
                                int32_t nbins, const double* bin_edges, double* Ic, double* Is,
                                int64_t* counts, double* qmean, double* Ac, double* As,
                                int32_t out_is_device);

/* 2D correlation function of a per-pixel image (paper, Eq. crav2d):
 *   C(rho_m, alpha_n) = sum_p W_p f_p exp(+i q_p . rho_vec),
 *   rho_vec = rho_m (0, sin alpha_n, cos alpha_n)  (so q.rho_vec = q rho cos(theta - alpha)),
 * with the trapezoid rule of the grid as W_p: POLAR W = w_i q_i 2 pi/n1
 * (w_i the trapezoid weights of the q nodes: q dq dtheta), CARTESIAN
 * W = w_a w_b (trapezoid weights of the q_y and q_z nodes: dq_y dq_z).
 * LIST grids have no quadrature: UNSUPPORTED.  rho [n_rho] and alpha
 * [n_alpha] on the host, n_rho * n_alpha <= 2^24.  C: [n_rho][n_alpha][2]
 * (re, im).  scale (may be NULL) = sum_p |W_p f_p|, the magnitude the
 * rounding error is relative to (FP32 terms, two-float sums: |error| is of
 * order 1e-7 scale).  Outputs host or device per out_is_device.
 * Synchronous. */
nms_status nms_correlation_2d(nms_plan_t plan, const double* img, int32_t img_is_device, int32_t n_rho,
                              const double* rho, int32_t n_alpha, const double* alpha, double* C,
                              double* scale, int32_t out_is_device);

/* Correlation and pair-distance distribution functions (paper, Eqs. crrad
 * and prrad): c(r_m) = prefactor * trapz_i [ I(q_i) j0(q_i r_m) q_i^2 ],
 * p(r_m) = r_m^2 c(r_m), trapezoid over the nodes in the given order with
 * non-finite (q_i, I_i) nodes dropped; j0(0) = 1.  The printed prefactor is
 * 1/(2 pi^2); pass 0 to get it.  All arrays host or device per is_device
 * (c_r or p_r may be NULL).  cuda_stream as in nms_plan_create.
 * Synchronous. */
nms_status nms_correlation(int32_t nq, const double* q, const double* Iq, int32_t nr,
                           const double* r, double prefactor, double* c_r, double* p_r,
                           int32_t is_device, void* cuda_stream);

/* Per-object, orientation-averaged azimuthal averages (paper, Eq. iqazi on
 * ring bins, averaged over the plan's rotations; Sec. "Summation approach"
 * form factors of the objects without interparticle interference).  Call
 * after nms_plan_create and before nms_amplitudes: every following
 * nms_amplitudes then also bins, for each object k (or for the whole sample
 * when the plan has one object or want_dilute = 0), the response
 * response_id (N, M, P, SF or UNPOL) of its own amplitude F_k over the ring
 * bins edges[b] <= |q| < edges[b+1] (bin_edges host [nbins+1], increasing,
 * nbins <= 8192).  This is how surrogate training data are generated in one
 * batched pass.  Tensor-core path on a CARTESIAN grid only (UNSUPPORTED
 * otherwise). */
nms_status nms_plan_object_iq(nms_plan_t plan, int32_t response_id, int32_t nbins, const double* bin_edges);

/* Results of nms_plan_object_iq after nms_amplitudes: Iq[k][b] = mean over
 * the bin's pixels and over the rotations (NaN for empty bins), counts[b] =
 * pixels in bin b, qmean[b] = their mean |q| (counts, qmean may be NULL).
 * Host or device per out_is_device.  Synchronous. */
nms_status nms_get_object_iq(nms_plan_t plan, double* Iq, int64_t* counts, double* qmean, int32_t out_is_device);

/* Per-stage device times in milliseconds, summed over all nms_amplitudes
 * calls since the plan was created or the last reset (needs opt.timing=1):
 * stage 0 = rotation/weights, 1 = phase tables, 2 = tensor-core GEMM,
 * 3 = direct sum, 4 = promotion/reduction of partials, 5 = G accumulation.
 * launches[s] counts the kernel launches of stage s.  Synchronises. */
nms_status nms_plan_stage_ms(nms_plan_t plan, double ms[8], int64_t launches[8], int32_t reset);

/* ---------------------------------------------------------------------
 * Learned surrogate.  The paper has no learned component: this MLP maps the
 * parameters of a magnetization family to its orientation-averaged
 * log10 I(q), trained on curves the batched transform computes
 * (nms_plan_object_iq); the exact transform stays the reference for its
 * error.  Architecture n_in -> H -> H -> n_out with SiLU, FP32 master
 * weights, BF16 weights/activations in the GEMMs with FP32 accumulation,
 * mean-squared error on standardised targets, Adam.  Parameters are one
 * flat FP32 vector: W1[H][n_in] b1[H] W2[H][H] b2[H] W3[n_out][H] b3[n_out].
 * Inputs are scaled to [-1, 1] with the per-input bounds given at create.
 * --------------------------------------------------------------------- */
typedef struct nms_surrogate_s* nms_surrogate_t;

/* x_lo, x_hi: host [n_in] input bounds; weights He-uniform from seed. */
nms_status nms_surrogate_create(nms_surrogate_t* out, int32_t n_in, int32_t n_hidden, int32_t n_out,
                                const float* x_lo, const float* x_hi, uint64_t seed, void* cuda_stream);

/* Target standardisation (host [n_out] each, y_std > 0).  When not set, the
 * first nms_surrogate_train computes them from its targets. */
nms_status nms_surrogate_set_target_stats(nms_surrogate_t s, const float* y_mean, const float* y_std);

/* Mini-batch Adam over device data X [n][n_in], Y [n][n_out] (FP32,
 * unnormalised targets), epochs passes with a seeded shuffle per epoch;
 * final_loss (host, may be NULL) = mean 0.5 (y_n - t_n)^2 of the last epoch
 * on standardised targets. */
nms_status nms_surrogate_train(nms_surrogate_t s, const float* X, const float* Y, int64_t n, int32_t batch,
                               int32_t epochs, float lr, uint64_t shuffle_seed, float* final_loss);

/* One forward + backward over device rows X [n][n_in], Y [n][n_out] without
 * an update: grad (host [n_params]) = d loss / d params, loss (host) = mean
 * 0.5 (y_n - t_n)^2.  For gradient checks. */
nms_status nms_surrogate_gradients(nms_surrogate_t s, const float* X, const float* Y, int32_t n, float* grad,
                                   double* loss);

/* Y [n][n_out] (device, FP32, de-standardised log10 I) for device X [n][n_in].
 * With H = 256, n_out <= 256 and n_in <= 8 the whole network runs as one
 * tensor-core kernel per 128 outputs and the call synchronises the
 * surrogate's stream to read that kernel's error word (TIMEOUT if a bounded
 * wait gave up); otherwise it is asynchronous on the surrogate's stream. */
nms_status nms_surrogate_infer(nms_surrogate_t s, const float* X, int64_t n, float* Y);

/* Master parameters to/from host (count = number of parameters). */
nms_status nms_surrogate_get_params(nms_surrogate_t s, float* host, int64_t* count);
nms_status nms_surrogate_set_params(nms_surrogate_t s, const float* host, int64_t count);

/* Checkpoint (weights, Adam state, step, standardisation, bounds) to a file,
 * and back into a surrogate of the same shape. */
nms_status nms_surrogate_save(nms_surrogate_t s, const char* path);
nms_status nms_surrogate_load(nms_surrogate_t s, const char* path);
nms_status nms_surrogate_destroy(nms_surrogate_t s);

/* Direct Fourier sums with no device allocation.  The paper has no
 * counterpart: this entry point exists for callers that cannot let a library
 * allocate GPU memory -- applications whose device memory is owned by their
 * own allocator or budget, and latency-sensitive loops in which a
 * cudaMalloc/cudaFree pair would stall or synchronise the device.
 * It computes the same sums as the FP32_DIRECT path of a plan with identity
 * rotation and a LIST grid:
 *   F[c][p] = sum_j w[c][j] exp(-i (qy[p] Y[j] + qz[p] Z[j])),
 *   out F[c][p][2] = (Re, Im), c = 0..3.
 *   Y, Z    device [n_cells] FP64 (already rotated) coordinates.
 *   w       device [4][n_cells] FP64 weights (V N, V M_x, V M_y, V M_z).
 *   qy, qz  device [n_q] FP64 detector points.
 *   F       device [4][n_q][2] FP64 output (overwritten).
 * The only scratch is a 16 MiB array inside the library image (resident on
 * every GPU that loads libnms until the process exits), so n_q is limited to
 * 262144 points (a 512 x 512 detector); larger n_q returns
 * NMS_ERR_INVALID_ARG.  The first call on a device looks up that array's
 * device address (cudaGetSymbolAddress) and caches it with the device's
 * current context: make that first call before any stream capture.  The
 * cached address does not outlive its context: a call that finds a new
 * context (after cudaDeviceReset) looks it up again, so make the first call
 * after a reset outside a capture too.  All calls share the array, so calls
 * whose kernels can overlap on the GPU (different streams without ordering)
 * race.  n_cells = 0 writes zeros; n_q = 0 does nothing.
 * Asynchronous on cuda_stream; no cudaMalloc, cudaFree or other allocating
 * call is made. */
nms_status nms_dsft_direct_noalloc(int64_t n_cells, const double* Y, const double* Z, const double* w,
                                   int64_t n_q, const double* qy, const double* qz, double* F,
                                   void* cuda_stream);

/* The evaluation the plan settled on: precision = the nms_precision in use
 * (AUTO resolved), kc_cells = cells per TMEM accumulation chunk and
 * items_per_sm = work items per SM of each GEMM launch (tensor path; 0
 * otherwise), after autotuning when it was requested; gemm_form = 0 (one
 * CTA per 128 x 128 tile), 2 (two-SM MMA over pairs of A tiles) or 3 (POLAR
 * grid whose ray GEMM has one B tile and at most three A tiles, at most
 * 48 x 64 |q| nodes and one weight set: the operands are generated in the
 * GEMM's shared memory, no phase tables; environment NMS_RAY_FUSED=0 keeps
 * the tables), -1 off the tensor path; mirror_y / mirror_z = 1 where the detector axis is
 * symmetric about q = 0 (lo = -hi) and the GEMM evaluates its q >= 0 half,
 * writing both signs (cos is even and sin odd in q; Sec. "Summation
 * approach" sum, split by parity).  Any pointer may be NULL. */
nms_status nms_plan_info(nms_plan_t plan, int32_t* precision, int32_t* kc_cells, int32_t* items_per_sm,
                         int32_t* gemm_form, int32_t* mirror_y, int32_t* mirror_z);

/* Loop mode (paper, Sec. "Program description": batch runs over field-,
 * temperature- or time-dependent data sets of one geometry): select which
 * weight set 0 <= set < n_sets subsequent nms_get_amplitudes and
 * nms_response calls report.  The default is set 0.  The Fourier sums of
 * all sets are computed by each nms_amplitudes call. */
nms_status nms_select_set(nms_plan_t plan, int32_t set);

/* Failure-path self-test (the paper has no counterpart): one thread waits on
 * a device mbarrier that nothing arrives on, with the bounded wait every
 * kernel of the library uses (%globaltimer, limit_us microseconds,
 * 1 <= limit_us <= 1e7).  The wait runs out, the kernel records an error
 * code and returns, so this returns NMS_ERR_TIMEOUT and leaves the CUDA
 * context usable.  Synchronous on cuda_stream. */
nms_status nms_selftest_bounded_wait(int64_t limit_us, void* cuda_stream);

/* Self-test of the sine and cosine that the fused ray GEMM form generates
 * its operands with (the phase 2 pi t of Eq. qdef's exponential, t in turns,
 * |t| <= 1/2, taken in quarter turns, split at the nearest one, Taylor series
 * of the remainder; the paper has no counterpart): for each of the n host
 * values t[i],
 * out[4i], out[4i + 1] = sin, cos of 2 pi t[i] by that routine and
 * out[4i + 2], out[4i + 3] = the same by CUDA's sincospif, for comparison
 * with each other and with exact values.  out (host) holds 4n floats.
 * n = 0 does nothing; n < 0 or a NULL array with n > 0 is
 * NMS_ERR_INVALID_ARG.  Synchronous on cuda_stream. */
nms_status nms_selftest_sincos(int64_t n, const float* t, float* out, void* cuda_stream);

/* Release every device resource of the plan.  NULL is accepted. */
nms_status nms_plan_destroy(nms_plan_t plan);

/* Thread-local text of the last failure in this thread ("" if none).  It
 * takes no plan: a failed nms_plan_create has no plan to ask, and with one
 * plan per host thread the thread's last failure is the plan's. */
const char* nms_last_error(void);

/* Library version, e.g. "nms 0.1.0 sm_103a". */
const char* nms_version(void);

#ifdef __cplusplus
}
#endif

#endif /* NMS_H */
