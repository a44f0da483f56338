// Internal declarations of libnms (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "nms.h"

namespace nms {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
nms_status cuda_fail(cudaError_t e, const char* what);

#define NMS_CUDA_TRY(expr)                                        \
    do {                                                          \
        cudaError_t _e = (expr);                                  \
        if (_e != cudaSuccess) return ::nms::cuda_fail(_e, #expr); \
    } while (0)

// ---------------------------------------------------------------- stages
enum Stage { ST_PREP = 0, ST_TABLES = 1, ST_GEMM = 2, ST_DIRECT = 3, ST_REDUCE = 4, ST_GACC = 5, ST_COUNT = 8 };

struct StageTimer {
    bool on = false;
    cudaStream_t stream = nullptr;
    struct Pending { int stage; cudaEvent_t a, b; };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> pool;
    double ms[ST_COUNT] = {0};
    int64_t launches[ST_COUNT] = {0};
    int open_stage = -1;
    cudaEvent_t open_ev = nullptr;
    cudaEvent_t get_event();
    void begin(int stage);
    void end(int stage, int n_launch);
    nms_status collect();
    void release();
};

// A row-major 3x3 rotation passed to kernels by value.
struct RotMat {
    double m[9];
};

// Amplitudes of a batch of tensor-path outputs (F_b), complex FP32 values
// (float2) in two planes: high words, and low words of a two-float value.
// Value (output o, channel row m = nch a + c, q_z index b) sits at
// o * ostride2 + (b - zs0) * mrows + m in each plane, with mrows = nch * ny
// and ostride2 = (nz - zs0) * mrows: the GEMM row index runs fastest, so the
// 32 rows an epilogue warp holds go out as 256 contiguous bytes, and a
// pixel's channels are adjacent.  An output assembled from one piece keeps
// its value, rounded to FP32, in the high plane only; an output whose pieces
// (table chunks) add up keeps the two-float value, normalised, in both
// planes (two[o] = 1).  Either way the high plane holds the value rounded to
// FP32, which is what the Hermitian products and bins read.
//
// zs0 > 0: the detector is point-symmetric (both axes symmetric about
// q = 0), and only the q_z rows b >= zs0 (q_z >= 0) are stored.  The weights
// are real, so F(-q) = conj F(q): the value at (a, b < zs0) is the conjugate
// of the stored value at the mirror pixel (ny - 1 - a, nz - 1 - b).  The
// products F F^dagger at -q are the conjugates of those at q, and so is a
// sum of shifted amplitudes (its phase factors conjugate as well).
struct FbView {
    const float2* hi;       // channel 0 of the chosen weight set, output 0
    const float2* lo;
    const uint8_t* two;     // per output of the batch: 1 = low plane in use
    int64_t ostride2;       // float2 between outputs
    int mrows;              // float2 between consecutive q_z (nch * ny)
    int nch, ny, nz;
    int zs0;                // first stored q_z row (0: all rows stored)
    __host__ __device__ int64_t idx(int64_t o, int a, int b) const
    {
        return o * ostride2 + (int64_t)(b - zs0) * mrows + (int64_t)nch * a;
    }
    // pixels held in the planes: ny * (nz - zs0)
    __host__ __device__ int64_t stored_pixels() const { return (int64_t)ny * (nz - zs0); }
    // a stored pixel at q_z row b >= zs0 whose point mirror is not stored
    // (every stored row but the q_z = 0 row of an odd node count)
    __host__ __device__ bool mirror_unstored(int b) const { return zs0 > 0 && nz - 1 - b < zs0; }
#ifdef __CUDACC__
    // channel c of output o at (a, b), rounded to FP32
    __device__ __forceinline__ float2 load(int64_t o, int a, int b, int c) const
    {
        if (b >= zs0) return hi[idx(o, a, b) + c];
        const float2 v = hi[idx(o, ny - 1 - a, nz - 1 - b) + c];
        return make_float2(v.x, -v.y);
    }
    // the same in FP64 with the low word, where the output has one
    __device__ __forceinline__ double2 load_f64(int64_t o, int a, int b, int c) const
    {
        const bool m = b < zs0;
        const int64_t j = m ? idx(o, ny - 1 - a, nz - 1 - b) + c : idx(o, a, b) + c;
        const float2 h = hi[j];
        const float2 l = two[o] ? lo[j] : make_float2(0.f, 0.f);
        const double re = (double)h.x + (double)l.x, im = (double)h.y + (double)l.y;
        return make_double2(re, m ? -im : im);
    }
#endif
};

// Detector axes of one tensor-path GEMM: the full grid (ny x nz), the first
// node of the GEMM's part of each axis (hy, hz: 0, or the first q >= 0 node of
// an axis symmetric about q = 0) and its length (nyg = ny - hy, nzg = nz - hz);
// my, mz = 1: the axis is symmetric and the epilogue also writes the mirrored
// nodes n - 1 - h - i (except a node that is its own mirror, q = 0).  zs0:
// first q_z row of the stored amplitudes (FbView); zs0 = hz > 0 when both
// axes are symmetric, and then the -q_z writes are left out.
struct AxisMap {
    int ny, nz, hy, hz, nyg, nzg, my, mz, zs0;
};

// ---------------------------------------------------------------- plan
struct Plan {
    cudaStream_t stream = nullptr;
    nms_options opt{};
    nms_qgrid grid{};
    int path = 0;                 // nms_precision actually used
    int64_t n_cells = 0, n_objects = 1, npix = 0;
    int32_t n_rot = 1;
    int32_t n_sets = 1;           // weight sets (loop mode); nuc/mag [S][n]
    int32_t sel_set = 0;          // set reported by nms_response / nms_get_amplitudes
    double V = 1.0, bH = 1.0, P[3] = {0, 0, 1};
    bool has_nuc = false, has_mag = false, has_centers = false;
    std::vector<int64_t> h_off;   // [K+1]
    std::vector<double> h_rot;    // [n_rot][9]
    std::vector<double> h_cen;    // [K][3]

    // device inputs (FP64)
    double* d_pos = nullptr;      // [n][3]
    double* d_vol = nullptr;      // [n]
    double* d_nuc = nullptr;      // [S][n] or null
    double* d_mag = nullptr;      // [S][n][3] or null
    double* d_cen_cell = nullptr; // [n][3] object centre of each cell, or null
    // q-grid (FP64) and the turns form used by the kernels
    double* d_qy = nullptr; double* d_qz = nullptr;
    double* d_hy = nullptr; double* d_hz = nullptr; double* d_qa = nullptr;
    float4* d_qturn = nullptr;    // per pixel (qy/2pi hi, lo, qz/2pi hi, lo)
    // per-rotation cell data
    float4* d_cpos = nullptr;     // global positions R(x + r^k): (Yh, Yl, Zh, Zl)
    float4* d_cposl = nullptr;    // local positions R x (dilute), may alias d_cpos
    float4* d_cw = nullptr;       // weights (wN, wMx', wMy', wMz') FP32
    double* d_yz = nullptr;       // FP64 (Y, Z) global, [2][n] (tensor-path tables)
    double* d_yzl = nullptr;      // FP64 (Y, Z) local
    double* d_w64 = nullptr;      // FP64 weights [4][n]
    // results
    double* d_F = nullptr;        // [S][4][npix][2] amplitudes of the last sum
    double* d_Ftot = nullptr;     // [S][4][npix][2] total amplitude (object path)
    double* d_Fpart = nullptr;    // split partials [splits][4][npix][2]
    int64_t fpart_splits = 0;
    double* d_Gtot = nullptr;     // [S][16][npix]
    double* d_Gdil = nullptr;     // [S][16][npix] (want_dilute)
    int32_t* d_err = nullptr;     // device error word (timeouts)
    bool have_G = false;
    int32_t rot_done = 0;

    // tensor path workspace
    void* d_tab = nullptr;        // split-FP16 operand tables
    size_t tab_bytes = 0;
    int64_t tab_cells = 0;        // cells per table chunk
    double* d_wscale = nullptr;   // per-channel power-of-two weight scales [4]
    void* tc_state = nullptr;     // tensor-path state (k_gemm.cu)
    double h_wmax[2] = {0, 0};    // max_j V_j |N_j|, max_j V_j |M_j| (rotation invariant)
    // per-object azimuthal averages (nms_plan_object_iq)
    int32_t oiq_id = -1;
    int oiq_nbins = 0;
    int32_t* d_bin_of = nullptr;  // bin of each pixel or -1
    double* d_Iobj = nullptr;     // [objects][nbins] sums of the response
    std::vector<int64_t> oiq_counts;
    std::vector<double> oiq_qmean;
    int64_t max_sum_cells = 0;    // largest cell range summed in one call

    StageTimer timer;
};

// ---------------------------------------------------------------- kernels (launchers)
// Rotation and weights for cells [0, n): FP64 positions -> two-float, FP32 weights.
cudaError_t launch_prep(Plan& p, const double* R9, cudaStream_t s, int set = 0);
cudaError_t launch_weight_max(const Plan& p, double wmax[2], cudaStream_t s);
// Direct sum over cells [c0, c1) of the given position array into split partials.
cudaError_t launch_direct(const Plan& p, const float4* cpos, int64_t c0, int64_t c1,
                          bool compensated, int splits, cudaStream_t s);
// Sum split partials into out [4][npix][2] (assign).
cudaError_t launch_reduce_splits(const Plan& p, int splits, double* out, cudaStream_t s);
// G += F F^dagger for every pixel (F: [4][npix][2]).
cudaError_t launch_gacc(const Plan& p, const double* F, double* G, cudaStream_t s);
// out[p] = factor * F_tot accumulate with object phase (total from objects).
cudaError_t launch_shift_add(const Plan& p, const double* Fk, double cy, double cz, double* Ftot,
                             cudaStream_t s);
// Response id from G (FP64), divided by norm (number of rotations).
cudaError_t launch_response(const Plan& p, int id, const double* Ga, const double* Gb, double norm,
                            double* out, cudaStream_t s);
// Azimuthal averages.
cudaError_t launch_polar_nodes(const Plan& p, int64_t* counts, double* qmean, cudaStream_t s);
cudaError_t launch_angspec_polar(const Plan& p, const double* img, int kmax, double* Ic, double* Is, cudaStream_t s);
cudaError_t launch_angspec_rings(const Plan& p, const double* img, const double* d_edges, int nbins, int kmax,
                                 void* work, double* Ic, double* Is, int64_t* counts, double* qmean, cudaStream_t s);
size_t angspec_rings_work_bytes(int64_t npix, int nbins, int kmax);
cudaError_t launch_modal_amplitudes(const double* Ic, const double* Is, int nb, int kmax, double* Ac, double* As,
                                    cudaStream_t s);
cudaError_t launch_corr2d(const Plan& p, const double* img, const double* d_rho, int n_rho, const double* d_alpha,
                          int n_alpha, float* d_w, double* d_wabs, float4* d_pts, double2* d_part, int splits,
                          double2* d_C, cudaStream_t s);
int corr2d_splits(int64_t npix, int n_out);
cudaError_t launch_azimuthal_polar(const Plan& p, const double* img, double* Iq, cudaStream_t s);
cudaError_t launch_correlation(int nq, const double* q, const double* Iq, int nr, const double* r,
                               double pref, double* c, double* pr, double* scratch_q, double* scratch_f,
                               int* scratch_n, cudaStream_t s);

// Tensor-core path (split-FP16 tcgen05 GEMM): schedule at plan creation,
// all rotations/objects of one nms_amplitudes call, release.
nms_status tc_setup(Plan& p);
struct TcState;
nms_status tc_autotune(Plan& p, TcState& t);
nms_status tc_amplitudes(Plan& p, cudaStream_t s);
void tc_release(Plan& p);

int device_sm_count();
// Fused ray GEMM: with ray_sc set, cpos / cw are the cells rotated once per
// rotation ([n_rot][n_cells]) and the kernel projects them on the rays of
// slots slot0 .. slot0 + n_rl - 1 (n_rl <= 64); ray_sc = null: cpos / cw are
// the per-slot projections of the batch.
struct RayProjection {
    const float4* ray_sc = nullptr;   // [n_rays] (sin hi, lo, cos hi, lo)
    int64_t n_cells = 0;
    int slot0 = 0, n_rays = 0, n_rl = 0;
};
cudaError_t launch_selftest_wait(uint64_t limit_ns, int32_t* err, cudaStream_t s);
cudaError_t launch_selftest_sincos(const float* t, int64_t n, float* out, cudaStream_t s);

// Device memory of plans: a per-device library memory pool that keeps up to
// 16 GiB of freed memory for later plans (creating and destroying a plan
// then maps and unmaps no pages).  The memory is usable on any stream when
// plan_malloc returns.  plan_free(ptr, s) releases it stream-ordered after
// all work issued so far on s, the stream every use of it was issued on (or
// ordered before): memory a kernel may still read is never handed out again
// or returned to the driver.
cudaError_t plan_malloc_raw(void** ptr, size_t bytes);
void plan_free(void* ptr, cudaStream_t used_on);
template <class T>
inline cudaError_t plan_malloc(T** ptr, size_t bytes)
{
    return plan_malloc_raw(reinterpret_cast<void**>(ptr), bytes);
}

// Ring bin of |q| = x: b with e[b] <= x < e[b+1] (e increasing, nb bins), or
// -1 outside [e[0], e[nb]) and for NaN.
__device__ __forceinline__ int find_bin(const double* __restrict__ e, int nb, double x)
{
    if (!(x >= e[0]) || !(x < e[nb])) return -1;
    int lo = 0, hi = nb;  // e[lo] <= x < e[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (x >= e[mid]) lo = mid;
        else hi = mid;
    }
    return lo;
}
// Direct sum of cells [c0, c1) (compensated unless the plan asked for the
// naive phase) into out [4][npix][2] through the split partials.
nms_status direct_sum_range(Plan& p, const float4* cpos, int64_t c0, int64_t c1, double* out);
int tc_tuned_kc_cells(const Plan& p);
int tc_tuned_items_per_sm(const Plan& p);
// GEMM form (0 one CTA per tile, 2 two-SM MMA; -1 without a tensor path) and
// which detector axes the GEMM covers on their q >= 0 half only
void tc_form_info(const Plan& p, int32_t* form, int32_t* mirror_y, int32_t* mirror_z);
cudaError_t launch_grid(const nms_qgrid& g, int64_t np, const double* d_qlist, double* qy, double* qz, double* hy,
                        double* hz, double* qa, float4* qturn, cudaStream_t s);
cudaError_t launch_obj_bin(const FbView& F, int n_out, const int32_t* out_obj, const Plan& p, const int32_t* bin_of,
                           int nbins, int id, double* Iobj, cudaStream_t s);
int64_t tc_object_count(const Plan& p);

}  // namespace nms

// The opaque handle of the C ABI is the plan itself.
struct nms_plan_s : public nms::Plan {};
