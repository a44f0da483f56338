// nms_dsft_direct_noalloc: the compensated FP32 direct Fourier sum for callers
// that cannot let the library allocate device memory.
//
// Who needs this: applications whose device memory is owned by their own
// allocator or budget (a framework that forbids libraries from calling
// cudaMalloc behind its back), and latency-sensitive loops in which a
// cudaMalloc/cudaFree pair would stall or synchronise the device.  The plan
// API allocates its workspace; this entry point takes device inputs and a
// device output from the caller and uses only a fixed scratch area that is
// part of the library image.
//
// The scratch is a file-scope __device__ array of NOALLOC_SCRATCH_BYTES
// (16 MiB).  Every GPU that loads libnms keeps those 16 MiB until the process
// exits.  Host code cannot use the array's name as a device address, so the
// first call on each device looks the address up with cudaGetSymbolAddress
// (with that device current) and caches it together with the device's
// current context; make that first call before any stream capture.  A call
// that finds another context current on the device (after cudaDeviceReset,
// or a primary context torn down and created again) looks the address up
// again instead of using the cached one; that call, too, belongs outside a
// stream capture.  All calls share the array: two calls whose kernels overlap
// on the GPU (different streams, no ordering between them) race on it.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>
#include <string>

#include "nms.h"
#include "nms_internal.h"

namespace nms {

constexpr int64_t NOALLOC_SCRATCH_BYTES = 16ll << 20;
constexpr int64_t NOALLOC_SCRATCH_DOUBLES = NOALLOC_SCRATCH_BYTES / 8;
constexpr int64_t NOALLOC_MAX_Q = NOALLOC_SCRATCH_DOUBLES / 8;   // one split of [4][n_q][2]
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

static double* g_scratch_addr[NOALLOC_MAX_DEVICES];
static void* g_scratch_ctx[NOALLOC_MAX_DEVICES];   // context the cached address belongs to
static std::mutex g_scratch_mu;

// The driver's current context (cuCtxGetCurrent through the runtime's
// driver entry point; no link-time dependency on libcuda).
static void* current_context()
{
    typedef int (*GetCurrent)(void**);
    static GetCurrent fn = nullptr;
    if (!fn) {
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !f) {
            cudaGetLastError();
            return nullptr;
        }
        fn = (GetCurrent)f;
    }
    void* ctx = nullptr;
    return fn(&ctx) == 0 ? ctx : nullptr;
}

// Device address of the scratch array on the current device: looked up once
// per device and context, with that device current.
static nms_status scratch_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
        set_error("device ordinal beyond the supported range of the static scratch table");
        return NMS_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    // before the first runtime call on the device there may be no context
    // yet (ctx = NULL): cudaGetSymbolAddress creates it
    void* ctx = current_context();
    if (!g_scratch_addr[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_addr[dev] = (double*)p;
        g_scratch_ctx[dev] = current_context();
    }
    *out = g_scratch_addr[dev];
    return NMS_OK;
}

constexpr int NA_THREADS = 256;
constexpr int NA_TILE = 512;
constexpr int NA_GROUP = 8;

__device__ __forceinline__ void na_two_sum(float& hi, float& lo, float x)
{
    float s = hi + x;
    float bb = s - hi;
    float e = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo += e;
}

// One pixel per thread; cells staged in shared memory as two-float (Y, Z)
// and FP32 weights.  Partials [split][4][n_q][2] go to the scratch array.
__global__ void __launch_bounds__(NA_THREADS)
k_direct_noalloc(int64_t n, const double* __restrict__ Y, const double* __restrict__ Z,
                 const double* __restrict__ w, int64_t nq, const double* __restrict__ qy,
                 const double* __restrict__ qz, double* __restrict__ part)
{
    __shared__ float4 s_pos[NA_TILE];
    __shared__ float4 s_w[NA_TILE];
    const int splits = gridDim.y;
    const int64_t per = (n + splits - 1) / splits;
    const int64_t b0 = (int64_t)blockIdx.y * per;
    const int64_t b1 = min(n, b0 + per);
    const int64_t p = (int64_t)blockIdx.x * NA_THREADS + threadIdx.x;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (p < nq) {
        const double ty = qy[p] / (2.0 * M_PI), tz = qz[p] / (2.0 * M_PI);
        const float tyh = (float)ty, tzh = (float)tz;
        q = make_float4(tyh, (float)(ty - (double)tyh), tzh, (float)(tz - (double)tzh));
    }
    float hi[8], lo[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) { hi[a] = 0.f; lo[a] = 0.f; }
    for (int64_t t0 = b0; t0 < b1; t0 += NA_TILE) {
        const int nt = (int)min((int64_t)NA_TILE, b1 - t0);
        const int npad = ((nt + NA_GROUP - 1) / NA_GROUP) * NA_GROUP;
        __syncthreads();
        for (int i = threadIdx.x; i < npad; i += NA_THREADS) {
            if (i < nt) {
                const int64_t j = t0 + i;
                const double y = Y[j], z = Z[j];
                const float yh = (float)y, zh = (float)z;
                s_pos[i] = make_float4(yh, (float)(y - (double)yh), zh, (float)(z - (double)zh));
                s_w[i] = make_float4((float)w[j], (float)w[n + j], (float)w[2 * n + j], (float)w[3 * n + j]);
            } else {
                s_pos[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                s_w[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        for (int g = 0; g < npad / NA_GROUP; ++g) {
            float acc[8];
#pragma unroll
            for (int a = 0; a < 8; ++a) acc[a] = 0.f;
#pragma unroll 4
            for (int u = 0; u < NA_GROUP; ++u) {
                const float4 c = s_pos[g * NA_GROUP + u];
                const float4 wv = s_w[g * NA_GROUP + u];
                // two-float phase in turns, exact reduction, sincospif
                const float py = q.x * c.x;
                const float ey = fmaf(q.x, c.x, -py) + fmaf(q.x, c.y, q.y * c.x);
                const float pz = q.z * c.z;
                const float ez = fmaf(q.z, c.z, -pz) + fmaf(q.z, c.w, q.w * c.z);
                const float s = py + pz;
                const float bb = s - py;
                const float es = (py - (s - bb)) + (pz - bb);
                const float t = (s - rintf(s)) + (es + ey + ez);
                float sn, cs;
                sincospif(2.0f * t, &sn, &cs);
                acc[0] = fmaf(wv.x, cs, acc[0]);
                acc[1] = fmaf(-wv.x, sn, acc[1]);
                acc[2] = fmaf(wv.y, cs, acc[2]);
                acc[3] = fmaf(-wv.y, sn, acc[3]);
                acc[4] = fmaf(wv.z, cs, acc[4]);
                acc[5] = fmaf(-wv.z, sn, acc[5]);
                acc[6] = fmaf(wv.w, cs, acc[6]);
                acc[7] = fmaf(-wv.w, sn, acc[7]);
            }
#pragma unroll
            for (int a = 0; a < 8; ++a) na_two_sum(hi[a], lo[a], acc[a]);
        }
    }
    if (p < nq) {
        double2* out = reinterpret_cast<double2*>(part + (int64_t)blockIdx.y * 8 * nq);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            out[(int64_t)c * nq + p] = make_double2((double)hi[2 * c] + (double)lo[2 * c],
                                                    (double)hi[2 * c + 1] + (double)lo[2 * c + 1]);
    }
}

__global__ void k_noalloc_reduce(const double* __restrict__ part, int splits, int64_t m, double* __restrict__ F)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double acc = 0.0;
    for (int s = 0; s < splits; ++s) acc += part[(int64_t)s * m + i];
    F[i] = acc;
}

}  // namespace nms

using namespace nms;

extern "C" nms_status nms_dsft_direct_noalloc(int64_t n_cells, const double* Y, const double* Z, const double* w,
                                              int64_t n_q, const double* qy, const double* qz, double* F,
                                              void* cuda_stream)
{
    set_error("");
    if (n_cells < 0 || n_q < 0) {
        set_error("n_cells and n_q must be >= 0");
        return NMS_ERR_INVALID_ARG;
    }
    if (n_q > NOALLOC_MAX_Q) {
        set_error("n_q = " + std::to_string(n_q) + " exceeds the static scratch capacity of " +
                  std::to_string(NOALLOC_MAX_Q) + " q-points (16 MiB); use the plan API for larger grids");
        return NMS_ERR_INVALID_ARG;
    }
    if ((n_cells > 0 && (!Y || !Z || !w)) || (n_q > 0 && (!qy || !qz || !F))) {
        set_error("NULL device pointer");
        return NMS_ERR_INVALID_ARG;
    }
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
        cudaGetLastError();
        set_error("no CUDA device available (libnms has no CPU fallback)");
        return NMS_ERR_CUDA;
    }
    if (n_q == 0) return NMS_OK;
    double* scratch = nullptr;
    nms_status st = scratch_address(&scratch);
    if (st != NMS_OK) return st;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int64_t pix_blocks = (n_q + NA_THREADS - 1) / NA_THREADS;
    int64_t splits = ((int64_t)device_sm_count() * 8 + pix_blocks - 1) / pix_blocks;
    splits = std::min<int64_t>(splits, std::max<int64_t>(1, n_cells / 2048));
    splits = std::min<int64_t>(splits, NOALLOC_SCRATCH_DOUBLES / (8 * n_q));
    splits = std::max<int64_t>(1, std::min<int64_t>(splits, 65535));
    // every partial slot the reduction reads is written by this call first,
    // so the scratch needs no clearing
    k_direct_noalloc<<<dim3((unsigned)pix_blocks, (unsigned)splits), NA_THREADS, 0, s>>>(n_cells, Y, Z, w, n_q, qy,
                                                                                          qz, scratch);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_direct_noalloc launch");
    const int64_t m = 8 * n_q;
    k_noalloc_reduce<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(scratch, (int)splits, m, F);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "k_noalloc_reduce launch");
    return NMS_OK;
}
