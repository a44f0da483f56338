// C ABI of libnms: plan creation, orchestration of the kernels, results.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "nms.h"
#include "nms_internal.h"

#include <map>
#include <mutex>

// Stream-ordered scratch of the host-called helpers comes from a private
// memory pool per device that keeps its memory on release: the default pool
// hands freed memory back to the driver at every synchronisation, so each
// call would map fresh pages again.
namespace {
// The memory pools are bypassed (plain cudaMalloc / cudaFree and the default
// stream-ordered pool) when NMS_NO_POOL is set or a CUDA injection tool such
// as a profiler is attached: kernel replay with device-memory save and
// restore is only known to work on ordinary allocations.
bool pools_enabled()
{
    static const bool on = getenv("NMS_NO_POOL") == nullptr && getenv("CUDA_INJECTION64_PATH") == nullptr;
    return on;
}

struct PlanPool {
    cudaMemPool_t pool = nullptr;
    cudaStream_t stream = nullptr;   // allocation-ordering stream
};
std::mutex g_plan_pool_mu;
std::map<int, PlanPool> g_plan_pools;

cudaError_t plan_pool(PlanPool& out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_plan_pool_mu);
    auto it = g_plan_pools.find(dev);
    if (it != g_plan_pools.end()) {
        out = it->second;
        return cudaSuccess;
    }
    PlanPool pp;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    e = cudaMemPoolCreate(&pp.pool, &props);
    if (e != cudaSuccess) return e;
    uint64_t keep = 16ull << 30;
    cudaMemPoolSetAttribute(pp.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    e = cudaStreamCreateWithFlags(&pp.stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
    g_plan_pools[dev] = pp;
    out = pp;
    return cudaSuccess;
}
}  // namespace

namespace nms {
cudaError_t plan_malloc_raw(void** ptr, size_t bytes)
{
    *ptr = nullptr;
    if (!pools_enabled()) return cudaMalloc(ptr, bytes > 0 ? bytes : 8);
    PlanPool pp;
    cudaError_t e = plan_pool(pp);
    if (e != cudaSuccess) return e;
    e = cudaMallocFromPoolAsync(ptr, bytes > 0 ? bytes : 8, pp.pool, pp.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(pp.stream);
    return e;
}

void plan_free(void* ptr, cudaStream_t used_on)
{
    if (!ptr) return;
    if (!pools_enabled()) {
        cudaFree(ptr);   // waits for the device's outstanding work
        return;
    }
    // stream-ordered after the last work that used the memory: the pool can
    // hand it out again (or trim it) only once that stream has passed here
    cudaFreeAsync(ptr, used_on);
}
}  // namespace nms

static cudaError_t tmp_alloc(void** ptr, size_t bytes, cudaStream_t s)
{
    if (!pools_enabled()) return cudaMallocAsync(ptr, bytes > 0 ? bytes : 8, s);
    static std::mutex mu;
    static std::map<int, cudaMemPool_t> pools;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    cudaMemPool_t pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(mu);
        auto it = pools.find(dev);
        if (it == pools.end()) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            e = cudaMemPoolCreate(&pool, &props);
            if (e != cudaSuccess) return e;
            uint64_t keep = 1ull << 30;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
            pools[dev] = pool;
        } else {
            pool = it->second;
        }
    }
    return cudaMallocFromPoolAsync(ptr, bytes > 0 ? bytes : 8, pool, s);
}

namespace nms {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

nms_status cuda_fail(cudaError_t e, const char* what)
{
    set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e));
    if (e == cudaErrorMemoryAllocation) return NMS_ERR_OUT_OF_MEMORY;
    return NMS_ERR_CUDA;
}

static nms_status fail(nms_status st, const std::string& msg)
{
    set_error(msg);
    return st;
}

int device_sm_count()
{
    static thread_local int cached = 0;
    if (!cached) {
        int dev = 0, n = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
            cached = n;
        else
            cached = 148;
    }
    return cached;
}

// ------------------------------------------------------------ stage timer
cudaEvent_t StageTimer::get_event()
{
    if (!pool.empty()) {
        cudaEvent_t e = pool.back();
        pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void StageTimer::begin(int stage)
{
    if (!on) return;
    open_stage = stage;
    open_ev = get_event();
    cudaEventRecord(open_ev, stream);
}

void StageTimer::end(int stage, int n_launch)
{
    launches[stage] += n_launch;
    if (!on || open_stage != stage) return;
    cudaEvent_t b = get_event();
    cudaEventRecord(b, stream);
    pending.push_back({stage, open_ev, b});
    open_stage = -1;
    open_ev = nullptr;
    if (pending.size() > 4096) collect();
}

nms_status StageTimer::collect()
{
    for (auto& pe : pending) {
        cudaError_t e = cudaEventSynchronize(pe.b);
        if (e != cudaSuccess) return cuda_fail(e, "cudaEventSynchronize");
        float t = 0.f;
        cudaEventElapsedTime(&t, pe.a, pe.b);
        ms[pe.stage] += t;
        pool.push_back(pe.a);
        pool.push_back(pe.b);
    }
    pending.clear();
    return NMS_OK;
}

void StageTimer::release()
{
    for (auto& pe : pending) {
        cudaEventDestroy(pe.a);
        cudaEventDestroy(pe.b);
    }
    pending.clear();
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
    if (open_ev) cudaEventDestroy(open_ev);
    open_ev = nullptr;
}

// ------------------------------------------------------------ helpers
template <class T>
static nms_status dalloc(T** p, size_t count, const char* what)
{
    *p = nullptr;
    if (count == 0) return NMS_OK;
    cudaError_t e = plan_malloc(p, count * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? NMS_ERR_OUT_OF_MEMORY : NMS_ERR_CUDA,
                    std::string("device allocation failed for ") + what + ": " + cudaGetErrorString(e));
    }
    return NMS_OK;
}

static void dfree(void* p, cudaStream_t s) { plan_free(p, s); }

static void free_plan(nms_plan_s* p)
{
    if (!p) return;
    cudaStreamSynchronize(p->stream);   // nothing of the plan may still run

    void* bufs[] = {p->d_pos, p->d_vol, p->d_nuc, p->d_mag, p->d_cen_cell, p->d_qy, p->d_qz, p->d_hy,
                    p->d_hz, p->d_qa, p->d_qturn, p->d_cpos, p->d_w64, p->d_cw, p->d_yz, p->d_F,
                    p->d_Ftot, p->d_Fpart, p->d_Gtot, p->d_Gdil, p->d_err, p->d_tab, p->d_wscale};
    for (void* b : bufs) dfree(b, p->stream);
    tc_release(*p);
    if (p->d_cposl && p->d_cposl != p->d_cpos) dfree(p->d_cposl, p->stream);
    if (p->d_yzl && p->d_yzl != p->d_yz) dfree(p->d_yzl, p->stream);
    dfree(p->d_bin_of, p->stream);
    dfree(p->d_Iobj, p->stream);
    cudaStreamSynchronize(p->stream);   // the frees are done before the stream can go away
    p->timer.release();
    delete p;
}

// Per-pixel q-grid arrays, computed on the device (launch_grid) on the
// plan's stream; a list grid is checked here and copied up first.
static nms_status build_grid(Plan& p, const nms_qgrid& g)
{
    int64_t np = 0;
    if (g.kind == NMS_QGRID_CARTESIAN || g.kind == NMS_QGRID_POLAR) {
        if (g.n0 < 1 || g.n1 < 1) return fail(NMS_ERR_INVALID_ARG, "grid: n0 and n1 must be >= 1");
        if (!std::isfinite(g.lo0) || !std::isfinite(g.hi0) ||
            (g.kind == NMS_QGRID_CARTESIAN && (!std::isfinite(g.lo1) || !std::isfinite(g.hi1))))
            return fail(NMS_ERR_INVALID_ARG, "grid: non-finite q");
        np = (int64_t)g.n0 * g.n1;
    } else if (g.kind == NMS_QGRID_LIST) {
        if (g.n0 < 1 || !g.qlist) return fail(NMS_ERR_INVALID_ARG, "grid: LIST needs n0 >= 1 and qlist");
        np = g.n0;
        for (int64_t i = 0; i < 2 * np; ++i)
            if (!std::isfinite(g.qlist[i])) return fail(NMS_ERR_INVALID_ARG, "grid: non-finite q");
    } else {
        return fail(NMS_ERR_INVALID_ARG, "grid: unknown kind");
    }
    p.npix = np;
    nms_status st;
    if ((st = dalloc(&p.d_qy, np, "qy")) || (st = dalloc(&p.d_qz, np, "qz")) || (st = dalloc(&p.d_hy, np, "hy")) ||
        (st = dalloc(&p.d_hz, np, "hz")) || (st = dalloc(&p.d_qa, np, "qa")) || (st = dalloc(&p.d_qturn, np, "qturn")))
        return st;
    double* d_list = nullptr;
    if (g.kind == NMS_QGRID_LIST) {
        if ((st = dalloc(&d_list, 2 * np, "qlist"))) return st;
        NMS_CUDA_TRY(cudaMemcpyAsync(d_list, g.qlist, 2 * np * sizeof(double), cudaMemcpyHostToDevice, p.stream));
    }
    NMS_CUDA_TRY(launch_grid(g, np, d_list, p.d_qy, p.d_qz, p.d_hy, p.d_hz, p.d_qa, p.d_qturn, p.stream));
    if (d_list) {
        NMS_CUDA_TRY(cudaStreamSynchronize(p.stream));   // the copy from the caller's buffer has completed
        dfree(d_list, p.stream);
    }
    return NMS_OK;
}

static int direct_splits(const Plan& p, int64_t ncell)
{
    const int64_t per_block = 256 * 2;
    int64_t pix_blocks = (p.npix + per_block - 1) / per_block;
    int64_t target = (int64_t)device_sm_count() * 8;
    int64_t s = (target + pix_blocks - 1) / pix_blocks;
    int64_t by_cells = std::max<int64_t>(1, ncell / 2048);
    s = std::min(s, by_cells);
    s = std::min(s, p.fpart_splits);
    return (int)std::max<int64_t>(1, s);
}

// Direct sum of cells [c0, c1) with positions cpos into out [4][npix][2].
nms_status direct_sum_range(Plan& p, const float4* cpos, int64_t c0, int64_t c1, double* out)
{
    cudaStream_t s = p.stream;
    int splits = direct_splits(p, c1 - c0);
    p.timer.begin(ST_DIRECT);
    // the tensor path uses this as its reference (compensated) in the autotuner
    NMS_CUDA_TRY(launch_direct(p, cpos, c0, c1, p.path != NMS_PREC_FP32_NAIVE, splits, s));
    p.timer.end(ST_DIRECT, 1);
    p.timer.begin(ST_REDUCE);
    NMS_CUDA_TRY(launch_reduce_splits(p, splits, out, s));
    p.timer.end(ST_REDUCE, 1);
    return NMS_OK;
}

static nms_status check_device_error(Plan& p)
{
    int32_t herr = 0;
    NMS_CUDA_TRY(cudaMemcpyAsync(&herr, p.d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, p.stream));
    NMS_CUDA_TRY(cudaStreamSynchronize(p.stream));
    if (herr != 0) {
        cudaMemsetAsync(p.d_err, 0, sizeof(int32_t), p.stream);
        return fail(NMS_ERR_TIMEOUT, "a bounded device wait gave up (code " + std::to_string(herr) + ")");
    }
    return NMS_OK;
}

}  // namespace nms

using namespace nms;

extern "C" {

const char* nms_last_error(void) { return g_last_error.c_str(); }

const char* nms_version(void) { return "nms 0.1.0 sm_103a"; }

nms_status nms_options_default(nms_options* opt)
{
    if (!opt) return fail(NMS_ERR_INVALID_ARG, "opt is NULL");
    memset(opt, 0, sizeof(*opt));
    opt->precision = NMS_PREC_AUTO;
    opt->volume_V = 1.0;
    opt->b_H = 1.0;
    opt->P[2] = 1.0;
    return NMS_OK;
}

nms_status nms_plan_create(nms_plan_t* out, int64_t n_cells, const double* pos, const double* cell_vol,
                           const double* nuc, const double* mag, int64_t n_objects, const int64_t* object_offsets,
                           const double* object_centers, int32_t n_rot, const double* rot, const nms_qgrid* grid,
                           const nms_options* opt, void* cuda_stream)
{
    set_error("");
    if (!out) return fail(NMS_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_cells < 1 || !pos) return fail(NMS_ERR_INVALID_ARG, "need n_cells >= 1 and pos");
    if (n_objects < 1) return fail(NMS_ERR_INVALID_ARG, "n_objects must be >= 1");
    if (n_objects > 1 && !object_offsets) return fail(NMS_ERR_INVALID_ARG, "object_offsets required for K > 1");
    if (n_rot < 1) return fail(NMS_ERR_INVALID_ARG, "n_rot must be >= 1");
    if (!rot && n_rot != 1) return fail(NMS_ERR_INVALID_ARG, "rot == NULL requires n_rot == 1");
    if (!grid) return fail(NMS_ERR_INVALID_ARG, "grid is NULL");
    int dev_count = 0;
    cudaError_t ce = cudaGetDeviceCount(&dev_count);
    if (ce != cudaSuccess || dev_count < 1) {
        cudaGetLastError();
        return fail(NMS_ERR_CUDA, "no CUDA device available (libnms has no CPU fallback)");
    }

    nms_plan_s* p = new (std::nothrow) nms_plan_s();
    if (!p) return fail(NMS_ERR_OUT_OF_MEMORY, "host allocation failed");
    if (opt) p->opt = *opt; else nms_options_default(&p->opt);
    p->grid = *grid;
    p->grid.qlist = nullptr;
    p->stream = (cudaStream_t)cuda_stream;
    p->timer.stream = p->stream;
    p->timer.on = p->opt.timing != 0;
    p->n_cells = n_cells;
    p->n_objects = n_objects;
    p->n_rot = n_rot;
    p->n_sets = p->opt.n_sets > 0 ? p->opt.n_sets : 1;
    p->V = p->opt.volume_V > 0 ? p->opt.volume_V : 1.0;
    p->bH = p->opt.b_H != 0 ? p->opt.b_H : 1.0;
    double pn = sqrt(p->opt.P[0] * p->opt.P[0] + p->opt.P[1] * p->opt.P[1] + p->opt.P[2] * p->opt.P[2]);
    if (pn == 0.0) { p->P[0] = 0; p->P[1] = 0; p->P[2] = 1; }
    else for (int a = 0; a < 3; ++a) p->P[a] = p->opt.P[a] / pn;
    p->has_nuc = nuc != nullptr;
    p->has_mag = mag != nullptr;
    p->has_centers = object_centers != nullptr;

    auto bail = [&](nms_status st) { free_plan(p); return st; };

    // precision / path
    int prec = p->opt.precision;
    if (prec < NMS_PREC_AUTO || prec > NMS_PREC_FP32_NAIVE) return bail(fail(NMS_ERR_INVALID_ARG, "bad precision"));
    if (prec == NMS_PREC_TC_F16X3 && grid->kind == NMS_QGRID_LIST)
        return bail(fail(NMS_ERR_INVALID_ARG, "the tensor-core path needs a CARTESIAN or POLAR grid"));
    // auto: the tensor path on CARTESIAN and POLAR grids (there one GEMM per
    // ray), the direct sum on point lists
    if (prec == NMS_PREC_AUTO) prec = grid->kind == NMS_QGRID_LIST ? NMS_PREC_FP32_DIRECT : NMS_PREC_TC_F16X3;
    p->path = prec;
    if (p->n_sets > 4096 || (prec == NMS_PREC_TC_F16X3 && p->n_sets > 32))
        return bail(fail(NMS_ERR_INVALID_ARG, "n_sets above 32 (tensor path) or 4096"));

    // offsets
    p->h_off.resize(n_objects + 1);
    if (object_offsets) {
        for (int64_t k = 0; k <= n_objects; ++k) p->h_off[k] = object_offsets[k];
        if (p->h_off[0] != 0 || p->h_off[n_objects] != n_cells)
            return bail(fail(NMS_ERR_INVALID_ARG, "object_offsets must start at 0 and end at n_cells"));
        for (int64_t k = 0; k < n_objects; ++k)
            if (p->h_off[k + 1] < p->h_off[k]) return bail(fail(NMS_ERR_INVALID_ARG, "object_offsets not monotone"));
    } else {
        p->h_off[0] = 0;
        p->h_off[1] = n_cells;
    }
    // rotations
    p->h_rot.resize((size_t)9 * n_rot);
    for (int32_t r = 0; r < n_rot; ++r)
        for (int a = 0; a < 9; ++a) p->h_rot[9 * r + a] = rot ? rot[9 * r + a] : (a % 4 == 0 ? 1.0 : 0.0);
    for (double v : p->h_rot)
        if (!std::isfinite(v)) return bail(fail(NMS_ERR_INVALID_ARG, "non-finite rotation entry"));
    if (object_centers) p->h_cen.assign(object_centers, object_centers + 3 * n_objects);

    nms_status st;
    if ((st = build_grid(*p, *grid))) return bail(st);

    // inputs to the device
    const int64_t n = n_cells;
    const int64_t nS = p->n_sets;
    if ((st = dalloc(&p->d_pos, 3 * n, "pos"))) return bail(st);
    // inputs go up on the plan's stream (asynchronous from pinned memory);
    // the stream is synchronised below, before the call returns
    NMS_CUDA_TRY(cudaMemcpyAsync(p->d_pos, pos, 3 * n * 8, cudaMemcpyHostToDevice, p->stream));
    if (cell_vol) {
        if ((st = dalloc(&p->d_vol, n, "vol"))) return bail(st);
        NMS_CUDA_TRY(cudaMemcpyAsync(p->d_vol, cell_vol, n * 8, cudaMemcpyHostToDevice, p->stream));
    }
    if (nuc) {
        if ((st = dalloc(&p->d_nuc, nS * n, "nuc"))) return bail(st);
        NMS_CUDA_TRY(cudaMemcpyAsync(p->d_nuc, nuc, nS * n * 8, cudaMemcpyHostToDevice, p->stream));
    }
    if (mag) {
        if ((st = dalloc(&p->d_mag, 3 * nS * n, "mag"))) return bail(st);
        NMS_CUDA_TRY(cudaMemcpyAsync(p->d_mag, mag, 3 * nS * n * 8, cudaMemcpyHostToDevice, p->stream));
    }
    if (object_centers) {
        std::vector<double> cc((size_t)3 * n);
        for (int64_t k = 0; k < n_objects; ++k)
            for (int64_t j = p->h_off[k]; j < p->h_off[k + 1]; ++j)
                for (int a = 0; a < 3; ++a) cc[3 * j + a] = object_centers[3 * k + a];
        if ((st = dalloc(&p->d_cen_cell, 3 * n, "centres"))) return bail(st);
        NMS_CUDA_TRY(cudaMemcpy(p->d_cen_cell, cc.data(), 3 * n * 8, cudaMemcpyHostToDevice));
    }
    // per-rotation work arrays
    if ((st = dalloc(&p->d_cpos, n, "cpos")) || (st = dalloc(&p->d_cw, n, "cw"))) return bail(st);
    bool need_local = p->opt.want_dilute && n_objects > 1 && object_centers;
    if (need_local) {
        if ((st = dalloc(&p->d_cposl, n, "cposl"))) return bail(st);
    } else {
        p->d_cposl = p->d_cpos;
    }
    const int64_t np = p->npix;
    p->fpart_splits = std::max<int64_t>(1, std::min<int64_t>(64, (int64_t)(256ll << 20) / (64 * np)));
    if ((st = dalloc(&p->d_F, nS * 8 * np, "F")) || (st = dalloc(&p->d_Fpart, 8 * np * p->fpart_splits, "Fpart")) ||
        (st = dalloc(&p->d_Gtot, nS * 16 * np, "Gtot")) || (st = dalloc(&p->d_err, 1, "err")))
        return bail(st);
    if (p->opt.want_dilute) {
        if ((st = dalloc(&p->d_Gdil, nS * 16 * np, "Gdil"))) return bail(st);
    }
    if (n_objects > 1 && p->opt.want_dilute) {
        if ((st = dalloc(&p->d_Ftot, nS * 8 * np, "Ftot"))) return bail(st);
    }
    NMS_CUDA_TRY(cudaMemset(p->d_err, 0, sizeof(int32_t)));
    // max_j V_j |N_j| and max_j V_j |M_j| over all weight sets, on the device
    NMS_CUDA_TRY(launch_weight_max(*p, p->h_wmax, p->stream));
    p->max_sum_cells = n_cells;
    if (n_objects > 1 && p->opt.want_dilute) {
        p->max_sum_cells = 0;
        for (int64_t k = 0; k < n_objects; ++k) p->max_sum_cells = std::max(p->max_sum_cells, p->h_off[k + 1] - p->h_off[k]);
    }
    if (p->path == NMS_PREC_TC_F16X3) {
        if ((st = tc_setup(*p))) return bail(st);
    }
    *out = p;
    return NMS_OK;
}

nms_status nms_amplitudes(nms_plan_t plan)
{
    set_error("");
    if (!plan) return fail(NMS_ERR_INVALID_ARG, "plan is NULL");
    Plan& p = *plan;
    cudaStream_t s = p.stream;
    const int64_t np = p.npix;
    const int64_t nS = p.n_sets;
    NMS_CUDA_TRY(cudaMemsetAsync(p.d_Gtot, 0, nS * 16 * np * 8, s));
    if (p.d_Gdil) NMS_CUDA_TRY(cudaMemsetAsync(p.d_Gdil, 0, nS * 16 * np * 8, s));
    if (p.d_Iobj)
        NMS_CUDA_TRY(cudaMemsetAsync(p.d_Iobj, 0, (size_t)tc_object_count(p) * p.oiq_nbins * sizeof(double), s));
    if (p.path == NMS_PREC_TC_F16X3) {
        nms_status st = tc_amplitudes(p, s);
        if (st) return st;
        p.rot_done = p.n_rot;
        p.have_G = true;
        return NMS_OK;
    }
    const bool objects = p.n_objects > 1 && p.opt.want_dilute;
    // loop mode on the direct path: one pass per weight set
    for (int32_t r = 0; r < p.n_rot; ++r)
        for (int32_t set = 0; set < p.n_sets; ++set) {
            const double* R = &p.h_rot[9 * r];
            double* F = p.d_F + (size_t)set * 8 * np;
            double* Gt = p.d_Gtot + (size_t)set * 16 * np;
            double* Gd = p.d_Gdil ? p.d_Gdil + (size_t)set * 16 * np : nullptr;
            p.timer.begin(ST_PREP);
            NMS_CUDA_TRY(launch_prep(p, R, s, set));
            p.timer.end(ST_PREP, 1);
            if (!objects) {
                nms_status st = direct_sum_range(p, p.d_cpos, 0, p.n_cells, F);
                if (st) return st;
                p.timer.begin(ST_GACC);
                NMS_CUDA_TRY(launch_gacc(p, F, Gt, s));
                if (Gd) NMS_CUDA_TRY(launch_gacc(p, F, Gd, s));
                p.timer.end(ST_GACC, Gd ? 2 : 1);
            } else {
                // per object: local amplitude F_k -> G_dil, and shifted into F_tot
                double* Ft = p.d_Ftot + (size_t)set * 8 * np;
                NMS_CUDA_TRY(cudaMemsetAsync(Ft, 0, 8 * np * 8, s));
                for (int64_t k = 0; k < p.n_objects; ++k) {
                    int64_t a = p.h_off[k], b = p.h_off[k + 1];
                    if (b == a) continue;
                    nms_status st = direct_sum_range(p, p.d_cposl, a, b, F);
                    if (st) return st;
                    double cy = 0.0, cz = 0.0;
                    if (!p.h_cen.empty()) {
                        const double* c = &p.h_cen[3 * k];
                        cy = R[3] * c[0] + R[4] * c[1] + R[5] * c[2];
                        cz = R[6] * c[0] + R[7] * c[1] + R[8] * c[2];
                    }
                    p.timer.begin(ST_GACC);
                    NMS_CUDA_TRY(launch_gacc(p, F, Gd, s));
                    NMS_CUDA_TRY(launch_shift_add(p, F, cy, cz, Ft, s));
                    p.timer.end(ST_GACC, 2);
                }
                p.timer.begin(ST_GACC);
                NMS_CUDA_TRY(launch_gacc(p, Ft, Gt, s));
                p.timer.end(ST_GACC, 1);
            }
        }
    p.rot_done = p.n_rot;
    p.have_G = true;
    return NMS_OK;
}

nms_status nms_get_amplitudes(nms_plan_t plan, double* out, int32_t out_is_device)
{
    set_error("");
    if (!plan || !out) return fail(NMS_ERR_INVALID_ARG, "plan/out is NULL");
    Plan& p = *plan;
    if (!p.have_G) return fail(NMS_ERR_BAD_STATE, "nms_amplitudes has not run");
    nms_status st = check_device_error(p);
    if (st) return st;
    const double* src = ((p.n_objects > 1 && p.opt.want_dilute) ? p.d_Ftot : p.d_F) + (size_t)p.sel_set * 8 * p.npix;
    NMS_CUDA_TRY(cudaMemcpyAsync(out, src, 8 * p.npix * 8,
                                 out_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, p.stream));
    NMS_CUDA_TRY(cudaStreamSynchronize(p.stream));
    return NMS_OK;
}

nms_status nms_response(nms_plan_t plan, int32_t id, int32_t part, double* out, int32_t out_is_device)
{
    set_error("");
    if (!plan || !out) return fail(NMS_ERR_INVALID_ARG, "plan/out is NULL");
    Plan& p = *plan;
    if (id < 0 || id >= NMS_RESP_COUNT) return fail(NMS_ERR_INVALID_ARG, "response id out of range");
    if (part < NMS_PART_TOTAL || part > NMS_PART_INTERFERENCE) return fail(NMS_ERR_INVALID_ARG, "bad part");
    if (!p.have_G) return fail(NMS_ERR_BAD_STATE, "nms_amplitudes has not run");
    if (part != NMS_PART_TOTAL && !p.d_Gdil) return fail(NMS_ERR_UNSUPPORTED, "dilute part needs want_dilute");
    const size_t gs = (size_t)p.sel_set * 16 * p.npix;   // the selected weight set's G
    const double* Ga = (part == NMS_PART_DILUTE ? p.d_Gdil : p.d_Gtot) + gs;
    const double* Gb = part == NMS_PART_INTERFERENCE ? p.d_Gdil + gs : nullptr;
    double norm = 1.0 / (double)(p.rot_done > 0 ? p.rot_done : 1);
    double* dst = out;
    if (!out_is_device) {
        NMS_CUDA_TRY(tmp_alloc((void**)&dst, p.npix * 8, p.stream));
    }
    cudaError_t e = launch_response(p, id, Ga, Gb, norm, dst, p.stream);
    if (e == cudaSuccess && !out_is_device)
        e = cudaMemcpyAsync(out, dst, p.npix * 8, cudaMemcpyDeviceToHost, p.stream);
    if (!out_is_device) cudaFreeAsync(dst, p.stream);
    if (e != cudaSuccess) return cuda_fail(e, "response");
    return check_device_error(p);
}

// Device staging of results: kernels write device buffers; results the
// caller wants on the host are copied back at the end of the call.
namespace {
struct Staged {
    void* user = nullptr;   // caller's buffer (may be NULL: not wanted)
    void* dev = nullptr;    // what the kernels write
    size_t bytes = 0;
    bool copy_back = false;
};

cudaError_t stage(Staged& st, void* user, size_t bytes, bool user_is_device, cudaStream_t s)
{
    st.user = user;
    st.bytes = bytes;
    if (user && user_is_device) {
        st.dev = user;
        return cudaSuccess;
    }
    st.copy_back = user != nullptr;
    return tmp_alloc(&st.dev, bytes > 0 ? bytes : 8, s);
}

cudaError_t unstage(Staged& st, cudaStream_t s, cudaError_t e)
{
    if (e == cudaSuccess && st.copy_back) e = cudaMemcpyAsync(st.user, st.dev, st.bytes, cudaMemcpyDeviceToHost, s);
    if (st.dev && st.dev != st.user) cudaFreeAsync(st.dev, s);
    st.dev = nullptr;
    return e;
}

// image on the device for the duration of a call
cudaError_t device_image(const Plan& p, const double* img, bool is_device, const double** d_img, double** tmp)
{
    *tmp = nullptr;
    *d_img = img;
    if (is_device) return cudaSuccess;
    cudaError_t e = tmp_alloc((void**)tmp, p.npix * 8, p.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(*tmp, img, p.npix * 8, cudaMemcpyHostToDevice, p.stream);
    *d_img = *tmp;
    return e;
}

nms_status check_edges(int nbins, const double* edges)
{
    if (nbins < 1 || !edges) return fail(NMS_ERR_INVALID_ARG, "need nbins >= 1 and bin_edges");
    for (int b = 0; b < nbins; ++b)
        if (!(edges[b + 1] > edges[b])) return fail(NMS_ERR_INVALID_ARG, "bin_edges not increasing");
    return NMS_OK;
}
}  // namespace

nms_status nms_azimuthal_average(nms_plan_t plan, const double* img, int32_t img_is_device, int32_t nbins,
                                 const double* bin_edges, double* Iq, int64_t* counts, double* qmean,
                                 int32_t out_is_device)
{
    set_error("");
    if (!plan || !img || !Iq || !counts) return fail(NMS_ERR_INVALID_ARG, "NULL argument");
    Plan& p = *plan;
    cudaStream_t s = p.stream;
    const bool polar = p.grid.kind == NMS_QGRID_POLAR;
    if (polar && nbins != p.grid.n0) return fail(NMS_ERR_INVALID_ARG, "POLAR grid: nbins must equal n0");
    if (!polar) {
        nms_status st = check_edges(nbins, bin_edges);
        if (st) return st;
        if (p.npix >= (1ll << 31)) return fail(NMS_ERR_UNSUPPORTED, "more than 2^31 pixels");
    }
    const double* d_img = nullptr;
    double* tmp_img = nullptr;
    NMS_CUDA_TRY(device_image(p, img, img_is_device != 0, &d_img, &tmp_img));
    Staged sI, sc, sq;
    cudaError_t e = stage(sI, Iq, (size_t)nbins * 8, out_is_device, s);
    if (e == cudaSuccess) e = stage(sc, counts, (size_t)nbins * 8, out_is_device, s);
    if (e == cudaSuccess) e = stage(sq, qmean, (size_t)nbins * 8, out_is_device, s);
    if (polar) {
        // the periodic trapezoid over theta (Eq. iqazi) is the mean over j
        if (e == cudaSuccess) e = launch_azimuthal_polar(p, d_img, (double*)sI.dev, s);
        if (e == cudaSuccess) e = launch_polar_nodes(p, (int64_t*)sc.dev, (double*)sq.dev, s);
    } else {
        // ring means: the k = 0 mode of the ring-binned angular spectrum
        double *d_e = nullptr, *Is0 = nullptr;
        void* work = nullptr;
        if (e == cudaSuccess) e = tmp_alloc((void**)&d_e, (nbins + 1) * 8, s);
        if (e == cudaSuccess) e = tmp_alloc((void**)&work, angspec_rings_work_bytes(p.npix, nbins, 0), s);
        if (e == cudaSuccess) e = tmp_alloc((void**)&Is0, (size_t)nbins * 8, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_e, bin_edges, (nbins + 1) * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = launch_angspec_rings(p, d_img, d_e, nbins, 0, work, (double*)sI.dev, Is0, (int64_t*)sc.dev,
                                     (double*)sq.dev, s);
        cudaFreeAsync(d_e, s);
        cudaFreeAsync(work, s);
        cudaFreeAsync(Is0, s);
    }
    e = unstage(sI, s, e);
    e = unstage(sc, s, e);
    e = unstage(sq, s, e);
    if (tmp_img) cudaFreeAsync(tmp_img, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "azimuthal average");
    return NMS_OK;
}

nms_status nms_angular_spectrum(nms_plan_t plan, const double* img, int32_t img_is_device, int32_t kmax,
                                int32_t nbins, const double* bin_edges, double* Ic, double* Is, int64_t* counts,
                                double* qmean, double* Ac, double* As, int32_t out_is_device)
{
    set_error("");
    if (!plan || !img || !Ic || !Is) return fail(NMS_ERR_INVALID_ARG, "NULL argument");
    if (kmax < 0 || kmax > 1023) return fail(NMS_ERR_INVALID_ARG, "need 0 <= kmax <= 1023");
    Plan& p = *plan;
    if (p.npix >= (1ll << 31)) return fail(NMS_ERR_UNSUPPORTED, "more than 2^31 pixels");
    cudaStream_t s = p.stream;
    const bool polar = p.grid.kind == NMS_QGRID_POLAR;
    if (polar) {
        if (nbins != p.grid.n0) return fail(NMS_ERR_INVALID_ARG, "POLAR grid: nbins must equal n0");
        if ((size_t)3 * p.grid.n1 * 8 > (200u << 10))
            return fail(NMS_ERR_UNSUPPORTED, "POLAR grid: n_theta above 8533");
    } else {
        nms_status st = check_edges(nbins, bin_edges);
        if (st) return st;
    }
    const int K = kmax + 1;
    const double* d_img = nullptr;
    double* tmp_img = nullptr;
    NMS_CUDA_TRY(device_image(p, img, img_is_device != 0, &d_img, &tmp_img));
    Staged sIc, sIs, sc, sq, sAc, sAs;
    const bool od = out_is_device != 0;
    cudaError_t e = stage(sIc, Ic, (size_t)K * nbins * 8, od, s);
    if (e == cudaSuccess) e = stage(sIs, Is, (size_t)K * nbins * 8, od, s);
    if (e == cudaSuccess) e = stage(sc, counts, (size_t)nbins * 8, od, s);
    if (e == cudaSuccess) e = stage(sq, qmean, (size_t)nbins * 8, od, s);
    if (e == cudaSuccess) e = stage(sAc, Ac, (size_t)K * 8, od, s);
    if (e == cudaSuccess) e = stage(sAs, As, (size_t)K * 8, od, s);
    if (polar) {
        if (e == cudaSuccess) e = launch_angspec_polar(p, d_img, kmax, (double*)sIc.dev, (double*)sIs.dev, s);
        if (e == cudaSuccess) e = launch_polar_nodes(p, (int64_t*)sc.dev, (double*)sq.dev, s);
    } else {
        double* d_e = nullptr;
        void* work = nullptr;
        if (e == cudaSuccess) e = tmp_alloc((void**)&d_e, (nbins + 1) * 8, s);
        if (e == cudaSuccess) e = tmp_alloc((void**)&work, angspec_rings_work_bytes(p.npix, nbins, kmax), s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_e, bin_edges, (nbins + 1) * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = launch_angspec_rings(p, d_img, d_e, nbins, kmax, work, (double*)sIc.dev, (double*)sIs.dev,
                                     (int64_t*)sc.dev, (double*)sq.dev, s);
        cudaFreeAsync(d_e, s);
        cudaFreeAsync(work, s);
    }
    if (e == cudaSuccess)
        e = launch_modal_amplitudes((double*)sIc.dev, (double*)sIs.dev, nbins, kmax, (double*)sAc.dev,
                                    (double*)sAs.dev, s);
    e = unstage(sIc, s, e);
    e = unstage(sIs, s, e);
    e = unstage(sc, s, e);
    e = unstage(sq, s, e);
    e = unstage(sAc, s, e);
    e = unstage(sAs, s, e);
    if (tmp_img) cudaFreeAsync(tmp_img, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "angular spectrum");
    return NMS_OK;
}

nms_status nms_correlation_2d(nms_plan_t plan, const double* img, int32_t img_is_device, int32_t n_rho,
                              const double* rho, int32_t n_alpha, const double* alpha, double* C, double* scale,
                              int32_t out_is_device)
{
    set_error("");
    if (!plan || !img || !C || !rho || !alpha) return fail(NMS_ERR_INVALID_ARG, "NULL argument");
    if (n_rho < 1 || n_alpha < 1 || (int64_t)n_rho * n_alpha > (1 << 24))
        return fail(NMS_ERR_INVALID_ARG, "need n_rho, n_alpha >= 1 and n_rho * n_alpha <= 2^24");
    Plan& p = *plan;
    if (p.grid.kind == NMS_QGRID_LIST) return fail(NMS_ERR_UNSUPPORTED, "LIST grid has no quadrature weights");
    cudaStream_t s = p.stream;
    const int n_out = n_rho * n_alpha;
    const int splits = corr2d_splits(p.npix, n_out);
    const double* d_img = nullptr;
    double* tmp_img = nullptr;
    NMS_CUDA_TRY(device_image(p, img, img_is_device != 0, &d_img, &tmp_img));
    Staged sC, sS;
    cudaError_t e = stage(sC, C, (size_t)n_out * 16, out_is_device != 0, s);
    if (e == cudaSuccess) e = stage(sS, scale, 8, out_is_device != 0, s);
    double *d_rho = nullptr, *d_alpha = nullptr;
    float* d_w = nullptr;
    float4* d_pts = nullptr;
    double2* d_part = nullptr;
    if (e == cudaSuccess) e = tmp_alloc((void**)&d_rho, (size_t)n_rho * 8, s);
    if (e == cudaSuccess) e = tmp_alloc((void**)&d_alpha, (size_t)n_alpha * 8, s);
    if (e == cudaSuccess) e = tmp_alloc((void**)&d_w, (size_t)p.npix * 4, s);
    if (e == cudaSuccess) e = tmp_alloc((void**)&d_pts, (size_t)n_out * 16, s);
    if (e == cudaSuccess) e = tmp_alloc((void**)&d_part, (size_t)splits * n_out * 16, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_rho, rho, (size_t)n_rho * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_alpha, alpha, (size_t)n_alpha * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(sS.dev, 0, 8, s);
    if (e == cudaSuccess)
        e = launch_corr2d(p, d_img, d_rho, n_rho, d_alpha, n_alpha, d_w, (double*)sS.dev, d_pts, d_part, splits,
                          (double2*)sC.dev, s);
    for (void* x : {(void*)d_rho, (void*)d_alpha, (void*)d_w, (void*)d_pts, (void*)d_part})
        if (x) cudaFreeAsync(x, s);
    e = unstage(sC, s, e);
    e = unstage(sS, s, e);
    if (tmp_img) cudaFreeAsync(tmp_img, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "2D correlation");
    return NMS_OK;
}

nms_status nms_correlation(int32_t nq, const double* q, const double* Iq, int32_t nr, const double* r,
                           double prefactor, double* c_r, double* p_r, int32_t is_device, void* cuda_stream)
{
    set_error("");
    if (nq < 0 || nr < 0 || (nq > 0 && (!q || !Iq)) || (nr > 0 && !r)) return fail(NMS_ERR_INVALID_ARG, "bad sizes or NULL");
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
        cudaGetLastError();
        return fail(NMS_ERR_CUDA, "no CUDA device available (libnms has no CPU fallback)");
    }
    if (nr == 0) return NMS_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    double pref = prefactor != 0.0 ? prefactor : 1.0 / (2.0 * M_PI * M_PI);
    int nqa = std::max(nq, 1);
    double *dq = nullptr, *dI = nullptr, *dr = nullptr, *dc = nullptr, *dp = nullptr, *sq = nullptr, *sf = nullptr;
    int* sn = nullptr;
    NMS_CUDA_TRY(tmp_alloc((void**)&sq, nqa * 8, s));
    NMS_CUDA_TRY(tmp_alloc((void**)&sf, nqa * 8, s));
    NMS_CUDA_TRY(tmp_alloc((void**)&sn, sizeof(int), s));
    if (is_device) {
        dq = (double*)q; dI = (double*)Iq; dr = (double*)r; dc = c_r; dp = p_r;
    } else {
        NMS_CUDA_TRY(tmp_alloc((void**)&dq, nqa * 8, s));
        NMS_CUDA_TRY(tmp_alloc((void**)&dI, nqa * 8, s));
        NMS_CUDA_TRY(tmp_alloc((void**)&dr, nr * 8, s));
        NMS_CUDA_TRY(tmp_alloc((void**)&dc, nr * 8, s));
        NMS_CUDA_TRY(tmp_alloc((void**)&dp, nr * 8, s));
        if (nq) NMS_CUDA_TRY(cudaMemcpyAsync(dq, q, nq * 8, cudaMemcpyHostToDevice, s));
        if (nq) NMS_CUDA_TRY(cudaMemcpyAsync(dI, Iq, nq * 8, cudaMemcpyHostToDevice, s));
        NMS_CUDA_TRY(cudaMemcpyAsync(dr, r, nr * 8, cudaMemcpyHostToDevice, s));
    }
    cudaError_t e = launch_correlation(nq, dq, dI, nr, dr, pref, dc, dp, sq, sf, sn, s);
    if (e == cudaSuccess && !is_device) {
        if (c_r) e = cudaMemcpyAsync(c_r, dc, nr * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && p_r) e = cudaMemcpyAsync(p_r, dp, nr * 8, cudaMemcpyDeviceToHost, s);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFreeAsync(sq, s);
    cudaFreeAsync(sf, s);
    cudaFreeAsync(sn, s);
    if (!is_device) {
        cudaFreeAsync(dq, s);
        cudaFreeAsync(dI, s);
        cudaFreeAsync(dr, s);
        cudaFreeAsync(dc, s);
        cudaFreeAsync(dp, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "correlation");
    return NMS_OK;
}

nms_status nms_plan_object_iq(nms_plan_t plan, int32_t response_id, int32_t nbins, const double* bin_edges)
{
    set_error("");
    if (!plan) return fail(NMS_ERR_INVALID_ARG, "plan is NULL");
    Plan& p = *plan;
    if (p.path != NMS_PREC_TC_F16X3 || p.grid.kind != NMS_QGRID_CARTESIAN)
        return fail(NMS_ERR_UNSUPPORTED, "per-object averages need the tensor-core path on a CARTESIAN grid");
    if (p.n_sets > 1) return fail(NMS_ERR_UNSUPPORTED, "per-object averages take one weight set");
    if (!(response_id == NMS_RESP_N || response_id == NMS_RESP_M || response_id == NMS_RESP_P ||
          response_id == NMS_RESP_SF || response_id == NMS_RESP_UNPOL))
        return fail(NMS_ERR_UNSUPPORTED, "per-object averages support N, M, P, SF and UNPOL");
    if (nbins < 1 || nbins > 8192 || !bin_edges) return fail(NMS_ERR_INVALID_ARG, "need 1 <= nbins <= 8192 and bin_edges");
    for (int b = 0; b < nbins; ++b)
        if (!(bin_edges[b + 1] > bin_edges[b])) return fail(NMS_ERR_INVALID_ARG, "bin_edges not increasing");
    std::vector<int32_t> bin_of(p.npix);
    std::vector<double> h_qa(p.npix);
    NMS_CUDA_TRY(cudaMemcpyAsync(h_qa.data(), p.d_qa, p.npix * sizeof(double), cudaMemcpyDeviceToHost, p.stream));
    NMS_CUDA_TRY(cudaStreamSynchronize(p.stream));
    p.oiq_counts.assign(nbins, 0);
    p.oiq_qmean.assign(nbins, 0.0);
    for (int64_t i = 0; i < p.npix; ++i) {
        const double x = h_qa[i];
        int b = -1;
        if (x >= bin_edges[0] && x < bin_edges[nbins])
            b = (int)(std::upper_bound(bin_edges, bin_edges + nbins + 1, x) - bin_edges) - 1;
        bin_of[i] = b;
        if (b >= 0) {
            p.oiq_counts[b]++;
            p.oiq_qmean[b] += x;
        }
    }
    for (int b = 0; b < nbins; ++b) p.oiq_qmean[b] = p.oiq_counts[b] ? p.oiq_qmean[b] / p.oiq_counts[b] : NAN;
    cudaStreamSynchronize(p.stream);   // earlier amplitude calls may still use the old bins
    dfree(p.d_bin_of, p.stream);
    dfree(p.d_Iobj, p.stream);
    p.d_bin_of = nullptr;
    p.d_Iobj = nullptr;
    nms_status st;
    if ((st = dalloc(&p.d_bin_of, p.npix, "bin_of")) ||
        (st = dalloc(&p.d_Iobj, (size_t)tc_object_count(p) * nbins, "object I(q)")))
        return st;
    NMS_CUDA_TRY(cudaMemcpy(p.d_bin_of, bin_of.data(), p.npix * sizeof(int32_t), cudaMemcpyHostToDevice));
    p.oiq_id = response_id;
    p.oiq_nbins = nbins;
    p.have_G = false;
    return NMS_OK;
}

nms_status nms_get_object_iq(nms_plan_t plan, double* Iq, int64_t* counts, double* qmean, int32_t out_is_device)
{
    set_error("");
    if (!plan || !Iq) return fail(NMS_ERR_INVALID_ARG, "plan/Iq is NULL");
    Plan& p = *plan;
    if (p.oiq_id < 0) return fail(NMS_ERR_BAD_STATE, "nms_plan_object_iq has not been called");
    if (!p.have_G) return fail(NMS_ERR_BAD_STATE, "nms_amplitudes has not run");
    nms_status st = check_device_error(p);
    if (st) return st;
    const int64_t K = tc_object_count(p);
    const int nb = p.oiq_nbins;
    std::vector<double> h((size_t)K * nb);
    NMS_CUDA_TRY(cudaMemcpyAsync(h.data(), p.d_Iobj, h.size() * sizeof(double), cudaMemcpyDeviceToHost, p.stream));
    NMS_CUDA_TRY(cudaStreamSynchronize(p.stream));
    for (int64_t k = 0; k < K; ++k)
        for (int b = 0; b < nb; ++b) {
            const int64_t c = p.oiq_counts[b];
            h[(size_t)k * nb + b] = c ? h[(size_t)k * nb + b] / ((double)c * p.rot_done) : NAN;
        }
    cudaMemcpyKind kind = out_is_device ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    NMS_CUDA_TRY(cudaMemcpyAsync(Iq, h.data(), h.size() * sizeof(double), kind, p.stream));
    if (counts) NMS_CUDA_TRY(cudaMemcpyAsync(counts, p.oiq_counts.data(), nb * sizeof(int64_t), kind, p.stream));
    if (qmean) NMS_CUDA_TRY(cudaMemcpyAsync(qmean, p.oiq_qmean.data(), nb * sizeof(double), kind, p.stream));
    NMS_CUDA_TRY(cudaStreamSynchronize(p.stream));
    return NMS_OK;
}

nms_status nms_plan_stage_ms(nms_plan_t plan, double ms[8], int64_t launches[8], int32_t reset)
{
    set_error("");
    if (!plan) return fail(NMS_ERR_INVALID_ARG, "plan is NULL");
    Plan& p = *plan;
    nms_status st = p.timer.collect();
    if (st) return st;
    for (int i = 0; i < ST_COUNT; ++i) {
        if (ms) ms[i] = p.timer.ms[i];
        if (launches) launches[i] = p.timer.launches[i];
    }
    if (reset) {
        for (int i = 0; i < ST_COUNT; ++i) { p.timer.ms[i] = 0; p.timer.launches[i] = 0; }
    }
    return NMS_OK;
}

nms_status nms_plan_info(nms_plan_t plan, int32_t* precision, int32_t* kc_cells, int32_t* items_per_sm,
                         int32_t* gemm_form, int32_t* mirror_y, int32_t* mirror_z)
{
    set_error("");
    if (!plan) return fail(NMS_ERR_INVALID_ARG, "plan is NULL");
    if (precision) *precision = plan->path;
    if (kc_cells) *kc_cells = tc_tuned_kc_cells(*plan);
    if (items_per_sm) *items_per_sm = tc_tuned_items_per_sm(*plan);
    int32_t form = -1, my = 0, mz = 0;
    tc_form_info(*plan, &form, &my, &mz);
    if (gemm_form) *gemm_form = form;
    if (mirror_y) *mirror_y = my;
    if (mirror_z) *mirror_z = mz;
    return NMS_OK;
}

nms_status nms_select_set(nms_plan_t plan, int32_t set)
{
    set_error("");
    if (!plan) return fail(NMS_ERR_INVALID_ARG, "plan is NULL");
    if (set < 0 || set >= plan->n_sets) return fail(NMS_ERR_INVALID_ARG, "weight set out of range");
    plan->sel_set = set;
    return NMS_OK;
}

nms_status nms_selftest_bounded_wait(int64_t limit_us, void* cuda_stream)
{
    set_error("");
    if (limit_us < 1 || limit_us > 10000000) return fail(NMS_ERR_INVALID_ARG, "need 1 <= limit_us <= 1e7");
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
        cudaGetLastError();
        return fail(NMS_ERR_CUDA, "no CUDA device available (libnms has no CPU fallback)");
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int32_t* d_err = nullptr;
    NMS_CUDA_TRY(tmp_alloc((void**)&d_err, sizeof(int32_t), s));
    int32_t h_err = 0;
    cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int32_t), s);
    if (e == cudaSuccess) e = launch_selftest_wait((uint64_t)limit_us * 1000ull, d_err, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d_err, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test");
    if (h_err) return fail(NMS_ERR_TIMEOUT, "device wait gave up after the limit (expected)");
    return NMS_OK;
}

nms_status nms_selftest_sincos(int64_t n, const float* t, float* out, void* cuda_stream)
{
    set_error("");
    if (n < 0 || (n > 0 && (!t || !out))) return fail(NMS_ERR_INVALID_ARG, "need n >= 0 and host arrays t, out");
    if (n == 0) return NMS_OK;
    int dev_count = 0;
    if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count < 1) {
        cudaGetLastError();
        return fail(NMS_ERR_CUDA, "no CUDA device available (libnms has no CPU fallback)");
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    float* d = nullptr;
    NMS_CUDA_TRY(tmp_alloc((void**)&d, (size_t)n * 5 * sizeof(float), s));
    cudaError_t e = cudaMemcpyAsync(d, t, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_selftest_sincos(d, n, d + n, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d + n, (size_t)n * 4 * sizeof(float), cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "sincos self-test");
    return NMS_OK;
}

nms_status nms_plan_destroy(nms_plan_t plan)
{
    if (!plan) return NMS_OK;
    cudaStreamSynchronize(plan->stream);
    free_plan(plan);
    return NMS_OK;
}

}  // extern "C"
