// Host side of the tensor-core path: the work schedule and its launches.
//
// Every amplitude the plan needs is a "summand": the cells of one object (or
// all cells) under one rotation.  Summands are grouped into output batches
// (amplitude buffers F_b in HBM) and, within a batch, packed into table
// chunks that fit the table workspace (a large object is cut into several
// pieces that add into the same output).  For each chunk the phase tables
// are generated and one persistent GEMM launch walks a work list of
// (tile, k-range) items, longest first; a reduction adds the item tiles into
// F_b.  Batches then feed the Hermitian-product and shift kernels.
//
// The whole schedule is built and uploaded when the plan is created, so
// nms_amplitudes only launches kernels: no host synchronisation and no host
// to device copy happen inside it.
#include <cuda_runtime.h>
#include <math.h>

#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <cstring>
#include <functional>
#include <map>
#include <mutex>
#include <numeric>
#include <queue>
#include <string>
#include <utility>
#include <vector>

#include "nms_internal.h"

namespace nms {

// launchers in k_gemm.cu / k_batch.cu
cudaError_t tc_launch_tables(const float4* cpos, const float4* cw, int64_t wstride, int nch, const int64_t* kb_cell0,
                             const int32_t* kb_ncell, int64_t nkb, const float2* qy, int nyg, const float2* qz, int nzg,
                             int mtiles, int ntiles, const float wscale[4], void* tab, cudaStream_t s);
cudaError_t tc_launch_gemm(const void* tab, int64_t nkb, int mtiles, int ntiles, const void* items,
                           const int32_t* unit_item0, int grid, int kcb, double* P, double* F, int64_t lo_off,
                           const AxisMap& ax, int nch, const double scale[4], int32_t* err, uint64_t limit_ns, int mode,
                           cudaStream_t s);
cudaError_t tc_launch_gemm_rays(const float4* cpos, const float4* cw, const int64_t* kb_cell0, const int32_t* kb_ncell,
                                const RayProjection& pr, const float2* qy, int nyg, const float2* qz, int nzg,
                                const float wscale[4], const void* items, const int32_t* unit_item0, int grid, int kcb,
                                double* P, double* F, int64_t lo_off, const AxisMap& ax, int nch,
                                const double scale[4], int32_t* err, uint64_t limit_ns, cudaStream_t s);
cudaError_t tc_launch_reduce(const double* P, const void* reds, int n_red, const AxisMap& ax, int ntiles, int nch,
                             const double scale[4], double* F, int64_t lo_off, cudaStream_t s);
size_t tc_item_bytes();
size_t tc_red_bytes();
size_t tc_block_bytes();
int tc_block_cells();
float tc_operand_scale();
cudaError_t launch_prep_rot(const Plan& p, const RotMat& R, bool global, float4* cpos, float4* cw, int64_t wstride,
                            cudaStream_t s);
cudaError_t launch_prep_rot_batch(const Plan& p, const double* d_rot, int rot0, int nrl, bool global, float4* cpos,
                                  float4* cw, int64_t wstride, cudaStream_t s);
cudaError_t launch_centres(int n_out, const int32_t* out_obj, const int32_t* out_rot, int rot0, const double* rot,
                           const double* cen, float4* cyz, cudaStream_t s);
cudaError_t launch_gacc_batch(const FbView& V, int n_out, double* G, cudaStream_t s);
cudaError_t launch_gacc_totals(const double* T, int n_out, int64_t ostride, int64_t npix, double* G, cudaStream_t s);
cudaError_t launch_tf_to_f64(const FbView& V, int64_t o, double* dst, cudaStream_t s);
cudaError_t launch_dilute_shift_batch(const FbView& V, int n_out, const float2* eyz, const int32_t* out_rot,
                                      double* Gdil, double* Ftot, int64_t tstride, double* scratch, int32_t* err,
                                      uint64_t limit_ns, cudaStream_t s);
int dilute_slices(int64_t stored_pixels);
cudaError_t launch_prep_ray_batch(const Plan& p, const double* d_rot, const double2* ray_sc, int n_rays, int slot0,
                                  int nrl, bool global, float4* cpos, float4* cw, int64_t wstride, cudaStream_t s);
cudaError_t launch_ray_centres(int n_out, const int32_t* out_obj, const int32_t* out_rot, int slot0, const double* rot,
                               const double2* ray_sc, int n_rays, const double* cen, float4* cyz, cudaStream_t s);
cudaError_t launch_ray_totals(int nrl, int slot0, int n_rays, int mirror, int n0, int n1, int64_t npr,
                              const double* Ftot_b, int64_t fstride, const double* Gdil_b, int64_t gstride,
                              int last_rot, double* Gtot, double* Gdil, double* Ftot, cudaStream_t s);
cudaError_t launch_ray_gacc(const FbView& V, int n_out, int slot0, int n_rays, int mirror, int n0, int n1, int k2,
                            int last_rot, double* G, double* Gd, double* F, cudaStream_t s);
cudaError_t launch_prep_ray_from_rot(const Plan& p, const float4* rpos, const float4* rw, int64_t rwstride,
                                     const float4* ray_sc_tf, int n_rays, int slot0, int nrl, float4* cpos, float4* cw,
                                     int64_t wstride, cudaStream_t s);
cudaError_t launch_shift_factors(int n_out, const float4* cyz, const float2* qy, int ny, const float2* qz, int nz,
                                 float2* eyz, cudaStream_t s);

namespace {

struct HostItem {
    int32_t mt, nt, kb0, kb1, slot, slot1;   // mode 2: mt indexes an A-tile pair
    int32_t store, two;                      // direct items: first piece of the output stores; two: several pieces
};
struct HostRed {
    int32_t slot_base, splits, out, store;   // store: bit 0 first piece of the output, bit 1 several pieces
};

struct Chunk {
    int64_t kb_off = 0, nkb = 0;    // into the k-block arrays
    int64_t item_off = 0;
    int64_t unit_off = 0;           // into the unit runs: units + 1 first-item indices (chunk-relative)
    int n_items = 0, grid = 0;
    int64_t red_off = 0;
    int n_red = 0;
};

struct OutBatch {
    int out0 = 0, n_out = 0;        // outputs [out0, out0 + n_out) of the schedule
    std::vector<Chunk> chunks;
};

struct Schedule {
    int n_rot_local = 0;
    int n_out = 0;
    std::vector<OutBatch> batches;
    // device arrays
    int64_t* d_kb_cell0 = nullptr;
    int32_t* d_kb_ncell = nullptr;
    void* d_items = nullptr;
    int32_t* d_units = nullptr;
    void* d_reds = nullptr;
    int32_t* d_out_obj = nullptr;
    int32_t* d_out_rot = nullptr;
    uint8_t* d_out_two = nullptr;   // per output: 1 = assembled from several pieces (two-float F_b)
    std::vector<int32_t> h_out_rot; // per output: its slot in the batch (host copy)
    int64_t max_items = 0;
    int max_batch_out = 0;
};

}  // namespace

struct TcState {
    int ny = 0, nz = 0, mtiles = 0, ntiles = 0;
    AxisMap ax{};                // GEMM part of each detector axis (q >= 0 half of a symmetric axis)
    float2* d_qy = nullptr;      // full grid: q_y / 2 pi two-float [ny]
    float2* d_qz = nullptr;
    double W[4] = {1, 1, 1, 1};
    int kcb = 3;
    int items_per_sm = 8;        // work-list granularity of a GEMM launch
    int nsets = 1;               // weight sets (loop mode), stacked along the GEMM rows
    int nch = 4;                 // channels per output: 4 x (weight sets rounded up to a power of two)
    int64_t wstride = 0;         // cells between weight sets in d_cw_b (= R_b * n)
    int mode = 0;                // GEMM form: 0 one CTA per tile, 2 two-SM MMA over A-tile pairs (even mtiles)
    bool mode_forced = false;    // set by NMS_GEMM_MODE: the autotuner keeps it
    bool objects = false;        // per-object amplitudes (dilute split) with shifts
    int R_b = 1;                 // slots (rotations, or rotation x ray pairs) prepared per batch
    int n_slots = 1;             // n_rot, or n_rot x n_rays
    // POLAR grid (rays): slot s = ray s mod n_rays of rotation s / n_rays; the
    // GEMM's q_y axis is |q| = lo + k2 i1 dq (i1 < ny), its q_z axis i2 dq
    // (i2 < nz = k2), and both coordinates are the projection u of a cell on
    // the ray; with n_theta even only the rays theta < pi are computed
    bool rays = false;
    // rays with one weight set and one A and one B tile: the operands are
    // generated in the GEMM's shared memory (k_gemm_ray_fused), no tables
    bool fused = false;
    std::vector<float2> h_qy, h_qz;   // fused: the GEMM nodes in turns, passed as kernel parameters
    int n_rays = 0, ray_mirror = 0;
    double2* d_ray_sc = nullptr; // [n_rays] (sin theta, cos theta)
    float4* d_ray_sc_tf = nullptr;   // the same as two-float (sin hi, lo, cos hi, lo)
    float4* d_rpos = nullptr;    // rays: rotated (Y, Z) two-float [n_rot][n], or null (FP64 per slot)
    float4* d_rw = nullptr;      // rays: rotated weights [set][n_rot][n]
    double* d_Gdil_b = nullptr;  // rays with objects: dilute products per slot [R_b][set][16][ny nz]
    int64_t tab_kb = 0;          // table capacity in k-blocks
    float4* d_cpos_b = nullptr;  // [R_b][n]
    float4* d_cw_b = nullptr;
    double* d_Fb = nullptr;      // out_cap outputs, FbView layout: two planes [out][stored q_z][nch * n_y] of float2
    int out_cap = 1;             // outputs per batch
    double* d_Ftot_b = nullptr;  // [R_b][4][npix][2] (objects)
    float4* d_cyz = nullptr;     // [out_cap]
    float2* d_eyz = nullptr;     // objects: [out_cap][ny + nz] shift factors along q_y and q_z
    double* d_dscr = nullptr;    // objects: dilute-pass scratch planes of output slices 1.. (or null)
    double* d_rot = nullptr;     // [n_rot][9]
    double* d_cen = nullptr;     // [K][3]
    double* d_P = nullptr;       // item tiles
    Schedule full, last;
};

// float2 values in one plane of a batch of GEMM outputs (stored q_z rows)
static int64_t fb_plane(const TcState& t, int n_out) { return (int64_t)n_out * (t.nz - t.ax.zs0) * t.nch * t.ny; }

// view of a batch of GEMM outputs: high plane at F, low plane lo_off float2
// further, per-output piece flags two; weight set st
static FbView fb_view(const TcState& t, const double* F, int64_t lo_off, const uint8_t* two, int st)
{
    FbView v;
    v.hi = reinterpret_cast<const float2*>(F) + 4 * st;
    v.lo = v.hi + lo_off;
    v.two = two;
    v.mrows = t.nch * t.ny;
    v.ostride2 = (int64_t)(t.nz - t.ax.zs0) * v.mrows;
    v.nch = t.nch;
    v.ny = t.ny;
    v.nz = t.nz;
    v.zs0 = t.ax.zs0;
    return v;
}

static double pow2_ceil(double x)
{
    if (!(x > 0)) return 1.0;
    int e;
    frexp(x, &e);
    double r = ldexp(1.0, e);
    if (r / 2 >= x) r /= 2;
    return r;
}

template <class T>
static nms_status upload(T** d, const std::vector<T>& h)
{
    *d = nullptr;
    if (h.empty()) return NMS_OK;
    NMS_CUDA_TRY(plan_malloc((void**)d, h.size() * sizeof(T)));
    NMS_CUDA_TRY(cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return NMS_OK;
}

static void free_schedule(Schedule& s, cudaStream_t used_on)
{
    void* b[] = {s.d_kb_cell0, s.d_kb_ncell, s.d_items, s.d_units, s.d_reds, s.d_out_obj, s.d_out_rot, s.d_out_two};
    for (void* x : b)
        if (x) plan_free(x, used_on);
    s = Schedule();
}

struct Summand {
    int rl, obj;        // rotation slot in the stacked arrays, object index
    int64_t c0, c1;     // cells [c0, c1) of that rotation's arrays
};

// The summands of one rotation batch of n_rl rotations.
static std::vector<Summand> plan_summands(const Plan& p, const TcState& t, int n_rl)
{
    std::vector<Summand> sums;
    for (int rl = 0; rl < n_rl; ++rl) {
        if (t.objects) {
            for (int64_t k = 0; k < p.n_objects; ++k)
                if (p.h_off[k + 1] > p.h_off[k]) sums.push_back({rl, (int)k, p.h_off[k], p.h_off[k + 1]});
        } else {
            sums.push_back({rl, 0, 0, p.n_cells});
        }
    }
    return sums;
}

// Build the schedule of the given summands (n_rl rotation slots).
static nms_status build_schedule(const Plan& p, const TcState& t, const std::vector<Summand>& sums, int n_rl,
                                 int out_cap, Schedule& S)
{
    S.n_rot_local = n_rl;
    S.n_out = (int)sums.size();
    const int64_t KBC = tc_block_cells();   // cells per k-block
    const int sms = device_sm_count();
    const int tiles = t.mtiles * t.ntiles;
    std::vector<int64_t> kb_cell0;
    std::vector<int32_t> kb_ncell;
    std::vector<HostItem> items;
    std::vector<int32_t> unit_item0;
    std::vector<HostRed> reds;
    std::vector<int32_t> out_obj(sums.size()), out_rot(sums.size());
    std::vector<uint8_t> out_two(sums.size(), 0);
    for (size_t o = 0; o < sums.size(); ++o) {
        out_obj[o] = sums[o].obj;
        out_rot[o] = sums[o].rl;
    }
    for (int o0 = 0; o0 < S.n_out; o0 += out_cap) {
        OutBatch ob;
        ob.out0 = o0;
        ob.n_out = std::min(out_cap, S.n_out - o0);
        S.max_batch_out = std::max(S.max_batch_out, ob.n_out);
        // pieces: (out_local, first cell in the stacked arrays, cells)
        struct Piece {
            int out;
            int64_t g0, n;
        };
        std::vector<std::vector<Piece>> chunk_pieces(1);
        // an output's first piece (in launch order) stores, later pieces add,
        // so the batch's amplitudes need no clearing
        std::vector<char> started(ob.n_out, 0);
        int64_t cur_kb = 0;
        for (int o = o0; o < o0 + ob.n_out; ++o) {
            const Summand& sm = sums[o];
            int64_t c = sm.c0;
            while (c < sm.c1) {
                int64_t room = (t.tab_kb - cur_kb) * KBC;
                if (room <= 0) {
                    chunk_pieces.emplace_back();
                    cur_kb = 0;
                    room = t.tab_kb * KBC;
                }
                const int64_t take = std::min(room, sm.c1 - c);
                chunk_pieces.back().push_back({o - o0, (int64_t)sm.rl * p.n_cells + c, take});
                cur_kb += (take + KBC - 1) / KBC;
                c += take;
            }
        }
        // outputs cut into several pieces keep two-float values
        {
            std::vector<int> npieces(ob.n_out, 0);
            for (const auto& pieces : chunk_pieces)
                for (const Piece& pc : pieces) ++npieces[pc.out];
            for (int o = 0; o < ob.n_out; ++o) out_two[o0 + o] = npieces[o] > 1 ? 1 : 0;
        }
        for (auto& pieces : chunk_pieces) {
            if (pieces.empty()) continue;
            Chunk ch;
            ch.kb_off = (int64_t)kb_cell0.size();
            int64_t nkb_chunk = 0;
            for (const Piece& pc : pieces) nkb_chunk += (pc.n + KBC - 1) / KBC;
            ch.nkb = nkb_chunk;
            // work items: about items_per_sm per SM, never shorter than 2 TMEM
            // chunks.  Each piece's split count is rounded up, which adds up to
            // one item per piece and tile; when a few pieces share the chunk
            // those extra items are kept inside the items_per_sm x SMs slots
            // (beyond them the launch would take a second, mostly idle round)
            const int64_t ips = t.items_per_sm;
            const int64_t places = ips * sms;
            const int64_t extra = (int64_t)pieces.size() * tiles;
            const int64_t denom = (pieces.size() > 1 && 2 * extra <= places) ? places - extra : places;
            const int64_t kb_per_item = std::max<int64_t>(2 * t.kcb, (nkb_chunk * tiles + denom - 1) / denom);
            std::vector<HostItem> its;
            ch.red_off = (int64_t)reds.size();
            int slot = 0;
            int64_t kb = 0;
            for (const Piece& pc : pieces) {
                const int64_t nkb_p = (pc.n + KBC - 1) / KBC;
                for (int64_t i = 0; i < nkb_p; ++i) {
                    kb_cell0.push_back(pc.g0 + KBC * i);
                    kb_ncell.push_back((int32_t)std::min<int64_t>(KBC, pc.n - KBC * i));
                }
                // (mt, nt) of the first tile of a work unit and its step to the partner tile
                const int mstep = t.mode == 2 ? 2 : 1, nstep = 1;
                int splits = (int)((nkb_p + kb_per_item - 1) / kb_per_item);
                if (splits > 1 && pieces.size() == 1) {
                    // one output in the chunk: round the split count up so the
                    // (tile unit x split) items fill whole waves of the
                    // persistent CTAs (pairs)
                    const int units = (t.mtiles / mstep) * (t.ntiles / nstep);
                    const int conc = t.mode ? sms / 2 : sms;
                    int gcd = units, rem = conc;
                    while (rem) {
                        const int r = gcd % rem;
                        gcd = rem;
                        rem = r;
                    }
                    const int m = conc / gcd;
                    const int up = ((splits + m - 1) / m) * m;
                    if (up <= 2 * splits && up <= nkb_p / std::max(1, 2 * t.kcb)) splits = up;
                }
                if (splits == 1 && !(t.fused && out_two[o0 + pc.out])) {
                    // one item per tile spans the piece: the GEMM adds it into F directly
                    const int32_t direct = -1 - pc.out;
                    const int32_t first = started[pc.out] ? 0 : 1;
                    const int32_t two = out_two[o0 + pc.out];
                    started[pc.out] = 1;
                    for (int mt = 0; mt < t.mtiles; mt += mstep)
                        for (int nt = 0; nt < t.ntiles; nt += nstep)
                            its.push_back({mt / mstep, nt / nstep, (int32_t)kb, (int32_t)(kb + nkb_p), direct, direct,
                                           first, two});
                    kb += nkb_p;
                    continue;
                }
                reds.push_back({slot, splits, pc.out, (started[pc.out] ? 0 : 1) | (out_two[o0 + pc.out] ? 2 : 0)});
                started[pc.out] = 1;
                // k-range major: the CTAs of one wave share each k-range, so
                // every table block comes from HBM about once and is reused
                // by all tiles through L2
                for (int sp = 0; sp < splits; ++sp)
                    for (int mt = 0; mt < t.mtiles; mt += mstep)
                        for (int nt = 0; nt < t.ntiles; nt += nstep) {
                            const int64_t a = kb + (nkb_p * sp) / splits;
                            const int64_t b = kb + (nkb_p * (sp + 1)) / splits;
                            const int s0 = slot + (mt * t.ntiles + nt) * splits + sp;
                            // slot of the partner tile (mode 2): the next A tile
                            const int s1 = t.mode == 2 ? s0 + t.ntiles * splits : 0;
                            its.push_back({mt / mstep, nt / nstep, (int32_t)a, (int32_t)b, s0, s1, 0, 0});
                        }
                slot += tiles * splits;
                kb += nkb_p;
            }
            ch.n_red = (int)(reds.size() - ch.red_off);
            // longest items first, each to the unit (CTA or CTA pair) with the
            // least work so far (longest-processing-time rule; an item costs
            // its k-blocks plus one for its output).  Items of equal length
            // (the tiles of one k-range) stay adjacent in the list, so they
            // run at about the same time on different units and share the
            // k-range's table blocks through L2.
            std::stable_sort(its.begin(), its.end(),
                             [](const HostItem& x, const HostItem& y) { return (x.kb1 - x.kb0) > (y.kb1 - y.kb0); });
            ch.item_off = (int64_t)items.size();
            ch.n_items = (int)its.size();
            ch.grid = t.mode ? std::min(2 * ch.n_items, sms & ~1) : std::min(ch.n_items, sms);
            const int units = t.mode ? ch.grid / 2 : ch.grid;
            std::vector<std::vector<int>> run(units);
            {
                using Load = std::pair<int64_t, int>;   // (work so far, unit): the lowest unit wins a tie
                std::priority_queue<Load, std::vector<Load>, std::greater<Load>> least;
                for (int u = 0; u < units; ++u) least.push({0, u});
                for (int i = 0; i < ch.n_items; ++i) {
                    const Load l = least.top();
                    least.pop();
                    run[l.second].push_back(i);
                    least.push({l.first + (its[i].kb1 - its[i].kb0) + 1, l.second});
                }
            }
            ch.unit_off = (int64_t)unit_item0.size();
            int32_t first = 0;
            for (int u = 0; u < units; ++u) {
                unit_item0.push_back(first);
                for (int i : run[u]) items.push_back(its[i]);
                first += (int32_t)run[u].size();
            }
            unit_item0.push_back(first);
            S.max_items = std::max<int64_t>(S.max_items, slot);
            ob.chunks.push_back(ch);
        }
        S.batches.push_back(ob);
    }
    nms_status st;
    S.h_out_rot = out_rot;
    if ((st = upload(&S.d_kb_cell0, kb_cell0)) || (st = upload(&S.d_kb_ncell, kb_ncell)) ||
        (st = upload(&S.d_units, unit_item0)) ||
        (st = upload(&S.d_out_obj, out_obj)) || (st = upload(&S.d_out_rot, out_rot)) ||
        (st = upload(&S.d_out_two, out_two)))
        return st;
    if (!items.empty()) {
        NMS_CUDA_TRY(plan_malloc(&S.d_items, items.size() * sizeof(HostItem)));
        NMS_CUDA_TRY(cudaMemcpy(S.d_items, items.data(), items.size() * sizeof(HostItem), cudaMemcpyHostToDevice));
    }
    if (!reds.empty()) {
        NMS_CUDA_TRY(plan_malloc(&S.d_reds, reds.size() * sizeof(HostRed)));
        NMS_CUDA_TRY(cudaMemcpy(S.d_reds, reds.data(), reds.size() * sizeof(HostRed), cudaMemcpyHostToDevice));
    }
    return NMS_OK;
}

// ------------------------------------------------------------------ autotuner
// max over pixels of |A - B| per channel; A two-float (the GEMM's output
// format), B FP64
__global__ void k_amp_maxerr(FbView A, const double2* __restrict__ B, unsigned int* __restrict__ err)
{
    const int64_t npix = (int64_t)A.ny * A.nz;
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= npix) return;
    const int qa = (int)(p / A.nz), qb = (int)(p % A.nz);
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const double2 a = A.load_f64(0, qa, qb, c);
        const double2 b = B[(int64_t)c * npix + p];
        const float d = (float)hypot(a.x - b.x, a.y - b.y);
        atomicMax(&err[c], __float_as_uint(d));   // non-negative floats order as integers
    }
}

__global__ void k_wabs_sum(const float4* __restrict__ cw, int64_t c0, int64_t c1, double* __restrict__ sums)
{
    __shared__ double red[4][256];
    double a[4] = {0, 0, 0, 0};
    for (int64_t j = c0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < c1; j += (int64_t)gridDim.x * blockDim.x) {
        const float4 w = cw[j];
        a[0] += fabsf(w.x);
        a[1] += fabsf(w.y);
        a[2] += fabsf(w.z);
        a[3] += fabsf(w.w);
    }
    for (int c = 0; c < 4; ++c) red[c][threadIdx.x] = a[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int c = 0; c < 4; ++c) atomicAdd(&sums[c], red[c][0]);
}

struct TuneChoice {
    int kcb, ips, mode;
};

static std::mutex g_tune_mu;
static std::map<std::string, TuneChoice> g_tune_cache;
static bool g_tune_file_read = false;

static void tune_file_read()
{
    if (g_tune_file_read) return;
    g_tune_file_read = true;
    const char* path = getenv("NMS_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char key[256];
    int a, b, m;
    while (fscanf(f, "%255s %d %d %d", key, &a, &b, &m) == 4)
        if (a > 0 && b > 0 && m >= 0 && m <= 2) g_tune_cache[key] = {a, b, m};
    fclose(f);
}

static void tune_file_append(const std::string& key, TuneChoice c)
{
    const char* path = getenv("NMS_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d\n", key.c_str(), c.kcb, c.ips, c.mode);
    fclose(f);
}

// Time candidate GEMM forms, drain intervals and work-list granularities on
// a probe of the cells and keep the fastest whose error is within the bound.
nms_status tc_autotune(Plan& p, TcState& t)
{
    const int sms = device_sm_count();
    // probe: up to 131072 cells of the largest summand under the first rotation
    int64_t c0 = 0, c1 = p.n_cells;
    if (t.objects) {
        int64_t best = -1;
        for (int64_t k = 0; k < p.n_objects; ++k)
            if (p.h_off[k + 1] - p.h_off[k] > best) {
                best = p.h_off[k + 1] - p.h_off[k];
                c0 = p.h_off[k];
                c1 = p.h_off[k + 1];
            }
    }
    c1 = std::min<int64_t>({c1, c0 + 131072, c0 + t.tab_kb * tc_block_cells()});
    const int64_t nprobe = c1 - c0;
    char keybuf[256];
    snprintf(keybuf, sizeof keybuf, "f16x3:%dx%d:half%dx%d:ch%d:cells%lld:sm%d:forms%d", t.ny, t.nz, t.ax.nyg,
             t.ax.nzg, t.nch, (long long)(64 - __builtin_clzll(nprobe)), sms, t.mode_forced ? t.mode : -1);
    const std::string key(keybuf);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        tune_file_read();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            t.kcb = it->second.kcb;
            t.items_per_sm = it->second.ips;
            t.mode = it->second.mode;
            return NMS_OK;
        }
    }
    cudaStream_t s = p.stream;
    const int64_t np = p.npix;
    RotMat R;
    memcpy(R.m, &p.h_rot[0], sizeof(R.m));
    const bool timer_was_on = p.timer.on;
    int64_t launches_before[ST_COUNT];
    memcpy(launches_before, p.timer.launches, sizeof(launches_before));
    p.timer.on = false;          // probe launches are not part of the plan's stage counts
    // reference: the compensated direct sum over the probe cells
    NMS_CUDA_TRY(launch_prep(p, R.m, s));
    const float4* ref_pos = t.objects ? p.d_cposl : p.d_cpos;
    nms_status st = direct_sum_range(p, ref_pos, c0, c1, p.d_F);
    if (st) return st;
    NMS_CUDA_TRY(launch_prep_rot(p, R, !t.objects, t.d_cpos_b, t.d_cw_b, t.wstride, s));
    double* d_sw = nullptr;
    unsigned int* d_err = nullptr;
    double* d_Fp = nullptr;
    NMS_CUDA_TRY(plan_malloc(&d_sw, 4 * sizeof(double)));
    NMS_CUDA_TRY(plan_malloc(&d_err, 4 * sizeof(unsigned int)));
    NMS_CUDA_TRY(plan_malloc(&d_Fp, (size_t)t.nch * 2 * np * sizeof(double)));
    NMS_CUDA_TRY(cudaMemsetAsync(d_sw, 0, 4 * sizeof(double), s));
    k_wabs_sum<<<std::max(1, std::min(4 * sms, (int)((nprobe + 255) / 256))), 256, 0, s>>>(t.d_cw_b, c0, c1, d_sw);
    NMS_CUDA_TRY(cudaGetLastError());
    double wsum[4];
    NMS_CUDA_TRY(cudaMemcpyAsync(wsum, d_sw, sizeof(wsum), cudaMemcpyDeviceToHost, s));
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const float sc = tc_operand_scale();
    const float wscale[4] = {(float)(sc / t.W[0]), (float)(sc / t.W[1]), (float)(sc / t.W[2]), (float)(sc / t.W[3])};
    double scale[4];
    for (int c = 0; c < 4; ++c) scale[c] = t.W[c] / ((double)sc * (double)sc);
    const uint64_t limit = p.opt.max_spin > 0 ? (uint64_t)p.opt.max_spin * 1000ull : 4000000000ull;
    const std::vector<Summand> probe = {{0, 0, c0, c1}};
    const int mode0 = t.mode;
    TuneChoice best{3, 8, mode0};
    float best_ms = 1e30f;
    const int kcbs[4] = {1, 2, 3, 4};
    const int ipss[3] = {4, 8, 16};
    std::vector<int> modes;
    for (int m = 0; m < 3; ++m)
        if (t.mode_forced ? m == mode0 : (m == 0 || (m == 2 && t.mtiles % 2 == 0)))
            modes.push_back(m);
    double* saveP = t.d_P;
    std::vector<TuneChoice> cand;
    for (int mode : modes)
        for (int kcb : kcbs)
            for (int ips : ipss) cand.push_back({kcb, ips, mode});
    for (const TuneChoice& cd : cand) {
        const int mode = cd.mode, kcb = cd.kcb, ips = cd.ips;
        t.mode = mode;
        t.kcb = kcb;
        t.items_per_sm = ips;
        Schedule S;
        st = build_schedule(p, t, probe, 1, 1, S);
        if (st) break;
        double* P = nullptr;
        cudaError_t ce = plan_malloc(&P, (size_t)std::max<int64_t>(1, S.max_items) * 128 * 128 * sizeof(double));
        if (ce != cudaSuccess) { free_schedule(S, s); st = cuda_fail(ce, "autotune partials"); break; }
        float ms = 1e30f;
        const Chunk& ch = S.batches[0].chunks[0];
        const int64_t lo_off = fb_plane(t, 1);
        for (int rep = 0; rep < 2 && ce == cudaSuccess; ++rep) {
            ce = tc_launch_tables(t.d_cpos_b, t.d_cw_b, t.wstride, t.nch, S.d_kb_cell0, S.d_kb_ncell, ch.nkb,
                                  t.d_qy + t.ax.hy, t.ax.nyg, t.d_qz + t.ax.hz, t.ax.nzg, t.mtiles, t.ntiles, wscale,
                                  p.d_tab, s);
            if (ce == cudaSuccess) ce = cudaEventRecord(e0, s);
            if (ce == cudaSuccess)
                ce = tc_launch_gemm(p.d_tab, ch.nkb, t.mtiles, t.ntiles, S.d_items, S.d_units + ch.unit_off, ch.grid,
                                    kcb, P, d_Fp, lo_off, t.ax, t.nch, scale, p.d_err, limit, t.mode, s);
            if (ce == cudaSuccess) ce = cudaEventRecord(e1, s);
            if (ce == cudaSuccess)
                ce = tc_launch_reduce(P, S.d_reds, ch.n_red, t.ax, t.ntiles, t.nch, scale, d_Fp, lo_off, s);
            if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
            float m = 0.f;
            if (ce == cudaSuccess) cudaEventElapsedTime(&m, e0, e1);
            ms = std::min(ms, m);
        }
        unsigned int herr[4] = {0, 0, 0, 0};
        if (ce == cudaSuccess) ce = cudaMemsetAsync(d_err, 0, sizeof(herr), s);
        if (ce == cudaSuccess) {
            k_amp_maxerr<<<(unsigned)((np + 255) / 256), 256, 0, s>>>(fb_view(t, d_Fp, lo_off, S.d_out_two, 0),
                                                                    reinterpret_cast<const double2*>(p.d_F), d_err);
            ce = cudaGetLastError();
        }
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(herr, d_err, sizeof(herr), cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        // ordered after this candidate's launches on s, also when one failed
        plan_free(P, s);
        free_schedule(S, s);
        if (ce != cudaSuccess) { st = cuda_fail(ce, "autotune probe"); break; }
        double err = 0.0;
        for (int c = 0; c < 4; ++c)
            if (wsum[c] > 0) err = std::max(err, (double)__builtin_bit_cast(float, herr[c]) / wsum[c]);
        if (err <= 3e-7 && ms < best_ms) {
            best_ms = ms;
            best = {kcb, ips, mode};
        }
    }
    t.d_P = saveP;
    p.timer.on = timer_was_on;
    memcpy(p.timer.launches, launches_before, sizeof(launches_before));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    plan_free(d_sw, s);
    plan_free(d_err, s);
    plan_free(d_Fp, s);
    if (st) return st;
    NMS_CUDA_TRY(cudaMemsetAsync(p.d_err, 0, sizeof(int32_t), s));
    t.kcb = best.kcb;
    t.items_per_sm = best.ips;
    t.mode = best.mode;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tune_cache[key] = best;
    tune_file_append(key, best);
    return NMS_OK;
}

int tc_tuned_kc_cells(const Plan& p)
{
    const TcState* t = (const TcState*)p.tc_state;
    return t ? tc_block_cells() * t->kcb : 0;
}

int tc_tuned_items_per_sm(const Plan& p)
{
    const TcState* t = (const TcState*)p.tc_state;
    return t ? t->items_per_sm : 0;
}

void tc_form_info(const Plan& p, int32_t* form, int32_t* mirror_y, int32_t* mirror_z)
{
    const TcState* t = (const TcState*)p.tc_state;
    *form = t ? (t->fused ? 3 : t->mode) : -1;
    *mirror_y = t ? t->ax.my : 0;
    *mirror_z = t ? t->ax.mz : 0;
}

nms_status tc_setup(Plan& p)
{
    if (p.grid.kind != NMS_QGRID_CARTESIAN && p.grid.kind != NMS_QGRID_POLAR) {
        set_error("tensor-core path needs a CARTESIAN or POLAR grid");
        return NMS_ERR_INVALID_ARG;
    }
    if (tc_item_bytes() != sizeof(HostItem) || tc_red_bytes() != sizeof(HostRed)) {
        set_error("internal: work-list record size mismatch");
        return NMS_ERR_UNSUPPORTED;
    }
    TcState* t = new TcState();
    p.tc_state = t;
    t->rays = p.grid.kind == NMS_QGRID_POLAR;
    // rays: |q|_i = lo + i dq, i = k2 i1 + i2, split over the GEMM's two axes
    const int k2 = t->rays ? std::min(64, p.grid.n0) : 0;
    t->ny = t->rays ? (p.grid.n0 + k2 - 1) / k2 : p.grid.n0;
    t->nz = t->rays ? k2 : p.grid.n1;
    t->nsets = p.n_sets;
    {
        int sp = 1;
        while (sp < t->nsets) sp <<= 1;
        t->nch = 4 * sp;
    }
    // an axis symmetric about q = 0 (lo = -hi, two or more nodes): the GEMM
    // covers its q >= 0 half and the epilogue writes both signs
    // (NMS_GRID_MIRROR=0 turns this off, for comparisons)
    const char* mirror_env = getenv("NMS_GRID_MIRROR");
    const bool mirror_ok = !(mirror_env && atoi(mirror_env) == 0);
    t->ax.ny = t->ny;
    t->ax.nz = t->nz;
    t->ax.my = (!t->rays && mirror_ok && t->ny >= 2 && p.grid.lo0 == -p.grid.hi0) ? 1 : 0;
    t->ax.mz = (!t->rays && mirror_ok && t->nz >= 2 && p.grid.lo1 == -p.grid.hi1) ? 1 : 0;
    t->ax.hy = t->ax.my ? t->ny / 2 : 0;
    t->ax.hz = t->ax.mz ? t->nz / 2 : 0;
    t->ax.nyg = t->ny - t->ax.hy;
    t->ax.nzg = t->nz - t->ax.hz;
    // point-symmetric detector: amplitudes stored for q_z >= 0 only
    t->ax.zs0 = (t->ax.my && t->ax.mz) ? t->ax.hz : 0;
    // A rows: (q_y node, channel) x (cos, sin); B rows: q_z node x (cos, sin)
    t->mtiles = (2 * t->nch * t->ax.nyg + 127) / 128;
    t->ntiles = (2 * t->ax.nzg + 127) / 128;
    // default drain interval 3 k-blocks (192 cells): the error at a fully
    // coherent pixel (all products of one sign, q = 0) is 8.2e-7 .. 8.9e-7 of
    // sum |w| there, 5.2e-7 at 128 cells and 1.11e-6 (over the 1e-6 bar) at 256
    t->kcb = p.opt.kc_cells > 0 ? std::max(1, p.opt.kc_cells / tc_block_cells()) : 3;
    // rays: one output tile per slot, so a chunk's few outputs are split
    // over the CTAs and reduced; one item per SM keeps the splits (and the
    // serial sums of the reduction) few
    if (t->rays) t->items_per_sm = 1;
    if (p.opt.split_k > 0) t->items_per_sm = std::min(256, p.opt.split_k);
    t->objects = p.n_objects > 1 && p.opt.want_dilute;
    // One CTA per tile by default (the two-SM MMA writes fewer operand bytes
    // into shared memory per stage, but each SM still reads the whole B tile,
    // half of it from the peer, and it measured slower).  NMS_GEMM_MODE = 0
    // or 2 forces a form the grid allows (diagnostics, tests); the autotuner
    // times both.
    t->mode = 0;
    if (const char* gm = getenv("NMS_GEMM_MODE")) {
        const int want = atoi(gm);
        if (want == 0 || (want == 2 && t->mtiles % 2 == 0)) {
            t->mode = want;
            t->mode_forced = true;
        }
    }
    const int64_t n = p.n_cells;
    const int64_t np = p.npix;

    std::vector<float2> qy(t->ny), qz(t->nz);
    const double two_pi = 2.0 * M_PI;
    auto lin = [](int64_t a, int64_t nn, double lo, double hi) {
        return nn == 1 ? lo : lo + ((hi - lo) * (double)a) / (double)(nn - 1);
    };
    // rays: the q_y axis holds lo + k2 i1 dq, the q_z axis i2 dq, so that
    // node (i1, i2) is |q|_{k2 i1 + i2} (nodes past n0 are computed and not read)
    const double dq = (t->rays && p.grid.n0 > 1) ? (p.grid.hi0 - p.grid.lo0) / (double)(p.grid.n0 - 1) : 0.0;
    for (int a = 0; a < t->ny; ++a) {
        double v = (t->rays ? p.grid.lo0 + (double)k2 * a * dq : lin(a, t->ny, p.grid.lo0, p.grid.hi0)) / two_pi;
        float h = (float)v;
        qy[a] = make_float2(h, (float)(v - (double)h));
    }
    for (int b = 0; b < t->nz; ++b) {
        double v = (t->rays ? (double)b * dq : lin(b, t->nz, p.grid.lo1, p.grid.hi1)) / two_pi;
        float h = (float)v;
        qz[b] = make_float2(h, (float)(v - (double)h));
    }
    nms_status st;
    if ((st = upload(&t->d_qy, qy)) || (st = upload(&t->d_qz, qz))) return st;
    // rays whose GEMM has one B tile and at most three A tiles per slot (one
    // weight set, at most 48 x 64 |q| nodes): operands generated in shared
    // memory, each CTA building the A tile of its item and the B tile, with
    // eight work items per SM so the many equal splits balance
    // (NMS_RAY_FUSED=0 keeps the tables, for comparisons)
    {
        const char* fe = getenv("NMS_RAY_FUSED");
        t->fused = t->rays && t->nch == 4 && t->mtiles <= 3 && t->ntiles == 1 && t->mode == 0 &&
                   !(fe && atoi(fe) == 0);
        if (t->fused) {
            t->h_qy = qy;
            t->h_qz = qz;
            if (p.opt.split_k <= 0) t->items_per_sm = 8;
        }
    }
    t->n_slots = p.n_rot;
    if (t->rays) {
        // theta_j = 2 pi j / n1; with n1 even the ray theta + pi is the
        // conjugate of the ray theta (q negated), so only j < n1 / 2 is computed
        const int n1 = p.grid.n1;
        t->ray_mirror = (n1 % 2 == 0 && mirror_ok) ? 1 : 0;
        t->n_rays = t->ray_mirror ? n1 / 2 : n1;
        if ((int64_t)p.n_rot * t->n_rays > (int64_t)INT32_MAX / 2) {
            set_error("tensor-core path on a POLAR grid: n_rot x n_theta too large");
            return NMS_ERR_UNSUPPORTED;
        }
        t->n_slots = p.n_rot * t->n_rays;
        std::vector<double2> sc(t->n_rays);
        std::vector<float4> sct(t->n_rays);
        for (int j = 0; j < t->n_rays; ++j) {
            const double th = two_pi * (double)j / (double)n1;
            sc[j] = make_double2(sin(th), cos(th));
            const float sh = (float)sc[j].x, ch = (float)sc[j].y;
            sct[j] = make_float4(sh, (float)(sc[j].x - (double)sh), ch, (float)(sc[j].y - (double)ch));
        }
        if ((st = upload(&t->d_ray_sc, sc)) || (st = upload(&t->d_ray_sc_tf, sct))) return st;
        // the cells rotated once per rotation (positions and weights, up to
        // 1 GB), so that each ray only projects them
        // (NMS_RAY_PREP_FP64=1 takes the FP64 rotation per slot regardless,
        // for comparisons)
        const int64_t rbytes = (int64_t)p.n_rot * p.n_cells * 16 * (1 + p.n_sets);
        const char* fp64_env = getenv("NMS_RAY_PREP_FP64");
        const bool per_slot = fp64_env && atoi(fp64_env) != 0;
        if (!per_slot && p.n_rot <= 65535 && rbytes <= (1ll << 30)) {
            NMS_CUDA_TRY(plan_malloc(&t->d_rpos, (size_t)p.n_rot * p.n_cells * sizeof(float4)));
            NMS_CUDA_TRY(plan_malloc(&t->d_rw, (size_t)p.n_sets * p.n_rot * p.n_cells * sizeof(float4)));
        }
    }
    t->W[0] = pow2_ceil(p.h_wmax[0]);
    t->W[1] = t->W[2] = t->W[3] = pow2_ceil(p.h_wmax[1]);
    // the GEMM applies W_c / 2^24 in FP32 (a power of two: exact while normal)
    for (int c = 0; c < 4; ++c)
        if (!(t->W[c] >= 0x1p-90 && t->W[c] <= 0x1p+100)) {
            set_error("tensor-core path: cell weights V|N|, V|M| outside [2^-90, 2^100]; rescale the inputs");
            return NMS_ERR_UNSUPPORTED;
        }
    if ((st = upload(&t->d_rot, p.h_rot))) return st;
    if (t->objects && !p.h_cen.empty()) {
        if ((st = upload(&t->d_cen, p.h_cen))) return st;
    } else if (t->objects) {
        std::vector<double> z((size_t)3 * p.n_objects, 0.0);
        if ((st = upload(&t->d_cen, z))) return st;
    }

    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    // rotations prepared per batch: stacked positions and weights (every
    // weight set, [set][rotation][cell]) up to 2 GB
    const int64_t per_rot = n * 16 * (1 + t->nch / 4);
    t->R_b = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)t->n_slots, 64, (2ll << 30) / std::max<int64_t>(1, per_rot)}));
    t->wstride = (int64_t)t->R_b * n;
    NMS_CUDA_TRY(plan_malloc(&t->d_cpos_b, (size_t)t->R_b * n * sizeof(float4)));
    NMS_CUDA_TRY(plan_malloc(&t->d_cw_b, (size_t)(t->nch / 4) * t->wstride * sizeof(float4)));
    // padding sets (up to the power of two) keep zero weights
    NMS_CUDA_TRY(cudaMemset(t->d_cw_b, 0, (size_t)(t->nch / 4) * t->wstride * sizeof(float4)));
    // output amplitude batch: up to 1 GB, nch complex channels per output
    const int64_t out_bytes = (int64_t)t->nch * t->ny * (t->nz - t->ax.zs0) * 16;
    const int64_t outs_per_rb = t->objects ? (int64_t)t->R_b * p.n_objects : t->R_b;
    const int out_cap = (int)std::max<int64_t>(1, std::min<int64_t>(outs_per_rb, (1ll << 30) / out_bytes));
    t->out_cap = out_cap;
    NMS_CUDA_TRY(plan_malloc(&t->d_Fb, (size_t)out_cap * out_bytes));
    NMS_CUDA_TRY(plan_malloc(&t->d_cyz, (size_t)out_cap * sizeof(float4)));
    if (t->objects) NMS_CUDA_TRY(plan_malloc(&t->d_eyz, (size_t)out_cap * (t->ny + t->nz) * sizeof(float2)));
    // dilute pass: G_dil (16) and shifted-sum (4 complex) planes per extra output slice
    // pixels of one output's image: the detector, or (rays) the ray's node grid
    const int64_t npg = t->rays ? (int64_t)t->ny * t->nz : np;
    const int dsl = dilute_slices((int64_t)t->ny * (t->nz - t->ax.zs0));
    if (t->objects && dsl > 1) NMS_CUDA_TRY(plan_malloc(&t->d_dscr, (size_t)(dsl - 1) * 24 * npg * sizeof(double)));
    // total amplitude per prepared rotation and weight set
    if (t->objects) NMS_CUDA_TRY(plan_malloc(&t->d_Ftot_b, (size_t)t->R_b * t->nsets * 8 * npg * sizeof(double)));
    // rays: each slot's dilute products on its ray grid, scattered after the batch
    if (t->objects && t->rays)
        NMS_CUDA_TRY(plan_malloc(&t->d_Gdil_b, (size_t)t->R_b * t->nsets * 16 * npg * sizeof(double)));
    // phase tables: as many k-blocks as the workspace allows
    const int64_t per_kb = (int64_t)(t->mtiles + t->ntiles) * 2 * (int64_t)tc_block_bytes();
    const int64_t budget = p.opt.workspace_bytes > 0 ? p.opt.workspace_bytes
                                                     : (int64_t)std::min<size_t>(free_b / 3, (size_t)8 << 30);
    int64_t total_kb = 0;
    const int64_t kbc = tc_block_cells();
    if (t->objects) {
        for (int64_t k = 0; k < p.n_objects; ++k) total_kb += (p.h_off[k + 1] - p.h_off[k] + kbc - 1) / kbc;
    } else {
        total_kb = (n + kbc - 1) / kbc;
    }
    total_kb *= t->R_b;
    if (t->fused) {
        // no tables: a batch's slots form one chunk (one GEMM launch)
        t->tab_kb = std::max<int64_t>(1, std::min<int64_t>(total_kb, (int64_t)1 << 30));
        p.tab_bytes = 0;
    } else {
        t->tab_kb = std::max<int64_t>(1, std::min<int64_t>(total_kb, budget / per_kb));
        p.tab_bytes = (size_t)t->tab_kb * per_kb;
        NMS_CUDA_TRY(plan_malloc(&p.d_tab, p.tab_bytes));
    }
    // schedules: a full rotation batch and the remainder
    if (p.opt.autotune && !t->rays) {   // the tuner's error check reads the Cartesian pixel layout
        if ((st = tc_autotune(p, *t))) return st;
    }
    if ((st = build_schedule(p, *t, plan_summands(p, *t, t->R_b), t->R_b, out_cap, t->full))) return st;
    const int rem = t->n_slots % t->R_b;
    if (rem) {
        if ((st = build_schedule(p, *t, plan_summands(p, *t, rem), rem, out_cap, t->last))) return st;
    }
    const int64_t slots = std::max(t->full.max_items, t->last.max_items);
    NMS_CUDA_TRY(plan_malloc(&t->d_P, (size_t)std::max<int64_t>(1, slots) * 128 * 128 * sizeof(double)));
    return NMS_OK;
}

int64_t tc_object_count(const Plan& p)
{
    const TcState* t = (const TcState*)p.tc_state;
    return (t && t->objects) ? p.n_objects : 1;
}

void tc_release(Plan& p)
{
    TcState* t = (TcState*)p.tc_state;
    if (!t) return;
    void* b[] = {t->d_qy,  t->d_qz,  t->d_cpos_b, t->d_cw_b, t->d_Fb, t->d_Ftot_b,
                 t->d_cyz, t->d_eyz, t->d_dscr,   t->d_rot,  t->d_cen, t->d_P, t->d_ray_sc,
                 t->d_ray_sc_tf, t->d_rpos, t->d_rw, t->d_Gdil_b};
    for (void* x : b)
        if (x) plan_free(x, p.stream);
    free_schedule(t->full, p.stream);
    free_schedule(t->last, p.stream);
    delete t;
    p.tc_state = nullptr;
}

nms_status tc_amplitudes(Plan& p, cudaStream_t s)
{
    TcState& t = *(TcState*)p.tc_state;
    const int64_t np = p.npix;
    const int nS = t.nsets;
    const int64_t F4 = 8 * np;                   // doubles of one set's amplitudes [4][np] complex
    const int64_t npg = t.rays ? (int64_t)t.ny * t.nz : np;   // pixels of one output's image
    const int64_t F4g = 8 * npg;
    const float sc = tc_operand_scale();
    const float wscale[4] = {(float)(sc / t.W[0]), (float)(sc / t.W[1]), (float)(sc / t.W[2]), (float)(sc / t.W[3])};
    double scale[4];
    for (int c = 0; c < 4; ++c) scale[c] = t.W[c] / ((double)sc * (double)sc);
    const uint64_t limit = p.opt.max_spin > 0 ? (uint64_t)p.opt.max_spin * 1000ull : 4000000000ull;
    const int64_t lo_off = fb_plane(t, t.out_cap);   // float2 from the high to the low plane of F_b
    if (t.rays && t.d_rpos) {
        // every rotation's cells once (global positions), for the rays to project
        p.timer.begin(ST_PREP);
        NMS_CUDA_TRY(launch_prep_rot_batch(p, t.d_rot, 0, p.n_rot, !t.objects, t.d_rpos, t.d_rw,
                                           (int64_t)p.n_rot * p.n_cells, s));
        p.timer.end(ST_PREP, 1);
    }
    for (int rb0 = 0; rb0 < t.n_slots; rb0 += t.R_b) {
        const int nrl = std::min(t.R_b, t.n_slots - rb0);
        const Schedule& S = nrl == t.R_b ? t.full : t.last;
        // fused rays with the cells rotated once per rotation: the GEMM projects
        // them itself, so the batch needs no per-slot arrays
        const bool project = t.fused && t.d_rpos && nrl <= 64;
        if (!project) {
            p.timer.begin(ST_PREP);
            // the batch's slots in one launch (rotation, or rotation x ray, rb0 + rl into slot rl)
            if (t.rays && t.d_rpos)
                NMS_CUDA_TRY(launch_prep_ray_from_rot(p, t.d_rpos, t.d_rw, (int64_t)p.n_rot * p.n_cells,
                                                      t.d_ray_sc_tf, t.n_rays, rb0, nrl, t.d_cpos_b, t.d_cw_b,
                                                      t.wstride, s));
            else if (t.rays)
                NMS_CUDA_TRY(launch_prep_ray_batch(p, t.d_rot, t.d_ray_sc, t.n_rays, rb0, nrl, !t.objects, t.d_cpos_b,
                                                   t.d_cw_b, t.wstride, s));
            else
                NMS_CUDA_TRY(launch_prep_rot_batch(p, t.d_rot, rb0, nrl, !t.objects, t.d_cpos_b, t.d_cw_b, t.wstride,
                                                   s));
            p.timer.end(ST_PREP, 1);
        }
        if (t.objects) NMS_CUDA_TRY(cudaMemsetAsync(t.d_Ftot_b, 0, (size_t)nrl * nS * F4g * sizeof(double), s));
        if (t.d_Gdil_b) NMS_CUDA_TRY(cudaMemsetAsync(t.d_Gdil_b, 0, (size_t)nrl * nS * 16 * npg * sizeof(double), s));
        for (const OutBatch& ob : S.batches) {
            for (const Chunk& ch : ob.chunks) {
                if (t.fused) {
                    p.timer.begin(ST_GEMM);
                    RayProjection pr;
                    if (project) {
                        pr.ray_sc = t.d_ray_sc_tf;
                        pr.n_cells = p.n_cells;
                        pr.slot0 = rb0;
                        pr.n_rays = t.n_rays;
                        pr.n_rl = nrl;
                    }
                    NMS_CUDA_TRY(tc_launch_gemm_rays(project ? t.d_rpos : t.d_cpos_b, project ? t.d_rw : t.d_cw_b,
                                                     S.d_kb_cell0 + ch.kb_off, S.d_kb_ncell + ch.kb_off, pr,
                                                     t.h_qy.data(), t.ax.nyg, t.h_qz.data(),
                                                     t.ax.nzg, wscale, (const char*)S.d_items + ch.item_off * tc_item_bytes(),
                                                     S.d_units + ch.unit_off, ch.grid, t.kcb, t.d_P, t.d_Fb, lo_off,
                                                     t.ax, t.nch, scale, p.d_err, limit, s));
                    p.timer.end(ST_GEMM, 1);
                    p.timer.begin(ST_REDUCE);
                    NMS_CUDA_TRY(tc_launch_reduce(t.d_P, (const char*)S.d_reds + ch.red_off * tc_red_bytes(), ch.n_red,
                                                  t.ax, t.ntiles, t.nch, scale, t.d_Fb, lo_off, s));
                    p.timer.end(ST_REDUCE, ch.n_red > 0 ? 1 : 0);
                    continue;
                }
                p.timer.begin(ST_TABLES);
                NMS_CUDA_TRY(tc_launch_tables(t.d_cpos_b, t.d_cw_b, t.wstride, t.nch, S.d_kb_cell0 + ch.kb_off,
                                              S.d_kb_ncell + ch.kb_off, ch.nkb, t.d_qy + t.ax.hy, t.ax.nyg,
                                              t.d_qz + t.ax.hz, t.ax.nzg, t.mtiles, t.ntiles, wscale, p.d_tab, s));
                p.timer.end(ST_TABLES, 1);
                p.timer.begin(ST_GEMM);
                NMS_CUDA_TRY(tc_launch_gemm(p.d_tab, ch.nkb, t.mtiles, t.ntiles,
                                            (const char*)S.d_items + ch.item_off * tc_item_bytes(),
                                            S.d_units + ch.unit_off, ch.grid, t.kcb, t.d_P, t.d_Fb, lo_off, t.ax,
                                            t.nch, scale, p.d_err, limit, t.mode, s));
                p.timer.end(ST_GEMM, 1);
                p.timer.begin(ST_REDUCE);
                NMS_CUDA_TRY(tc_launch_reduce(t.d_P, (const char*)S.d_reds + ch.red_off * tc_red_bytes(), ch.n_red, t.ax,
                                              t.ntiles, t.nch, scale, t.d_Fb, lo_off, s));
                p.timer.end(ST_REDUCE, ch.n_red > 0 ? 1 : 0);
            }
            p.timer.begin(ST_GACC);
            int nl = 0;
            if (p.oiq_id >= 0) {   // one weight set (checked when requested)
                const FbView V0 = fb_view(t, t.d_Fb, lo_off, S.d_out_two + ob.out0, 0);
                NMS_CUDA_TRY(launch_obj_bin(V0, ob.n_out, S.d_out_obj + ob.out0, p, p.d_bin_of, p.oiq_nbins, p.oiq_id,
                                            p.d_Iobj, s));
                ++nl;
            }
            if (t.objects) {
                if (t.rays)
                    NMS_CUDA_TRY(launch_ray_centres(ob.n_out, S.d_out_obj + ob.out0, S.d_out_rot + ob.out0, rb0, t.d_rot,
                                                    t.d_ray_sc, t.n_rays, t.d_cen, t.d_cyz, s));
                else
                    NMS_CUDA_TRY(launch_centres(ob.n_out, S.d_out_obj + ob.out0, S.d_out_rot + ob.out0, rb0, t.d_rot,
                                                t.d_cen, t.d_cyz, s));
                NMS_CUDA_TRY(launch_shift_factors(ob.n_out, t.d_cyz, t.d_qy, t.ny, t.d_qz, t.nz, t.d_eyz, s));
                nl += 2;
            }
            for (int st = 0; st < nS; ++st) {
                const FbView V = fb_view(t, t.d_Fb, lo_off, S.d_out_two + ob.out0, st);   // set st of the batch's outputs
                if (t.objects && t.rays) {
                    // one dilute pass per slot: each ray's outputs have their own
                    // pixels, accumulated on its node grid and scattered later
                    for (int o = 0; o < ob.n_out;) {
                        const int rl = S.h_out_rot[ob.out0 + o];
                        int e = o + 1;
                        while (e < ob.n_out && S.h_out_rot[ob.out0 + e] == rl) ++e;
                        FbView Vs = V;
                        Vs.hi += (int64_t)o * V.ostride2;
                        Vs.lo += (int64_t)o * V.ostride2;
                        Vs.two += o;
                        NMS_CUDA_TRY(launch_dilute_shift_batch(Vs, e - o, t.d_eyz + (size_t)o * (t.ny + t.nz),
                                                               S.d_out_rot + ob.out0 + o,
                                                               t.d_Gdil_b + ((size_t)rl * nS + st) * 16 * npg,
                                                               t.d_Ftot_b + (size_t)st * F4g, (int64_t)nS * F4g,
                                                               t.d_dscr, p.d_err, limit, s));
                        nl += std::min(dilute_slices(Vs.stored_pixels()), e - o) > 1 && t.d_dscr ? 2 : 1;
                        o = e;
                    }
                } else if (t.objects) {
                    NMS_CUDA_TRY(launch_dilute_shift_batch(V, ob.n_out, t.d_eyz, S.d_out_rot + ob.out0,
                                                           p.d_Gdil + (size_t)st * 16 * np,
                                                           t.d_Ftot_b + (size_t)st * F4, (int64_t)nS * F4, t.d_dscr,
                                                           p.d_err, limit, s));
                    nl += std::min(dilute_slices(V.stored_pixels()), ob.n_out) > 1 && t.d_dscr ? 2 : 1;
                } else if (t.rays) {
                    // each ray's amplitudes into its POLAR pixels (and the mirror rays)
                    NMS_CUDA_TRY(launch_ray_gacc(V, ob.n_out, rb0 + ob.out0, t.n_rays, t.ray_mirror, p.grid.n0,
                                                 p.grid.n1, t.nz, p.n_rot - 1, p.d_Gtot + (size_t)st * 16 * np,
                                                 p.d_Gdil ? p.d_Gdil + (size_t)st * 16 * np : nullptr,
                                                 p.d_F + (size_t)st * F4, s));
                    ++nl;
                } else {
                    NMS_CUDA_TRY(launch_gacc_batch(V, ob.n_out, p.d_Gtot + (size_t)st * 16 * np, s));
                    ++nl;
                    if (p.d_Gdil) {
                        NMS_CUDA_TRY(launch_gacc_batch(V, ob.n_out, p.d_Gdil + (size_t)st * 16 * np, s));
                        ++nl;
                    }
                    if (rb0 + nrl == t.n_slots && &ob == &S.batches.back())
                        NMS_CUDA_TRY(launch_tf_to_f64(V, ob.n_out - 1, p.d_F + (size_t)st * F4, s));
                }
            }
            p.timer.end(ST_GACC, nl);
        }
        if (t.objects && t.rays) {
            // each slot's dilute products and total amplitude into the POLAR pixels
            p.timer.begin(ST_GACC);
            for (int st = 0; st < nS; ++st)
                NMS_CUDA_TRY(launch_ray_totals(nrl, rb0, t.n_rays, t.ray_mirror, p.grid.n0, p.grid.n1, npg,
                                               t.d_Ftot_b + (size_t)st * F4g, (int64_t)nS * F4g,
                                               t.d_Gdil_b + (size_t)st * 16 * npg, (int64_t)nS * 16 * npg, p.n_rot - 1,
                                               p.d_Gtot + (size_t)st * 16 * np, p.d_Gdil + (size_t)st * 16 * np,
                                               p.d_Ftot + (size_t)st * F4, s));
            p.timer.end(ST_GACC, nS);
        } else if (t.objects) {
            p.timer.begin(ST_GACC);
            for (int st = 0; st < nS; ++st) {
                const double* Ts = t.d_Ftot_b + (size_t)st * F4;
                NMS_CUDA_TRY(launch_gacc_totals(Ts, nrl, (int64_t)nS * F4, np, p.d_Gtot + (size_t)st * 16 * np, s));
                if (rb0 + nrl == t.n_slots)
                    NMS_CUDA_TRY(cudaMemcpyAsync(p.d_Ftot + (size_t)st * F4, Ts + (size_t)(nrl - 1) * nS * F4,
                                                 F4 * sizeof(double), cudaMemcpyDeviceToDevice, s));
            }
            p.timer.end(ST_GACC, nS);
        }
    }
    return NMS_OK;
}

}  // namespace nms
