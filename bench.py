#!/usr/bin/env python3
"""Benchmark of the SANS Fourier-sum hot path on GB300.

One step = one pass of the whole hot path over the workload: rotation and
weights, the four Fourier sums (tensor-core split-FP16 GEMM on the separable
detector grid, or the FP32 direct sum), the Hermitian products, the
unpolarized and spin-flip cross sections, their azimuthal averages and the
correlation functions.  Metric: cell x q-point terms per second (one term =
one (cell, pixel) pair, all four channels, real and imaginary part).

Default workload: the micromagnetic-style box, 256 x 256 x 64 cells at 2 nm
(4.19M cells, smooth random M from 64 Fourier modes, 200 pores), 512 x 512
detector on [-2, 2]^2 nm^-1: 1.10e12 terms per step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl nms|reference]
                  [--precision auto|tc|direct|naive] [--workload box|sphere]

With --gpus N > 1 (torchrun) every rank evaluates its own replica of the
workload (weak scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cell·q-point terms/s of SANS Fourier sum: tensor-core split vs FP32 at 1e-6 err"

# FP32-pipe operations per term of the compensated direct-sum kernel counted
# from its source (phase 22, sincospif ~20, 8 FMA, two-float fold 7).
DIRECT_OPS_PER_TERM = 57
# Executed tensor flops per term of the split-FP16 GEMM: 3 products x 32 flops.
TC_FLOPS_PER_TERM = 96
# DRAM bytes (read + write) the GEMM moves per byte of phase tables it
# consumes, from an ncu capture of one launch on the 64x64x64 box (512^2
# detector); the box workloads scale it by their own table bytes per launch.
TC_DRAM_PER_TABLE_BYTE = 1.329   # 8.559 GB for 6.442 GB of tables (ncu, box64)
TC_TRAFFIC_WORKLOADS = ("box", "box64")


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
        "fallback"


# ----------------------------------------------------------------- workloads
def make_workload(name, n_spheres=10000):
    from paper_2601_18444_gb300 import inputs as I
    if name == "box":
        f = I.box_field(256, 256, 64, a=2.0, n_modes=64, kmax=0.2, n_pores=200, seed=1)
        grid = dict(kind="cartesian", n0=512, n1=512, lo0=-2.0, hi0=2.0, lo1=-2.0, hi1=2.0)
        edges = np.linspace(0.0, 2.0, 129)
        r = np.linspace(0.0, 600.0, 64)
        desc = "box 256x256x64 cells a=2nm (4.19M), 64 modes k<=0.2, 200 pores; 512x512 detector [-2,2]^2 nm^-1"
    elif name == "box64":
        # small case of the same kernels for profiler captures (262k cells)
        f = I.box_field(64, 64, 64, a=2.0, n_modes=64, kmax=0.2, n_pores=20, seed=1)
        grid = dict(kind="cartesian", n0=512, n1=512, lo0=-2.0, hi0=2.0, lo1=-2.0, hi1=2.0)
        edges = np.linspace(0.0, 2.0, 129)
        r = np.linspace(0.0, 200.0, 64)
        desc = "box 64x64x64 cells a=2nm (262k), 512x512 detector [-2,2]^2 nm^-1 (profiling case)"
    elif name == "sphere":
        f = I.sphere_vortex(16.0, 2.0, seed=0)
        grid = dict(kind="cartesian", n0=128, n1=128, lo0=-1.0, hi0=1.0, lo1=-1.0, hi1=1.0)
        edges = np.linspace(0.0, 1.0, 65)
        r = np.linspace(0.0, 40.0, 64)
        desc = "sphere R=16nm a=2nm (2109 cells) seeded vortex; 128x128 detector [-1,1]^2 nm^-1"
    elif name == "ensemble":
        f = I.sphere_ensemble(n_spheres=n_spheres, median=8.0, sigma=0.35, clip=(5.0, 20.0), a=1.0, cube=2000.0,
                              seed=3)
        grid = dict(kind="cartesian", n0=256, n1=256, lo0=-1.0, hi0=1.0, lo1=-1.0, hi1=1.0)
        edges = np.linspace(0.0, 1.0, 129)
        r = np.linspace(0.0, 60.0, 64)
        desc = (f"ensemble of {n_spheres} spheres, lognormal R (median 8nm, sigma 0.35, 5-20nm) a=1nm ({f.n} cells), "
                "Neel-like canting, 2um cube; 256x256 detector [-1,1]^2 nm^-1; dilute + total + interference")
        return f, grid, edges, r, desc, None, True
    elif name == "rotations":
        f = I.ellipsoid_uniform((40.0, 25.0, 25.0), a=0.8, seed=4)
        rot = I.random_rotations(4096, seed=5)
        grid = dict(kind="cartesian", n0=256, n1=256, lo0=-2.0, hi0=2.0, lo1=-2.0, hi1=2.0)
        edges = np.geomspace(0.01, 2.0, 129)
        r = np.linspace(0.0, 120.0, 64)
        desc = (f"ellipsoid 40/25/25nm a=0.8nm ({f.n} cells) uniform M, 4096 random orientations (Shoemake); "
                "256x256 detector [-2,2]^2 nm^-1; 128 log bins 0.01-2 nm^-1")
        return f, grid, edges, r, desc, rot, False
    else:
        raise SystemExit(f"unknown workload {name}")
    return f, grid, edges, r, desc, None, False


# ----------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, max_mhz):
        sm = []
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                max_mhz = mx
            except (ValueError, IndexError):
                continue
            for k, v in zip(names, r[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(k)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max_mhz,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------- oracle timing
def oracle_sample_rate(field, grid_kw, target_s=12.0, seed=0, R=None):
    """Oracle terms/s on a random sample of pixels (all cells, rotation R, object
    centres applied); returns (rate, sample, F_ref, idx, threads)."""
    from oracle import sans as S
    kw = dict(grid_kw)
    kind = kw.pop("kind")
    g = S.q_grid(kind, **kw)
    rng = np.random.default_rng(seed)
    R = np.eye(3) if R is None else R
    w = S.cell_weights(field.vol, field.nuc, field.mag, R)
    pr = S.rotate_cells(field.pos, R, field.offsets, field.centers)
    Y, Z = pr[:, 1].copy(), pr[:, 2].copy()
    del pr
    npix = g[0].shape[0]
    probe = rng.choice(npix, size=min(8, npix), replace=False)
    t0 = time.perf_counter()
    S.dsft(Y, Z, w, g[0][probe], g[1][probe])
    dt = max(time.perf_counter() - t0, 1e-4)
    per_pix = dt / len(probe)
    n_s = int(max(8, min(npix, target_s / per_pix)))
    idx = np.sort(rng.choice(npix, size=n_s, replace=False))
    t0 = time.perf_counter()
    F = S.dsft(Y, Z, w, g[0][idx], g[1][idx])
    dt = time.perf_counter() - t0
    terms = float(n_s) * field.n
    return terms / dt, f"{n_s} random pixels x {field.n} cells (seed {seed}), {dt:.1f} s", F, idx, S.oracle_threads()


# ----------------------------------------------------------------- dist helpers
def dist_setup(n_gpus):
    rank, world = 0, 1
    if n_gpus > 1 or "RANK" in os.environ:
        import torch.distributed as dist
        world = int(os.environ.get("WORLD_SIZE", "1"))
        rank = int(os.environ.get("RANK", "0"))
        if world > 1:
            import torch
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
            dist.init_process_group(backend=backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job(units_per_rank, ms_local, world):
    """(slowest rank's time in ms, aggregate rate of all ranks' units per s):
    every rank processes the same units (replicas, weak scaling)."""
    ms = max_over_ranks(ms_local, world)
    return ms, world * units_per_rank / (ms * 1e-3)


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world = dist_setup(args.gpus)
    if rank != 0:
        return 0
    field, grid_kw, edges, r, desc, rot, dilute = make_workload(args.workload)
    from oracle import sans as S
    kw = dict(grid_kw)
    kind = kw.pop("kind")
    g = S.q_grid(kind, **kw)
    w = S.cell_weights(field.vol, field.nuc, field.mag, np.eye(3))
    Y, Z = field.pos[:, 1].copy(), field.pos[:, 2].copy()
    rng = np.random.default_rng(1)
    npix = g[0].shape[0]
    n_s = min(npix, 48 if field.n > 1e6 else npix)
    times = []
    for it in range(args.warmup + args.steps):
        idx = rng.choice(npix, size=n_s, replace=False)
        t0 = time.perf_counter()
        S.dsft(Y, Z, w, g[0][idx], g[1][idx])
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
    terms = float(n_s) * field.n
    rate = terms * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "terms/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "sample": f"{n_s} random pixels x {field.n} cells per step"},
            "cpu_baseline": {"value": rate, "unit": "terms/s", "cores": S.oracle_threads(), "kind": "oracle",
                             "sample": f"{n_s} random pixels x {field.n} cells per step"},
            "e2e": {"value": rate, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------- main arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="nms", choices=["nms", "reference"])
    ap.add_argument("--precision", default="auto", choices=["auto", "tc", "direct", "naive"])
    ap.add_argument("--workload", default="box",
                    choices=["box", "box64", "sphere", "ensemble", "rotations", "post2d", "surrogate"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--kc", type=int, default=0, help="cells per TMEM accumulation chunk (0: library default)")
    ap.add_argument("--workspace-gb", type=float, default=0.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--spheres", type=int, default=10000, help="ensemble: number of spheres")
    ap.add_argument("--items-per-sm", type=int, default=0, help="tensor path: GEMM work items per SM (0: library)")
    ap.add_argument("--single-sum", action="store_true",
                    help="ensemble: the same cells as one sum (centres applied, no per-object amplitudes)")
    ap.add_argument("--sets", type=int, default=1,
                    help="loop mode: S magnetization states of the workload along a field sweep in one plan")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2601_18444_gb300 import nms

    rank, world = dist_setup(args.gpus)
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    nms.load()
    if args.workload == "post2d":
        return run_post2d(args, rank, world, dev)
    if args.workload == "surrogate":
        return run_surrogate(args, rank, world, dev)
    field, grid_kw, edges, r, desc, rot, dilute = make_workload(args.workload, args.spheres)
    if args.single_sum and field.offsets is not None:
        # batching overhead reference: every cell moved to its object's centre, one summand
        from paper_2601_18444_gb300 import inputs as I
        cen = np.repeat(field.centers, np.diff(field.offsets), axis=0) if field.centers is not None else 0.0
        field = I.Field(field.pos + cen, field.vol, field.nuc, field.mag, name=field.name)
        dilute = False
        desc += "; one sum over all cells (no per-object amplitudes)"
    field0 = field
    if args.sets > 1:
        from paper_2601_18444_gb300 import inputs as I
        nuc_s, mag_s = I.field_sweep(field, np.linspace(0.0, 2.0, args.sets))
        field0 = I.Field(field.pos, field.vol, nuc_s[0], mag_s[0], field.offsets, field.centers, field.name)
        field = I.Field(field.pos, field.vol, nuc_s, mag_s, field.offsets, field.centers, field.name)
        desc += f"; loop mode: {args.sets} magnetization states (field sweep h = 0..2) in one plan"
    prec = {"auto": nms.PREC_AUTO, "tc": nms.PREC_TC_F16X3, "direct": nms.PREC_FP32_DIRECT,
            "naive": nms.PREC_FP32_NAIVE}[args.precision]
    stream = torch.cuda.current_stream()
    g = nms.make_grid(**grid_kw)
    opt = nms.nms_options_default(precision=prec, timing=1, kc_cells=args.kc, want_dilute=1 if dilute else 0,
                                  workspace_bytes=int(args.workspace_gb * (1 << 30)), n_sets=max(1, args.sets),
                                  split_k=args.items_per_sm)
    plan = nms.plan_from_field(field, g, opt, rot=rot, stream=stream.cuda_stream)
    npix = plan.npix
    n_rot = 1 if rot is None else len(rot)
    # with the dilute split the per-object form factors are the summed terms
    terms = float(field.n) * npix * n_rot * max(1, args.sets)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    img_u = torch.empty(npix, dtype=torch.float64, device="cuda")
    img_s = torch.empty(npix, dtype=torch.float64, device="cuda")
    r_dev = torch.tensor(r, dtype=torch.float64, device="cuda")

    def step():
        nms.nms_amplitudes(plan)
        nms.nms_response(plan, "UNPOL", out=img_u)
        nms.nms_response(plan, "SF", out=img_s)
        out = []
        for img in (img_u, img_s):
            I, c, qm = nms.nms_azimuthal_average(plan, img, edges)
            cc, pp = nms.nms_correlation(qm, I, r, stream=stream.cuda_stream)
            out.append((I, cc, pp))
        return out

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    nms.nms_plan_stage_ms(plan, reset=True)
    peaks, peak_src = load_peaks()
    times = []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            flush.fill_(1)                       # L2 flush between timed steps (256 MB > 129 MB L2)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    barrier(world)
    stage = nms.nms_plan_stage_ms(plan)
    ms_step, value = whole_job(terms, float(np.mean(times)), world)
    launches_per_step = sum(v[1] for v in stage.values()) / args.steps + 2 + 2 + 4
    clocks = clk.summary(peaks.get("sm_max_mhz", 2070.0))

    # dominant kernel roofline
    if plan_path_is_tc(stage):
        k_ms = stage["gemm"][0] / args.steps
        achieved = terms * TC_FLOPS_PER_TERM / (k_ms * 1e-3) / 1e12
        peak = peaks.get("bf16_tflops", 1900.0)
        traffic = None
        if TC_DRAM_PER_TABLE_BYTE and args.workload in TC_TRAFFIC_WORKLOADS and args.sets <= 1:
            traffic = TC_DRAM_PER_TABLE_BYTE * table_bytes(field, grid_kw, n_rot) / (stage["gemm"][1] / args.steps)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
                "kernel": "k_gemm_f16x3", "peak_source": f"{peak_src} bf16 dense (f16 same rate)"}
    else:
        k_ms = stage["direct"][0] / args.steps
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
        peak = sms * 128 * mhz * 1e6 / 1e12
        achieved = terms * DIRECT_OPS_PER_TERM / (k_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": None, "kernel": "k_direct<compensated>",
                "peak_source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz (median SM clock under load)"}

    # error on a sample of pixels vs the oracle, and the oracle's own rate
    cpu = None
    err = None
    if rank == 0 and not args.no_cpu_baseline:
        R_last = np.eye(3) if rot is None else rot[-1]
        rate, sample, F_ref, idx, cores = oracle_sample_rate(field0, grid_kw, args.cpu_seconds, R=R_last)
        F = nms.nms_get_amplitudes(plan)       # weight set 0
        from oracle import sans as S
        wsum = np.abs(S.cell_weights(field0.vol, field0.nuc, field0.mag, R_last)).sum(1)
        err = [float(np.max(np.abs(F[c][idx] - F_ref[c])) / wsum[c]) if wsum[c] > 0 else 0.0 for c in range(4)]
        cpu = {"value": rate, "unit": "terms/s", "cores": cores, "kind": "oracle", "sample": sample}

    # end to end through the C ABI from pinned host buffers (the timed plan is
    # released first: every e2e step creates and destroys its own)
    plan.close()
    e2e = None
    if args.steps > 0 and not args.no_e2e:
        pin = {}
        for k in ("pos", "vol", "nuc", "mag"):
            a = getattr(field, k)
            t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
            t.numpy()[...] = a
            pin[k] = t.numpy()
        out_u = torch.empty(npix, dtype=torch.float64, pin_memory=True).numpy()
        out_s = torch.empty(npix, dtype=torch.float64, pin_memory=True).numpy()
        e2e_times = []
        for _ in range(3):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            p2 = nms.nms_plan_create(pin["pos"], pin["vol"], pin["nuc"], pin["mag"], field.offsets, field.centers,
                                     rot, grid=g, opt=opt, stream=stream.cuda_stream)
            nms.nms_amplitudes(p2)
            nms.nms_response(p2, "UNPOL", out=out_u)
            nms.nms_response(p2, "SF", out=out_s)
            for img in (out_u, out_s):
                I, c, qm = nms.nms_azimuthal_average(p2, img, edges)
                nms.nms_correlation(qm, I, r)
            p2.close()
            torch.cuda.synchronize()
            e2e_times.append(time.perf_counter() - t0)
        t_e2e = max_over_ranks(min(e2e_times), world)
        h2d = sum(pin[k].nbytes for k in pin)
        d2h = 2 * npix * 8
        e2e = {"value": world * terms / t_e2e, "unit": "terms/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "s_per_step": t_e2e}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f16x3->f32(two-float)" if plan_path_is_tc(stage) else "f32(two-float)",
                "data": "synthetic",
                "config": {"workload": desc, "parallelism": f"replicas x{world}", "l2": "flushed between steps",
                           "precision": args.precision, "terms_per_step": terms,
                           "stage_ms_per_step": {k: v[0] / args.steps for k, v in stage.items() if v[1]}},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(round(launches_per_step
                                                                                           * args.steps)),
                "clocks": clocks, "amp_err_vs_oracle": err}
        print(json.dumps(line), flush=True)
    return 0


def table_bytes(field, grid_kw, n_rot):
    """Bytes of split-FP16 phase tables one step writes and the GEMM reads:
    per 32-cell k-block, (A tiles + B tiles) x (hi, lo) x 16 KB."""
    mt = -(-4 * grid_kw["n0"] // 128)
    nt = -(-2 * grid_kw["n1"] // 128)
    if field.offsets is not None and len(field.offsets) > 2:
        nkb = int(sum(-(-(b - a) // 32) for a, b in zip(field.offsets[:-1], field.offsets[1:])))
    else:
        nkb = -(-field.n // 32)
    return float(nkb * n_rot * (mt + nt) * 2 * 16384)


# FP32-pipe operations per (pixel, output point) term of k_corr2d, counted
# from its source (two-float phase and exact reduction 16, sincospif ~20,
# 2 FMA, two-float fold of 8-term partials ~2).
CORR2D_OPS_PER_TERM = 40


def run_post2d(args, rank, world, dev):
    """2D post-processing of the box's unpolarized image: the angular spectrum
    (kmax 16 on 128 ring bins) and the 2D correlation C(rho, alpha) on a
    64 x 64 output grid, timed with CUDA events; one step = both calls."""
    import torch
    from paper_2601_18444_gb300 import nms
    field, grid_kw, edges, r, desc, rot, dilute = make_workload("box")
    stream = torch.cuda.current_stream()
    plan = nms.plan_from_field(field, nms.make_grid(**grid_kw), nms.nms_options_default(), stream=stream.cuda_stream)
    nms.nms_amplitudes(plan)
    npix = plan.npix
    img = torch.empty(npix, dtype=torch.float64, device="cuda")
    nms.nms_response(plan, "UNPOL", out=img)
    rho = np.linspace(0.0, 300.0, 64)
    alpha = np.linspace(0.0, np.pi, 64, endpoint=False)
    C = torch.empty((64, 64, 2), dtype=torch.float64, device="cuda")
    terms = float(npix) * 64 * 64
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        nms.nms_angular_spectrum(plan, img, kmax=16, bin_edges=edges)
        nms.nms_correlation_2d(plan, img, rho, alpha, out=C)

    def corr_only():
        nms.nms_correlation_2d(plan, img, rho, alpha, out=C)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    peaks, _ = load_peaks()
    times, tcorr = [], []
    barrier(world)
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            step()
            e1.record(stream)
            corr_only()
            e2.record(stream)
            e2.synchronize()
            times.append(e0.elapsed_time(e1))
            tcorr.append(e1.elapsed_time(e2))
    barrier(world)
    ms = max_over_ranks(float(np.mean(times)), world)
    ms_corr = float(np.mean(tcorr))
    clocks = clk.summary(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    peak = sms * 128 * mhz * 1e6 / 1e12
    achieved = terms * CORR2D_OPS_PER_TERM / (ms_corr * 1e-3) / 1e12
    # end to end: host image in, host results out
    img_h = img.cpu().numpy()
    t0 = time.perf_counter()
    for _ in range(2):
        nms.nms_angular_spectrum(plan, img_h, kmax=16, bin_edges=edges)
        nms.nms_correlation_2d(plan, img_h, rho, alpha)
    t_e2e = (time.perf_counter() - t0) / 2
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle's 2D correlation on a bounded sample of output points
        from oracle import sans as S
        q0 = np.linspace(grid_kw["lo0"], grid_kw["hi0"], grid_kw["n0"])
        q1 = np.linspace(grid_kw["lo1"], grid_kw["hi1"], grid_kw["n1"])
        n_s, t0, dt = 0, time.perf_counter(), 0.0
        while dt < 3.0:
            S.correlation_2d_cartesian(img_h, q0, q1, rho[n_s % 64:n_s % 64 + 1], alpha[:4])
            n_s += 4
            dt = time.perf_counter() - t0
        cpu = {"value": n_s * npix / dt, "unit": "terms/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"{n_s} output points x {npix} pixels, {dt:.1f} s (numpy with its BLAS threads)"}
    if rank == 0:
        line = {"metric": "pixel x output-point terms/s of the 2D correlation (Eq. crav2d) with the angular spectrum",
                "value": world * terms / (ms * 1e-3), "unit": "terms/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32(two-float)", "data": "synthetic",
                "config": {"workload": "UNPOL image of " + desc + "; angular spectrum kmax 16 on 128 ring bins; "
                                       "C(rho, alpha) on 64 rho in [0, 300] nm x 64 alpha in [0, pi)",
                           "parallelism": f"replicas x{world}", "l2": "flushed between steps",
                           "corr2d_ms": ms_corr},
                "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                             "frac": achieved / peak, "traffic": None, "kernel": "k_corr2d",
                             "peak_source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz"},
                "cpu_baseline": cpu,
                "e2e": {"value": world * terms / t_e2e, "unit": "terms/s", "h2d_bytes_per_step": 2 * npix * 8,
                        "d2h_bytes_per_step": 64 * 64 * 16 + 17 * 128 * 16 + 128 * 16 + 17 * 16},
                "gpu_launches": args.steps * 7, "clocks": clocks}
        print(json.dumps(line), flush=True)
    plan.close()
    return 0


# Tensor flops of one MLP step per sample, 6 -> H -> H -> n_out: forward
# 2 (6 H + H^2 + H n_out); training adds about twice that for the backward GEMMs.
def mlp_flops(n_in, H, n_out):
    return 2.0 * (n_in * H + H * H + H * n_out)


def run_surrogate(args, rank, world, dev):
    """Learned surrogate (scaled-down vortex family): training curves from the
    batched transform, then timed training epochs and timed inference on 2^20
    queries; the MLP GEMMs against the bf16 dense peak."""
    import torch
    from paper_2601_18444_gb300 import inputs as I
    from paper_2601_18444_gb300 import nms
    from paper_2601_18444_gb300 import surrogate as SG
    edges = np.geomspace(0.04, 1.2, 65)
    params = I.vortex_family_params(2048, seed=21)
    t0 = time.perf_counter()
    Iq, _, t_tr, terms_tr = SG.generate_curves(params, edges, a=2.5, n_rot=16)
    ok = np.all(np.isfinite(Iq), axis=0)
    Y = torch.tensor(SG.log_targets(Iq[:, ok]), device="cuda")
    X = torch.tensor(params.astype(np.float32), device="cuda")
    n_out, H = int(ok.sum()), 256
    lo = I.VORTEX_FAMILY_BOUNDS[:, 0].astype(np.float32)
    hi = I.VORTEX_FAMILY_BOUNDS[:, 1].astype(np.float32)
    s = nms.nms_surrogate_create(6, H, n_out, lo, hi, seed=3, stream=torch.cuda.current_stream().cuda_stream)
    nms.nms_surrogate_train(s, X, Y, batch=128, epochs=max(1, args.warmup), lr=1e-3, seed=4)
    torch.cuda.synchronize()
    epochs = 20 * max(1, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        e0.record()
        nms.nms_surrogate_train(s, X, Y, batch=128, epochs=epochs, lr=1e-3, seed=5)
        e1.record()
        e1.synchronize()
        ms_train = e0.elapsed_time(e1)
        nq = 1 << 20
        q = torch.tensor(I.vortex_family_params(nq, seed=23).astype(np.float32), device="cuda")
        out = torch.empty((nq, n_out), device="cuda")   # 2^20 x n_out FP32 outputs: larger than L2
        for _ in range(max(3, args.warmup)):
            nms.nms_surrogate_infer(s, q, out)
        torch.cuda.synchronize()
        barrier(world)
        times = []
        for _ in range(max(1, args.steps)):
            e0.record()
            nms.nms_surrogate_infer(s, q, out)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        barrier(world)
    ms_inf, q_rate = whole_job(nq, float(np.mean(times)), world)
    peaks, peak_src = load_peaks()
    clocks = clk.summary(peaks.get("sm_max_mhz", 2070.0))
    f_inf = nq * mlp_flops(6, H, n_out)
    achieved = f_inf / (ms_inf * 1e-3) / 1e12
    peak = peaks.get("bf16_tflops", 1900.0)
    train_samples = epochs * len(params)
    if rank == 0:
        line = {"metric": "surrogate inference queries/s (MLP 6->256->256->n_out, bf16 GEMMs)",
                "value": q_rate, "unit": "queries/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_inf, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "bf16->f32", "data": "synthetic",
                "config": {"workload": f"vortex family, {len(params)} training curves from the batched transform "
                                       f"(a=2.5nm, 16 orientations, 128^2 detector, {n_out} log bins); "
                                       f"inference on 2^20 queries",
                           "curves_s": t_tr, "curve_terms_per_s": terms_tr / t_tr,
                           "train_samples_per_s": train_samples / (ms_train * 1e-3),
                           "exact_ms_per_curve": 1e3 * t_tr / len(params),
                           "surrogate_us_per_query": 1e3 * ms_inf / nq},
                "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                             "frac": achieved / peak, "traffic": None, "kernel": "k_mlp_infer (fused tcgen05 bf16)",
                             "peak_source": f"{peak_src} bf16 dense"},
                "cpu_baseline": None, "e2e": None,
                "gpu_launches": len(times) if (H == 256 and n_out <= 64) else None,   # one fused kernel per call
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    s.close()
    return 0


def plan_path_is_tc(stage):
    return stage.get("gemm", (0, 0))[1] > 0


if __name__ == "__main__":
    sys.exit(main())
