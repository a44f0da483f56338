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

  python bench.py [--steps K] [--warmup W] [--impl nms|reference]
                  [--precision auto|tc|direct|naive] [--workload box|...]

The library is single-GPU: with --gpus N > 1 (under torchrun) rank 0 prints
one "unavailable" line and every rank exits 0 without GPU work.  The
reference arm (--impl reference) times the FP64 CPU oracle on rank 0.

Besides the tensor path, the default line times the FP32 direct sum
(compensated and naive phase) on a sample of the same detector's pixels with
all cells: the metric compares the two at the 1e-6 error bar.
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
# Algorithmic flops per term of the Fourier sum: 4 channels x one complex
# multiply-add (8 real flops) per (cell, pixel).
ALGO_FLOPS_PER_TERM = 32
# DRAM bytes (read + write) the GEMM moves per byte of phase tables it
# consumes, from an ncu capture of one launch on the 64x64x64 box (512^2
# detector); the box workloads scale it by their own table bytes per launch.
TC_DRAM_PER_TABLE_BYTE = 1.134   # 3.045 GB for 2.684 GB of tables (ncu, box64)
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


# ----------------------------------------------------------------- launch
def launch_rank():
    """(rank, world) from torchrun's environment (1 process when absent)."""
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))


def unavailable_multi_gpu(args):
    """The library drives one GPU; a multi-GPU request prints one line on rank 0."""
    rank, world = launch_rank()
    if rank == 0:
        print(json.dumps({"metric": METRIC, "unavailable": f"single-GPU library: --gpus {args.gpus} "
                          f"(world size {world}) is not supported; run with --gpus 1",
                          "n_gpus": args.gpus}), flush=True)
    return 0


# ----------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world = launch_rank()
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
                    choices=["box", "box64", "sphere", "ensemble", "rotations", "post2d", "surrogate", "e4", "paper"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--kc", type=int, default=0, help="cells per TMEM accumulation chunk (0: library default)")
    ap.add_argument("--workspace-gb", type=float, default=0.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32-leg", action="store_true", help="skip the FP32 direct-sum comparison")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--spheres", type=int, default=10000, help="ensemble: number of spheres")
    ap.add_argument("--items-per-sm", type=int, default=0, help="tensor path: GEMM work items per SM (0: library)")
    ap.add_argument("--objects", action="store_true",
                    help="paper: the 800 particles as objects (dilute, total and interference parts)")
    ap.add_argument("--single-sum", action="store_true",
                    help="ensemble: the same cells as one sum (centres applied, no per-object amplitudes)")
    ap.add_argument("--sets", type=int, default=1,
                    help="loop mode: S magnetization states of the workload along a field sweep in one plan")
    ap.add_argument("--copies", type=int, default=0, help="e4: number of particle copies (0: the sweep)")
    ap.add_argument("--curves", type=int, default=2048, help="surrogate: training curves")
    ap.add_argument("--orientations", type=int, default=16, help="surrogate: orientations per curve")
    ap.add_argument("--bins", type=int, default=64, help="surrogate: log |q| bins")
    ap.add_argument("--qmin", type=float, default=0.04, help="surrogate: lower edge of the log bins (nm^-1)")
    ap.add_argument("--held-out", type=int, default=256, help="surrogate: held-out curves judged by the transform")
    ap.add_argument("--epochs", type=int, default=0, help="surrogate: timed training epochs (0: 20 x steps)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.gpus > 1 or launch_rank()[1] > 1:
        return unavailable_multi_gpu(args)

    import torch
    from paper_2601_18444_gb300 import nms

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    nms.load()
    if args.workload == "post2d":
        return run_post2d(args, dev)
    if args.workload == "surrogate":
        return run_surrogate(args, dev)
    if args.workload == "e4":
        return run_e4(args, dev)
    if args.workload == "paper":
        return run_paper_shape(args, dev)
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
    stage = nms.nms_plan_stage_ms(plan)
    ms_step = float(np.mean(times))
    value = terms / (ms_step * 1e-3)
    launches_per_step = sum(v[1] for v in stage.values()) / args.steps + 2 + 2 + 4
    clocks = clk.summary(peaks.get("sm_max_mhz", 2070.0))
    is_tc = plan_path_is_tc(stage)

    # dominant kernel roofline
    if is_tc:
        k_ms = stage["gemm"][0] / args.steps
        info = nms.nms_plan_info(plan)
        mirror = info.get("mirror", (0, 0))
        exec_per_term = 3 * ALGO_FLOPS_PER_TERM / ((2 if mirror[0] else 1) * (2 if mirror[1] else 1))
        achieved = terms * ALGO_FLOPS_PER_TERM / (k_ms * 1e-3) / 1e12
        executed = terms * exec_per_term / (k_ms * 1e-3) / 1e12
        peak = peaks.get("bf16_tflops", 1900.0)
        traffic = None
        if TC_DRAM_PER_TABLE_BYTE and args.workload in TC_TRAFFIC_WORKLOADS and args.sets <= 1:
            traffic = TC_DRAM_PER_TABLE_BYTE * table_bytes(field, grid_kw, n_rot) / (stage["gemm"][1] / args.steps)
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_unit": "bytes per launch",
                "kernel": "k_gemm_f16x3",
                "flops_per_term": ALGO_FLOPS_PER_TERM,
                "peak_source": f"{peak_src} bf16 dense (f16 same rate), burst",
                "executed": {"flops_per_term": exec_per_term, "tflops": executed, "frac": executed / peak,
                             "note": "3 split-FP16 MMAs per product; symmetric detector axes (q_y, q_z) "
                                     f"computed on their q >= 0 half: {mirror}"}}
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
    oracle_sample = None
    if not args.no_cpu_baseline:
        R_last = np.eye(3) if rot is None else rot[-1]
        rate, sample, F_ref, idx, cores = oracle_sample_rate(field0, grid_kw, args.cpu_seconds, R=R_last)
        F = nms.nms_get_amplitudes(plan)       # weight set 0
        from oracle import sans as S
        wsum = np.abs(S.cell_weights(field0.vol, field0.nuc, field0.mag, R_last)).sum(1)
        err = [float(np.max(np.abs(F[c][idx] - F_ref[c])) / wsum[c]) if wsum[c] > 0 else 0.0 for c in range(4)]
        cpu = {"value": rate, "unit": "terms/s", "cores": cores, "kind": "oracle", "sample": sample}
        oracle_sample = (idx, F_ref, wsum, R_last)
    plan.close()

    # the FP32 direct sum on the same box (compensated: the 1e-6 comparison;
    # naive: throughput and error only), on a sample of the detector's pixels
    fp32 = None
    if is_tc and not args.no_fp32_leg and args.sets <= 1 and not dilute and rot is None:
        fp32 = fp32_leg(nms, field0, grid_kw, stream, peaks, clocks, dev, oracle_sample)
        if fp32 is not None:
            fp32["tc_over_fp32_compensated"] = value / fp32["compensated"]["value"]

    # end to end through the C ABI from pinned host buffers (the timed plan is
    # released first: every e2e step creates and destroys its own)
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
        t_e2e = min(e2e_times)
        h2d = sum(pin[k].nbytes for k in pin)
        d2h = 2 * npix * 8
        e2e = {"value": terms / t_e2e, "unit": "terms/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "s_per_step": t_e2e}

    stage_ms = {k: v[0] / args.steps for k, v in stage.items() if v[1]}
    line = {"metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16x3->f32(two-float)" if is_tc else "f32(two-float)",
            "data": "synthetic",
            "config": {"workload": desc, "parallelism": "1 GPU", "l2": "flushed between steps",
                       "precision": args.precision, "terms_per_step": terms, "stage_ms_per_step": stage_ms,
                       "tables_over_gemm": (stage_ms.get("tables", 0.0) / stage_ms["gemm"]) if is_tc else None},
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "fp32_direct": fp32,
            "gpu_launches": int(round(launches_per_step * args.steps)),
            "clocks": clocks, "amp_err_vs_oracle": err}
    print(json.dumps(line), flush=True)
    return 0


def fp32_leg(nms, field, grid_kw, stream, peaks, clocks, dev, oracle_sample, n_pix=8192, reps=3):
    """Compensated and naive FP32 direct sums of the workload's cells on a
    random sample of its detector pixels (a LIST grid; the oracle's pixels
    first, so their error is measured): terms/s, error against the oracle and
    the compensated kernel's FP32-lane roofline."""
    import torch
    from oracle import sans as S
    kw = dict(grid_kw)
    kind = kw.pop("kind")
    qy, qz = S.q_grid(kind, **kw)[:2]
    npix = qy.shape[0]
    rng = np.random.default_rng(11)
    first = oracle_sample[0] if oracle_sample is not None else np.zeros(0, dtype=np.int64)
    rest = rng.choice(np.setdiff1d(np.arange(npix), first), size=max(0, min(n_pix, npix) - len(first)),
                      replace=False)
    idx = np.concatenate([first, rest]).astype(np.int64)
    ql = np.stack([qy[idx], qz[idx]], axis=1)
    g = nms.make_grid("list", len(idx), qlist=ql)
    terms = float(field.n) * len(idx)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    lanes_peak = sms * 128 * mhz * 1e6 / 1e12
    res = {"sample": f"{len(idx)} random pixels of the same detector x {field.n} cells (LIST grid)"}
    for name, prec in (("compensated", nms.PREC_FP32_DIRECT), ("naive", nms.PREC_FP32_NAIVE)):
        plan = nms.plan_from_field(field, g, nms.nms_options_default(precision=prec), stream=stream.cuda_stream)
        nms.nms_amplitudes(plan)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nms.nms_amplitudes(plan)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = float(np.mean(ts))
        r = {"value": terms / (ms * 1e-3), "unit": "terms/s", "ms": ms}
        if oracle_sample is not None and len(first):
            F = nms.nms_get_amplitudes(plan)
            F_ref, wsum = oracle_sample[1], oracle_sample[2]
            r["amp_err_vs_oracle"] = [float(np.max(np.abs(F[c][:len(first)] - F_ref[c])) / wsum[c])
                                      if wsum[c] > 0 else 0.0 for c in range(4)]
        if name == "compensated":
            achieved = terms * DIRECT_OPS_PER_TERM / (ms * 1e-3) / 1e12
            r["roofline"] = {"bound": "alu", "achieved": achieved, "peak": lanes_peak, "unit": "Tops/s",
                             "frac": achieved / lanes_peak, "ops_per_term": DIRECT_OPS_PER_TERM,
                             "peak_source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz"}
        res[name] = r
        plan.close()
    return res


def gemm_axis(n, lo, hi):
    """Nodes of one detector axis the GEMM covers: the q >= 0 half of an axis
    symmetric about q = 0, else all of them."""
    return n - n // 2 if (n >= 2 and lo == -hi) else n


def table_bytes(field, grid_kw, n_rot):
    """Bytes of split-FP16 phase tables one step writes and the GEMM reads:
    per 64-cell k-block, (A tiles + B tiles) x (hi, lo) x 16 KB, with A rows
    (q_y node, channel) x (cos, sin) and B rows q_z node x (cos, sin)."""
    mt = -(-8 * gemm_axis(grid_kw["n0"], grid_kw["lo0"], grid_kw["hi0"]) // 128)
    nt = -(-2 * gemm_axis(grid_kw["n1"], grid_kw["lo1"], grid_kw["hi1"]) // 128)
    if field.offsets is not None and len(field.offsets) > 2:
        nkb = int(sum(-(-(b - a) // 64) for a, b in zip(field.offsets[:-1], field.offsets[1:])))
    else:
        nkb = -(-field.n // 64)
    return float(nkb * n_rot * (mt + nt) * 2 * 16384)


# FP32-pipe operations per (pixel, output point) term of k_corr2d, counted
# from its source (two-float phase and exact reduction 16, sincospif ~20,
# 2 FMA, two-float fold of 8-term partials ~2).
CORR2D_OPS_PER_TERM = 40


def run_post2d(args, dev):
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
    ms = float(np.mean(times))
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
    if not args.no_cpu_baseline:
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
    line = {"metric": "pixel x output-point terms/s of the 2D correlation (Eq. crav2d) with the angular spectrum",
            "value": terms / (ms * 1e-3), "unit": "terms/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32(two-float)", "data": "synthetic",
            "config": {"workload": "UNPOL image of " + desc + "; angular spectrum kmax 16 on 128 ring bins; "
                                   "C(rho, alpha) on 64 rho in [0, 300] nm x 64 alpha in [0, pi)",
                       "parallelism": "1 GPU", "l2": "flushed between steps",
                       "corr2d_ms": ms_corr},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "k_corr2d",
                         "peak_source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz"},
            "cpu_baseline": cpu,
            "e2e": {"value": terms / t_e2e, "unit": "terms/s", "h2d_bytes_per_step": 2 * npix * 8,
                    "d2h_bytes_per_step": 64 * 64 * 16 + 17 * 128 * 16 + 128 * 16 + 17 * 16},
            "gpu_launches": args.steps * 7, "clocks": clocks}
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


# Tensor flops of one MLP step per sample, 6 -> H -> H -> n_out: forward
# 2 (6 H + H^2 + H n_out); training adds about twice that for the backward GEMMs.
def mlp_flops(n_in, H, n_out):
    return 2.0 * (n_in * H + H * H + H * n_out)


def run_surrogate(args, dev):
    """Learned surrogate on the vortex family: training curves from the
    batched transform (orientation-averaged unpolarized I(q) on log |q| bins),
    timed training epochs, the held-out error against the transform, and
    timed inference on 2^20 queries; the MLP GEMMs against the bf16 dense
    peak.  Default: a scaled-down family (2048 curves x 16 orientations, 64
    bins); --curves 200000 --orientations 256 --bins 128 runs the stated
    scale (members built by spawned worker processes, chunks of 8000 per
    plan)."""
    import torch
    from paper_2601_18444_gb300 import inputs as I
    from paper_2601_18444_gb300 import nms
    from paper_2601_18444_gb300 import surrogate as SG
    edges = np.geomspace(args.qmin, 1.2, args.bins + 1)
    a_lat = 2.5
    params = I.vortex_family_params(args.curves, seed=21)
    p_test = I.vortex_family_params(args.held_out, seed=22)
    big = args.curves > 4096
    t_host = 0.0
    if big:
        Iq, _, t_tr, terms_tr, t_host = SG.generate_curves_chunked(params, edges, a=a_lat, n_rot=args.orientations)
        I_te, _, t_te, terms_te, _ = SG.generate_curves_chunked(p_test, edges, a=a_lat, n_rot=args.orientations)
    else:
        Iq, _, t_tr, terms_tr = SG.generate_curves(params, edges, a=a_lat, n_rot=args.orientations)
        I_te, _, t_te, terms_te = SG.generate_curves(p_test, edges, a=a_lat, n_rot=args.orientations)
    ok = np.all(np.isfinite(Iq), axis=0) & np.all(np.isfinite(I_te), axis=0)
    Y_tr, Y_te = SG.log_targets(Iq[:, ok]), SG.log_targets(I_te[:, ok])
    Y = torch.tensor(Y_tr, device="cuda")
    X = torch.tensor(params.astype(np.float32), device="cuda")
    n_out, H = int(ok.sum()), 256
    lo = I.VORTEX_FAMILY_BOUNDS[:, 0].astype(np.float32)
    hi = I.VORTEX_FAMILY_BOUNDS[:, 1].astype(np.float32)
    s = nms.nms_surrogate_create(6, H, n_out, lo, hi, seed=3, stream=torch.cuda.current_stream().cuda_stream)
    nms.nms_surrogate_train(s, X, Y, batch=128, epochs=max(1, args.warmup), lr=1e-3, seed=4)
    torch.cuda.synchronize()
    epochs = args.epochs if args.epochs > 0 else 20 * max(1, args.steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        e0.record()
        loss = nms.nms_surrogate_train(s, X, Y, batch=128, epochs=epochs, lr=1e-3, seed=5)
        e1.record()
        e1.synchronize()
        ms_train = e0.elapsed_time(e1)
        # held-out error against the exact transform
        Xt = torch.tensor(p_test.astype(np.float32), device="cuda")
        pred_t = torch.empty((len(p_test), n_out), device="cuda")
        nms.nms_surrogate_infer(s, Xt, pred_t)
        pred = pred_t.cpu().numpy()
        rms = float(np.sqrt(np.mean((pred - Y_te) ** 2)))
        rms_mean = float(np.sqrt(np.mean((Y_tr.mean(0) - Y_te) ** 2)))
        nq = 1 << 20
        q = torch.tensor(I.vortex_family_params(nq, seed=23).astype(np.float32), device="cuda")
        out = torch.empty((nq, n_out), device="cuda")   # 2^20 x n_out FP32 outputs: larger than L2
        for _ in range(max(3, args.warmup)):
            nms.nms_surrogate_infer(s, q, out)
        torch.cuda.synchronize()
        times = []
        for _ in range(max(1, args.steps)):
            e0.record()
            nms.nms_surrogate_infer(s, q, out)
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
    ms_inf = float(np.mean(times))
    q_rate = nq / (ms_inf * 1e-3)
    peaks, peak_src = load_peaks()
    clocks = clk.summary(peaks.get("sm_max_mhz", 2070.0))
    f_inf = nq * mlp_flops(6, H, n_out)
    achieved = f_inf / (ms_inf * 1e-3) / 1e12
    peak = peaks.get("bf16_tflops", 1900.0)
    train_samples = epochs * len(params)
    exact_ms = 1e3 * t_te / len(p_test)
    line = {"metric": "surrogate inference queries/s (MLP 6->256->256->n_out, bf16 GEMMs)",
            "value": q_rate, "unit": "queries/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_inf, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16->f32", "data": "synthetic",
            "config": {"workload": f"vortex family, {len(params)} training curves from the batched transform "
                                   f"(a={a_lat}nm, {args.orientations} orientations, 128^2 detector [-1.2,1.2]^2, "
                                   f"{args.bins} log bins {args.qmin}-1.2 nm^-1, {n_out} non-empty in every curve); "
                                   f"{len(p_test)} held-out curves; inference on 2^20 queries",
                       "curves_s": t_tr, "curve_terms_per_s": terms_tr / t_tr, "host_wait_s": t_host,
                       "train_epochs": epochs, "train_samples_per_s": train_samples / (ms_train * 1e-3),
                       "train_loss": loss,
                       "held_out_rms_dex": rms, "mean_curve_rms_dex": rms_mean,
                       "exact_ms_per_curve": exact_ms, "surrogate_us_per_query": 1e3 * ms_inf / nq,
                       "speedup_per_query": exact_ms * 1e-3 / (ms_inf * 1e-3 / nq)},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None, "kernel": "k_mlp_infer (fused tcgen05 bf16)",
                         "peak_source": f"{peak_src} bf16 dense"},
            "cpu_baseline": None, "e2e": None,
            # the fused kernel runs once per 128 outputs of each call
            "gpu_launches": len(times) * -(-n_out // 128) if (H == 256 and n_out <= 256) else None,
            "clocks": clocks}
    print(json.dumps(line), flush=True)
    s.close()
    return 0


def lattice_copies(particle, n_copies, spacing=45.0, objects=False):
    """n_copies of a particle on the simple-cubic sites (spacing in nm)
    nearest the origin, as one field (one sum over all cells), or with
    objects=True as n_copies objects (local positions, the sites as centres)."""
    from paper_2601_18444_gb300 import inputs as I
    side = int(np.ceil(n_copies ** (1.0 / 3.0))) + 2
    ax = (np.arange(side) - (side - 1) / 2.0) * spacing
    sites = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), axis=-1).reshape(-1, 3)
    sites = sites[np.argsort(np.linalg.norm(sites, axis=1), kind="stable")[:n_copies]]
    n = particle.n
    if objects:
        return I.Field(np.tile(particle.pos, (n_copies, 1)), np.tile(particle.vol, n_copies),
                       np.tile(particle.nuc, n_copies), np.tile(particle.mag, (n_copies, 1)),
                       offsets=np.arange(n_copies + 1, dtype=np.int64) * n, centers=sites,
                       name=f"{particle.name}_x{n_copies}_objects")
    pos = (particle.pos[None, :, :] + sites[:, None, :]).reshape(-1, 3)
    return I.Field(pos, np.tile(particle.vol, n_copies), np.tile(particle.nuc, n_copies),
                   np.tile(particle.mag, (n_copies, 1)), name=f"{particle.name}_x{n_copies}")


E4_COPIES = (10, 40, 160, 640, 2560, 10240, 25600)


def run_e4(args, dev):
    """Runtime-scaling shape of the paper's runtime experiment: N identical
    D = 40 nm linear-vortex spheres (a = 2 nm, 4169 cells) on a 45 nm simple
    cubic lattice, N = 10 ... 25,600 (4.2e4 ... 1.07e8 cells), one sum over
    all cells on a 256^2 detector [-1.5, 1.5]^2 nm^-1 (tensor path).  One step
    = amplitudes + the unpolarized image + its azimuthal average; terms/s
    against the total cell count W."""
    import torch
    from paper_2601_18444_gb300 import inputs as I
    from paper_2601_18444_gb300 import nms
    particle = I.linear_vortex_sphere(20.0, 2.0, normalised=True)
    grid_kw = dict(kind="cartesian", n0=256, n1=256, lo0=-1.5, hi0=1.5, lo1=-1.5, hi1=1.5)
    g = nms.make_grid(**grid_kw)
    edges = np.linspace(0.0, 1.5, 129)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    peaks, _ = load_peaks()
    copies = (args.copies,) if args.copies > 0 else E4_COPIES
    sweep = []
    with ClockSampler(dev) as clk:
        for nc in copies:
            f = lattice_copies(particle, nc)
            plan = nms.plan_from_field(f, g, nms.nms_options_default(timing=1), stream=stream.cuda_stream)
            img = torch.empty(plan.npix, dtype=torch.float64, device="cuda")

            def step():
                nms.nms_amplitudes(plan)
                nms.nms_response(plan, "UNPOL", out=img)
                nms.nms_azimuthal_average(plan, img, edges)

            for _ in range(max(1, args.warmup)):
                step()
            torch.cuda.synchronize()
            nms.nms_plan_stage_ms(plan, reset=True)
            ts = []
            for _ in range(max(1, args.steps)):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                step()
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            st = nms.nms_plan_stage_ms(plan)
            ms = float(np.mean(ts))
            terms = float(f.n) * plan.npix
            sweep.append({"copies": nc, "cells": int(f.n), "ms_per_step": ms, "terms_per_s": terms / (ms * 1e-3),
                          "stage_ms": {k: v[0] / max(1, args.steps) for k, v in st.items() if v[1]}})
            plan.close()
            del f
    clocks = clk.summary(peaks.get("sm_max_mhz", 2070.0))
    last = sweep[-1]
    line = {"metric": "cell·q-point terms/s of the SANS Fourier sum vs total cells (runtime-experiment shape)",
            "value": last["terms_per_s"], "unit": "terms/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": last["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16x3->f32(two-float)", "data": "synthetic",
            "config": {"workload": "N x linear-vortex sphere D=40nm a=2nm (4169 cells) on a 45nm simple-cubic "
                                   "lattice, one sum; 256x256 detector [-1.5,1.5]^2 nm^-1; value at the largest N",
                       "l2": "flushed between steps", "sweep": sweep,
                       "paper_context": "RTX 3090: linear in W from 4.169e4 to 1.067e8 cells (values only in "
                                        "a figure, not in the text)"},
            "roofline": None, "cpu_baseline": None, "e2e": None,
            "gpu_launches": None, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_paper_shape(args, dev):
    """The paper's interparticle-interference example as a shape: 800 D = 40 nm
    spheres (4169 cells each, linear vortex) on a 45 nm simple-cubic lattice,
    one sum over 3.34e6 cells on the paper's polar (q, theta) grid of 1000 x
    1000 nodes, q in [0, 1.5] nm^-1.  The library's default path there is the
    tensor path, one GEMM per ray (--precision direct: the compensated FP32
    direct sum).  One step = amplitudes, the unpolarized and spin-flip images,
    their azimuthal averages and c(r).  With the tensor path the line also
    times one step of the direct sum on the same plan inputs and gives the
    largest difference of the two unpolarized images."""
    import torch
    from paper_2601_18444_gb300 import inputs as I
    from paper_2601_18444_gb300 import nms
    particle = I.linear_vortex_sphere(20.0, 2.0, normalised=True)
    f = lattice_copies(particle, 800, objects=args.objects)
    g = nms.make_grid("polar", 1000, 1000, 0.0, 1.5)
    stream = torch.cuda.current_stream()
    prec = {"auto": nms.PREC_AUTO, "tc": nms.PREC_TC_F16X3, "direct": nms.PREC_FP32_DIRECT,
            "naive": nms.PREC_FP32_NAIVE}[args.precision]
    r = np.linspace(0.0, 400.0, 200)

    def make(pr):
        plan = nms.plan_from_field(f, g, nms.nms_options_default(timing=1, precision=pr,
                                                                 want_dilute=1 if args.objects else 0),
                                   stream=stream.cuda_stream)
        img_u = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
        img_s = torch.empty(plan.npix, dtype=torch.float64, device="cuda")

        def step():
            nms.nms_amplitudes(plan)
            nms.nms_response(plan, "UNPOL", out=img_u)
            nms.nms_response(plan, "SF", out=img_s)
            if args.objects:   # the interparticle split of the unpolarized image
                nms.nms_response(plan, "UNPOL", nms.PART_DILUTE, out=img_s)
                nms.nms_response(plan, "UNPOL", nms.PART_INTERFERENCE, out=img_s)
            for img in (img_u, img_s):
                Iq, c, qm = nms.nms_azimuthal_average(plan, img, nbins=1000)
                nms.nms_correlation(qm, Iq, r, stream=stream.cuda_stream)
        return plan, step, img_u

    def timed(step, n):
        ts = []
        for _ in range(n):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.mean(ts))

    plan, step, img_u = make(prec)
    path = nms.nms_plan_info(plan)["precision"]
    if path == nms.PREC_TC_F16X3:
        warm, steps = max(3, args.warmup), max(1, args.steps)
    else:   # seconds per step: a short run
        warm, steps = max(1, min(args.warmup, 1)), max(1, min(args.steps, 2))
    for _ in range(warm):
        step()
    torch.cuda.synchronize()
    nms.nms_plan_stage_ms(plan, reset=True)
    peaks, peak_src = load_peaks()
    with ClockSampler(dev) as clk:
        ms = timed(step, steps)
    st = nms.nms_plan_stage_ms(plan)
    terms = float(f.n) * plan.npix
    clocks = clk.summary(peaks.get("sm_max_mhz", 2070.0))
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = clocks["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
    extra = {}
    if path == nms.PREC_TC_F16X3 and nms.nms_plan_info(plan)["gemm_form"] == 3:
        # one GEMM per ray with its operands generated in shared memory: no
        # tables; the kernel reads 32 B per cell and ray and is paced by the
        # generation (instruction issue), so the tensor roofline of the
        # algorithmic flops is reported with that limit stated
        k_ms = st["gemm"][0] / steps
        n0, n1 = 1000, 1000
        n_rays = n1 // 2 if n1 % 2 == 0 else n1
        tflops = terms * ALGO_FLOPS_PER_TERM / (k_ms * 1e-3) / 1e12
        peak = peaks.get("bf16_tflops", 1900.0)
        roof = {"bound": "tensor", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                "traffic": None, "kernel": "k_gemm_ray_fused", "flops_per_term": ALGO_FLOPS_PER_TERM,
                "peak_source": f"{peak_src} bf16 dense (f16 same rate), burst",
                "cell_bytes_per_step": n_rays * f.n * 32.0,
                "limit": "operand generation in shared memory (instruction issue), not the tensor pipe",
                "note": f"one GEMM per ray: {n0} |q| nodes as 16 x 64 (padded to 1024), operands built in shared "
                        "memory from the cells' projections; the ray theta + pi taken as the conjugate"}
    elif path == nms.PREC_TC_F16X3:
        # one GEMM per ray: |q| nodes as k1 x k2 (k2 = 64), one 128 x 128 output
        # tile per ray, so each table block (32 KB per tile and 64 cells) feeds
        # one tile and the GEMM streams its tables from HBM: HBM roofline
        k_ms = st["gemm"][0] / steps
        n0, n1 = 1000, 1000
        k2 = min(64, n0)
        k1 = -(-n0 // k2)
        tiles = -(-(2 * 4 * k1) // 128) + -(-(2 * k2) // 128)
        n_rays = n1 // 2 if n1 % 2 == 0 else n1
        table_bytes = n_rays * (-(-f.n // 64)) * tiles * 32768.0
        achieved = table_bytes / (k_ms * 1e-3) / 1e9
        peak = peaks.get("hbm_gbs", 6800.0)
        tflops = terms * ALGO_FLOPS_PER_TERM / (k_ms * 1e-3) / 1e12
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "k_gemm_f16x3", "algorithmic_bytes_per_launch": "table bytes read",
                "table_bytes_per_step": table_bytes, "peak_source": f"{peak_src} HBM copy",
                "tensor": {"tflops_algorithmic": tflops, "flops_per_term": ALGO_FLOPS_PER_TERM,
                           "frac_of_bf16_burst": tflops / peaks.get("bf16_tflops", 1900.0)},
                "note": f"one GEMM per ray: {n0} |q| nodes as {k1} x {k2} (padded to {k1 * k2}), the ray "
                        "theta + pi taken as the conjugate"}
    else:
        peak = sms * 128 * mhz * 1e6 / 1e12
        k_ms = st["direct"][0] / steps
        achieved = terms * DIRECT_OPS_PER_TERM / (k_ms * 1e-3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Tops/s", "frac": achieved / peak,
                "traffic": None, "kernel": "k_direct<compensated>",
                "peak_source": f"{sms} SMs x 128 FP32 lanes x {mhz:.0f} MHz"}
    if path == nms.PREC_TC_F16X3 and not args.no_fp32_leg:
        ref_u = img_u.cpu().numpy()
        dplan, dstep, dimg = make(nms.PREC_FP32_DIRECT)
        dstep()
        torch.cuda.synchronize()
        d_ms = timed(dstep, 1)
        du = dimg.cpu().numpy()
        extra["fp32_direct"] = {"value": terms / (d_ms * 1e-3), "unit": "terms/s", "ms_per_step": d_ms,
                                "tc_over_fp32": d_ms / ms,
                                "unpol_max_abs_diff_over_max": float(np.max(np.abs(ref_u - du)) / np.max(np.abs(du)))}
        dplan.close()
    pname = "tensor path, one GEMM per ray" if path == nms.PREC_TC_F16X3 else "direct path"
    line = {"metric": f"cell·q-point terms/s of the SANS Fourier sum, paper's example shape (polar grid, {pname})",
            "value": terms / (ms * 1e-3), "unit": "terms/s", "n_gpus": 1, "steps": steps, "warmup": warm,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f16x3->f32(two-float)" if path == nms.PREC_TC_F16X3 else "f32(two-float)", "data": "synthetic",
            "config": {"workload": "800 x linear-vortex sphere D=40nm a=2nm (3.34e6 cells) on a 45nm simple-cubic "
                                   "lattice" + (" as 800 objects (dilute, total and interference parts)"
                                                if args.objects else "") +
                                   "; polar grid 1000 q in [0,1.5] nm^-1 x 1000 theta; UNPOL + SF, "
                                   "azimuthal averages, c(r) on 200 r",
                       "stage_ms_per_step": {k: v[0] / steps for k, v in st.items() if v[1]},
                       "paper_context": "about 60 s on an RTX 3090 for 3.38e6 cells on a 1000x1000 (q, theta) grid "
                                        "with all outputs incl. a 1000x1000 2D correlation and 670 MB of CSV "
                                        "(>= 5.6e10 terms/s)"},
            "roofline": roof, "cpu_baseline": None, "e2e": None,
            "gpu_launches": int(sum(v[1] for v in st.values()) + steps * (2 + (2 if args.objects else 0) + 2 + 4)),
            "clocks": clocks}
    line.update(extra)
    print(json.dumps(line), flush=True)
    plan.close()
    return 0


def plan_path_is_tc(stage):
    return stage.get("gemm", (0, 0))[1] > 0


if __name__ == "__main__":
    sys.exit(main())
