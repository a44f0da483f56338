"""Command-line contract of bench.py that needs no GPU.

The library drives one GPU.  A multi-GPU request (--gpus N > 1, or a torchrun
launch with WORLD_SIZE > 1) prints one "unavailable" JSON line on rank 0,
nothing on the other ranks, and exits 0 on every rank without touching a
GPU.  The symmetric-axis helper that sizes the tables matches the library's
rule (lo = -hi and at least two nodes).
"""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + args, cwd=ROOT, env=env,
                          capture_output=True, text=True, timeout=300)


def test_multi_gpu_request_prints_unavailable_on_rank0():
    r = _bench(["--gpus", "2", "--steps", "1", "--warmup", "1"], {"RANK": "0", "WORLD_SIZE": "2", "LOCAL_RANK": "0"})
    assert r.returncode == 0, r.stderr
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert "unavailable" in d and "single-GPU" in d["unavailable"] and d["n_gpus"] == 2


def test_multi_gpu_request_other_ranks_are_silent():
    r = _bench(["--gpus", "2"], {"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_gemm_axis_rule():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.gemm_axis(512, -2.0, 2.0) == 256
    assert bench.gemm_axis(63, -1.0, 1.0) == 32       # q = 0 node and the 31 nodes above it
    assert bench.gemm_axis(40, -0.7, 1.3) == 40
    assert bench.gemm_axis(1, 0.0, 0.0) == 1


def test_paper_shape_objects_place_the_same_cells():
    # --workload paper --objects: the same lattice of particles as objects
    # (local positions, sites as centres) puts every cell where the single
    # sum puts it, with the same weights
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    from paper_2601_18444_gb300 import inputs as I
    particle = I.linear_vortex_sphere(6.0, 2.0, normalised=True)
    one = bench.lattice_copies(particle, 27)
    objs = bench.lattice_copies(particle, 27, objects=True)
    assert objs.offsets[-1] == one.n and len(objs.offsets) == 28
    centres = np.repeat(objs.centers, np.diff(objs.offsets), axis=0)
    assert np.array_equal(objs.pos + centres, one.pos)
    assert np.array_equal(objs.vol, one.vol) and np.array_equal(objs.nuc, one.nuc) and np.array_equal(objs.mag, one.mag)
