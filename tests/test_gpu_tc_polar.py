"""POLAR grids on the tensor path (one GEMM per ray) against the FP64 oracle.

On the ray at angle theta the pixel q = |q| (sin theta, cos theta) has the
phase |q| u, u = Y sin theta + Z cos theta (paper, Eq. qdef and Sec.
"Summation approach"); |q|_i = lo + i dq splits as lo + 64 i1 dq + i2 dq,
so each ray is the Cartesian GEMM with both coordinates equal to u.  With an
even number of angles the ray theta + pi is the conjugate of the ray theta.
Covered: even and odd angle counts (mirrored rays or not), |q| counts below,
at and above 64 (one or several i1 nodes, ragged), a single |q| node,
rotation averages, many slots in several batches with a remainder batch, a
small table workspace (many chunks), several objects summed as one (their
centres applied), the dilute, total and interference parts of objects,
weight sets (loop mode), and the responses and azimuthal average of the
polar image.  A ray whose GEMM has one B tile and at most three A tiles (one
weight set, at most 48 x 64 |q| nodes) runs the fused form (operands generated in shared
memory): it is checked against the oracle and against the table form, at
every TMEM chunk length, with long work items (renormalised running sums)
and at the coherent |q| = 0 node.
"""
import numpy as np
import pytest

from oracle import sans as S
from paper_2601_18444_gb300 import inputs as I
from paper_2601_18444_gb300 import nms
from parity_util import AMP_TOL, IQ_TOL, amp_error, iq_rel_error, resp_tol, weight_sums

pytestmark = pytest.mark.gpu
TC = nms.PREC_TC_F16X3


def run(field, grid_kw, rot=None, **optkw):
    g = nms.make_grid(**grid_kw)
    opt = nms.nms_options_default(precision=TC, **optkw)
    plan = nms.plan_from_field(field, g, opt, rot=rot)
    nms.nms_amplitudes(plan)
    assert nms.nms_plan_info(plan)["precision"] == TC
    return plan


def og(grid_kw):
    kw = dict(grid_kw)
    kind = kw.pop("kind")
    return S.q_grid(kind, **kw)


POLAR_GRIDS = [
    dict(n0=33, n1=48, lo0=0.0, hi0=1.2),      # even angles (mirrored rays), one i1 node
    dict(n0=100, n1=37, lo0=0.0, hi0=1.5),     # odd angles (every ray computed), ragged second i1 node
    dict(n0=64, n1=10, lo0=0.1, hi0=2.0),      # exactly one full i1 node
    dict(n0=130, n1=20, lo0=0.05, hi0=2.5),    # three i1 nodes, the last ragged
    dict(n0=1, n1=8, lo0=0.7, hi0=0.7),        # a single |q| node
    dict(n0=1, n1=1, lo0=0.4, hi0=0.4),        # a single pixel
    dict(n0=50, n1=2, lo0=0.0, hi0=1.0),       # two angles: one ray and its mirror
    dict(n0=3000, n1=6, lo0=0.0, hi0=3.0),     # 47 i1 nodes: three A tiles, the last ragged
]


@pytest.mark.parametrize("gi", range(len(POLAR_GRIDS)))
def test_polar_tc_amplitudes(gi):
    kw = dict(kind="polar", **POLAR_GRIDS[gi])
    f = I.small_random_field(4000, seed=80 + gi, extent=12.0)
    plan = run(f, kw)
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    err = amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f))
    assert np.all(err <= AMP_TOL), err


def test_polar_tc_responses_and_average():
    f = I.linear_vortex_sphere(10.0, 1.0, M0=1.0, N0=0.7)
    kw = dict(kind="polar", n0=33, n1=48, lo0=0.0, hi0=1.2)
    plan = run(f, kw)
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f)) <= AMP_TOL)
    ref = S.responses(F_ref, g[2], g[3])
    for name in ("N", "M", "CHI", "NM", "SANSPOL_P", "UNPOL"):
        img = nms.nms_response(plan, name)
        assert np.max(np.abs(img - ref[name])) <= resp_tol(f), name
        Ig, cg, qg = nms.nms_azimuthal_average(plan, img, nbins=33)
        Ir = S.azimuthal_average_polar(ref[name], 33, 48)
        assert np.all(cg == 48)
        if name != "CHI":
            assert iq_rel_error(Ig, Ir) <= IQ_TOL, name
        else:
            assert np.max(np.abs(Ig)) <= resp_tol(f)


@pytest.mark.parametrize("fused", ["1", "0"])
def test_polar_tc_rotations_many_slots_small_workspace(fused, monkeypatch):
    # 3 rotations x 100 mirrored rays = 300 slots: several batches of at most
    # 64 slots and a remainder batch; with tables (NMS_RAY_FUSED=0) an 8 MB
    # workspace cuts each batch into many chunks
    monkeypatch.setenv("NMS_RAY_FUSED", fused)
    f = I.small_random_field(3000, seed=91, extent=10.0)
    kw = dict(kind="polar", n0=70, n1=200, lo0=0.0, hi0=1.4)
    Rs = I.random_rotations(3, seed=92)
    plan = run(f, kw, rot=Rs, workspace_bytes=8 << 20)
    assert nms.nms_plan_info(plan)["gemm_form"] == (3 if fused == "1" else 0)
    g = og(kw)
    acc = None
    for R in Rs:
        r = S.responses(S.amplitudes(f, R, g[0], g[1]), g[2], g[3])
        acc = r if acc is None else {k: acc[k] + r[k] for k in acc}
    for name in ("UNPOL", "SF", "M", "CHI"):
        assert np.max(np.abs(nms.nms_response(plan, name) - acc[name] / len(Rs))) <= resp_tol(f, rotations=Rs), name
    F_ref = S.amplitudes(f, Rs[-1], g[0], g[1])
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f, Rs[-1])) <= AMP_TOL)


def test_polar_tc_objects_summed_as_one():
    # several objects with centres and want_dilute = 0: one sum over the cells
    # at their global positions (the default path on a POLAR grid)
    rng = np.random.default_rng(95)
    sizes = rng.integers(50, 400, size=12)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    f = I.Field(rng.uniform(-4.0, 4.0, size=(n, 3)), rng.uniform(0.5, 1.5, n), rng.normal(size=n),
                rng.normal(size=(n, 3)), offsets=off, centers=rng.uniform(-30.0, 30.0, size=(len(sizes), 3)),
                name="objects")
    kw = dict(kind="polar", n0=50, n1=64, lo0=0.0, hi0=1.0)
    plan = nms.plan_from_field(f, nms.make_grid(**kw), nms.nms_options_default())
    nms.nms_amplitudes(plan)
    assert nms.nms_plan_info(plan)["precision"] == TC
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f)) <= AMP_TOL)


def test_polar_tc_weight_sets():
    # two weight sets (loop mode) on one ray GEMM: each set against the oracle
    f = I.box_field(16, 14, 12, a=2.0, n_modes=6, n_pores=3, seed=97)
    nuc2, mag2 = I.field_sweep(f, [0.0, 1.5])
    kw = dict(kind="polar", n0=40, n1=30, lo0=0.0, hi0=1.1)
    g = nms.make_grid(**kw)
    opt = nms.nms_options_default(precision=TC, n_sets=2)
    plan = nms.nms_plan_create(f.pos, f.vol, nuc2, mag2, grid=g, opt=opt)
    nms.nms_amplitudes(plan)
    go = og(kw)
    for st in range(2):
        fs = I.Field(f.pos, f.vol, nuc2[st], mag2[st], name="set")
        nms.nms_select_set(plan, st)
        F_ref = S.amplitudes(fs, np.eye(3), go[0], go[1])
        assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(fs)) <= AMP_TOL), st


@pytest.mark.parametrize("n1,ws", [(48, 0), (37, 0), (64, 4 << 20)])
def test_polar_tc_objects_dilute_total_interference(n1, ws):
    # per-object parts on the polar grid: each (rotation, ray) slot's objects
    # go through the dilute pass on the ray's node grid, whose products and
    # total amplitude are then scattered into the polar pixels; even and odd
    # angle counts, two rotations, one run with a small table workspace (a
    # large object cut into pieces across chunks)
    rng = np.random.default_rng(70 + n1)
    sizes = np.concatenate([[6000], rng.integers(1, 300, size=25)])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    f = I.Field(rng.uniform(-5.0, 5.0, size=(n, 3)), rng.uniform(0.5, 1.5, n), rng.normal(size=n),
                rng.normal(size=(n, 3)), offsets=off, centers=rng.uniform(-30.0, 30.0, size=(len(sizes), 3)),
                name="mixed_objects")
    kw = dict(kind="polar", n0=70, n1=n1, lo0=0.0, hi0=1.3)
    Rs = I.random_rotations(2, seed=71)
    plan = run(f, kw, rot=Rs, want_dilute=1, workspace_bytes=ws)
    g = og(kw)
    ids = ("N", "M", "SF", "CHI", "UNPOL")
    acc = {k: [0, 0, 0] for k in ids}
    for R in Rs:
        parts = S.response_parts(f, R, g, ids=ids)
        for k in ids:
            for i in range(3):
                acc[k][i] = acc[k][i] + parts[k][i] / len(Rs)
    tol = 2 * resp_tol(f, rotations=Rs)
    for k in ids:
        for i, part in enumerate((nms.PART_TOTAL, nms.PART_DILUTE, nms.PART_INTERFERENCE)):
            assert np.max(np.abs(nms.nms_response(plan, k, part) - acc[k][i])) <= tol, (k, part)
    F_ref = S.amplitudes(f, Rs[-1], g[0], g[1])   # the total amplitude of the last orientation
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f, Rs[-1])) <= AMP_TOL)


def test_polar_tc_refuses_per_object_bins():
    f = I.sphere_ensemble(n_spheres=3, median=2.0, sigma=0.1, clip=(1.5, 2.5), a=1.0, cube=20.0, seed=1)
    g = nms.make_grid("polar", 4, 4, 0, 1)
    plan = nms.plan_from_field(f, g, nms.nms_options_default(want_dilute=1))
    assert nms.nms_plan_info(plan)["precision"] == TC
    with pytest.raises(nms.NmsError) as e:
        nms.nms_plan_object_iq(plan, "UNPOL", np.linspace(0.0, 1.0, 5))
    assert e.value.status == 4


def test_polar_tc_objects_capture_in_cuda_graph():
    # the ray path with per-object parts (one dilute pass per slot, issued
    # from the host) captured once and replayed: bit for bit the eager result
    torch = pytest.importorskip("torch")
    f = I.small_random_field(2000, seed=61, extent=6.0, n_objects=7)
    kw = dict(kind="polar", n0=40, n1=24, lo0=0.0, hi0=1.2)
    side = torch.cuda.Stream()
    opt = nms.nms_options_default(precision=TC, want_dilute=1)
    plan = nms.plan_from_field(f, nms.make_grid(**kw), opt, rot=I.random_rotations(2, seed=62),
                               stream=side.cuda_stream)
    nms.nms_amplitudes(plan)
    ref = {pt: nms.nms_response(plan, "UNPOL", pt).copy()
           for pt in (nms.PART_TOTAL, nms.PART_DILUTE, nms.PART_INTERFERENCE)}
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        graph.capture_begin()
        nms.nms_amplitudes(plan)
        graph.capture_end()
    for _ in range(2):
        with torch.cuda.stream(side):
            graph.replay()
        torch.cuda.synchronize()
        for pt, r in ref.items():
            assert np.array_equal(nms.nms_response(plan, "UNPOL", pt), r), pt


def test_polar_tc_autotune_request_keeps_defaults():
    # the autotuner's error probe reads the Cartesian pixel layout, so a
    # POLAR plan keeps the default GEMM configuration and still matches
    f = I.small_random_field(3000, seed=63, extent=8.0)
    kw = dict(kind="polar", n0=30, n1=16, lo0=0.0, hi0=1.0)
    plan = run(f, kw, autotune=1)
    info = nms.nms_plan_info(plan)
    assert info["kc_cells"] == 192 and info["items_per_sm"] == 8 and info["gemm_form"] == 3
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f)) <= AMP_TOL)


@pytest.mark.parametrize("objects", [False, True])
def test_polar_tc_fp64_ray_preparation_path(objects, monkeypatch):
    # the FP64 rotation per (rotation, ray) slot, taken when the cells
    # rotated once per rotation would not fit their 1 GB buffer, forced here
    monkeypatch.setenv("NMS_RAY_PREP_FP64", "1")
    f = I.small_random_field(2500, seed=66, extent=7.0, n_objects=5 if objects else 1)
    kw = dict(kind="polar", n0=45, n1=20, lo0=0.0, hi0=1.2)
    Rs = I.random_rotations(2, seed=67)
    plan = run(f, kw, rot=Rs, want_dilute=1 if objects else 0)
    g = og(kw)
    F_ref = S.amplitudes(f, Rs[-1], g[0], g[1])
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f, Rs[-1])) <= AMP_TOL)
    if objects:
        acc = [0, 0, 0]
        for R in Rs:
            parts = S.response_parts(f, R, g, ids=("UNPOL",))
            for i in range(3):
                acc[i] = acc[i] + parts["UNPOL"][i] / len(Rs)
        tol = 2 * resp_tol(f, rotations=Rs)
        for i, part in enumerate((nms.PART_TOTAL, nms.PART_DILUTE, nms.PART_INTERFERENCE)):
            assert np.max(np.abs(nms.nms_response(plan, "UNPOL", part) - acc[i])) <= tol, part


def test_polar_tc_weight_sets_with_objects_and_rotations():
    # 3 states x 6 objects (dilute, total, interference) x 2 orientations on
    # the ray path: the per-slot buffers hold every set
    f = I.small_random_field(1500, seed=5, extent=5.0, n_objects=6)
    nuc, mag = I.field_sweep(f, [0.0, 0.7, 4.0])
    kw = dict(kind="polar", n0=36, n1=28, lo0=0.0, hi0=1.2)
    Rs = I.random_rotations(2, seed=4)
    opt = nms.nms_options_default(precision=TC, want_dilute=1, n_sets=3)
    plan = nms.nms_plan_create(f.pos, f.vol, nuc, mag, f.offsets, f.centers, Rs, grid=nms.make_grid(**kw), opt=opt)
    nms.nms_amplitudes(plan)
    q = og(kw)
    for s in range(3):
        fs = I.Field(f.pos, f.vol, nuc[s], mag[s], offsets=f.offsets, centers=f.centers, name=f"state{s}")
        nms.nms_select_set(plan, s)
        acc = {k: [0, 0, 0] for k in ("UNPOL", "SF")}
        for R in Rs:
            parts = S.response_parts(fs, R, q, ids=("UNPOL", "SF"))
            for k in acc:
                for i in range(3):
                    acc[k][i] = acc[k][i] + parts[k][i] / len(Rs)
        tol = 2 * resp_tol(fs, rotations=Rs)
        for k in acc:
            for i, part in enumerate((nms.PART_TOTAL, nms.PART_DILUTE, nms.PART_INTERFERENCE)):
                assert np.max(np.abs(nms.nms_response(plan, k, part) - acc[k][i])) <= tol, (s, k, part)


def test_polar_tc_fused_matches_tables_and_oracle(monkeypatch):
    # 1000 |q| nodes (15 full i1 nodes and a ragged 16th: one A tile),
    # 12 angles; the fused form and the table form each
    # against the oracle, and against each other
    f = I.small_random_field(5001, seed=71, extent=9.0)
    kw = dict(kind="polar", n0=1000, n1=12, lo0=0.0, hi0=2.0)
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    out = {}
    for fused in ("1", "0"):
        monkeypatch.setenv("NMS_RAY_FUSED", fused)
        plan = run(f, kw)
        assert nms.nms_plan_info(plan)["gemm_form"] == (3 if fused == "1" else 0)
        out[fused] = nms.nms_get_amplitudes(plan)
        assert np.all(amp_error(out[fused], F_ref, weight_sums(f)) <= AMP_TOL), fused
    assert np.all(amp_error(out["1"], out["0"], weight_sums(f)) <= 2 * AMP_TOL)


@pytest.mark.parametrize("kc", [64, 128, 192, 256])
def test_polar_tc_fused_chunk_lengths_long_items(kc):
    # one work item per SM (split_k = 1): ~15 k-blocks per item, so the
    # running sums in tensor memory pass several renormalisations; every
    # drain interval from one to four k-blocks
    f = I.small_random_field(150000, seed=72, extent=20.0)
    kw = dict(kind="polar", n0=64, n1=6, lo0=0.02, hi0=1.5)
    plan = run(f, kw, kc_cells=kc, split_k=1)
    info = nms.nms_plan_info(plan)
    assert info["gemm_form"] == 3 and info["kc_cells"] == kc
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f)) <= AMP_TOL)


@pytest.mark.parametrize("kc", [128, 192])
def test_polar_tc_fused_coherent_q0(kc):
    # all-positive constant weights and |q| from 0: the partial sums in the
    # FP32 accumulator are as coherent as they can be
    f = I.box_field(40, 40, 40, a=1.0, n_modes=4, seed=2, pores=False)
    kw = dict(kind="polar", n0=9, n1=8, lo0=0.0, hi0=0.02)
    plan = run(f, kw, kc_cells=kc)
    assert nms.nms_plan_info(plan)["gemm_form"] == 3
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f)) <= AMP_TOL)


def test_fused_form_sincos_against_exact_and_sincospif():
    # the fused form's sine and cosine of 2 pi t (quarter-turn reduction and
    # Taylor series) on reduced phases |t| <= 1/2: random and evenly spaced
    # values, the quarter-turn boundaries and their neighbours, and tiny t
    rng = np.random.default_rng(11)
    edges = np.array([-0.5, -0.375, -0.25, -0.125, 0.0, 0.125, 0.25, 0.375, 0.5], dtype=np.float32)
    near = np.concatenate([np.nextafter(edges, np.float32(1)), np.nextafter(edges, np.float32(-1))])
    t = np.concatenate([rng.uniform(-0.5, 0.5, 400000), np.linspace(-0.5, 0.5, 40001), edges, near,
                        [1e-30, -1e-30, 1e-8, -3e-6]]).astype(np.float32)
    t = t[np.abs(t) <= 0.5]
    out = nms.nms_selftest_sincos(t)
    x = 2.0 * np.pi * t.astype(np.float64)
    err = np.maximum(np.abs(out[:, 0] - np.sin(x)), np.abs(out[:, 1] - np.cos(x)))
    err_ref = np.maximum(np.abs(out[:, 2] - np.sin(x)), np.abs(out[:, 3] - np.cos(x)))
    assert err.max() <= 1.0e-7, err.max()                  # under one unit in the last place at 1
    assert err.max() <= err_ref.max() + 6e-8, (err.max(), err_ref.max())
    # exact at the quarter turns
    q = nms.nms_selftest_sincos(np.array([0.0, 0.25, -0.25, 0.5, -0.5], dtype=np.float32))
    np.testing.assert_array_equal(q[:, 0], [0.0, 1.0, -1.0, 0.0, 0.0])
    np.testing.assert_array_equal(q[:, 1], [1.0, 0.0, 0.0, -1.0, -1.0])


@pytest.mark.parametrize("n0,form", [(1024, 3), (1025, 3), (3072, 3), (3073, 0)])
def test_polar_tc_fused_form_boundary(n0, form):
    # 1024 |q| nodes (16 x 64) fill one A tile, 1025 start a second; 3072
    # (48 x 64, three A tiles) is the largest ray of the fused form, one node
    # more takes the tables
    f = I.small_random_field(3001, seed=73, extent=8.0)
    kw = dict(kind="polar", n0=n0, n1=4, lo0=0.0, hi0=2.5)
    plan = run(f, kw)
    assert nms.nms_plan_info(plan)["gemm_form"] == form
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f)) <= AMP_TOL)
