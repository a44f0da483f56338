"""GPU parity of the tensor-core path (split-FP16 tcgen05 GEMM) against the oracle.

Same bars as the direct path: max_p |dF|/sum_j|w_cj| <= 1e-6 per channel,
responses within the bound that implies, I(q) within 1e-5.  Shapes cover
several tiles with ragged tails in every GEMM dimension (q_y rows, q_z
columns, cells), a single cell, objects with the dilute/interference split,
rotation averages, the coherent q = 0 pixel, and the full-size box workload
on sampled pixels and on whole bins of its I(q).
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
    return plan


def og(grid_kw):
    kw = dict(grid_kw)
    kind = kw.pop("kind")
    return S.q_grid(kind, **kw)


def test_tc_single_tile_small():
    f = I.sphere_vortex(6.0, 2.0, seed=3)
    kw = dict(kind="cartesian", n0=8, n1=8, lo0=-1.0, hi0=1.0, lo1=-1.0, hi1=1.0)
    plan = run(f, kw)
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    err = amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f))
    assert np.all(err <= AMP_TOL), err


def test_tc_config1_all_responses():
    f = I.sphere_vortex(16.0, 2.0, seed=0)
    kw = dict(kind="cartesian", n0=128, n1=128, lo0=-1.0, hi0=1.0, lo1=-1.0, hi1=1.0)
    plan = run(f, kw)
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    err = amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f))
    assert np.all(err <= AMP_TOL), err
    ref = S.responses(F_ref, g[2], g[3])
    for name in nms.RESPONSE_NAMES:
        assert np.max(np.abs(nms.nms_response(plan, name) - ref[name])) <= resp_tol(f), name
    edges = np.linspace(0, 1, 65)
    for name in ("UNPOL", "SF"):
        Ig, cg, _ = nms.nms_azimuthal_average(plan, nms.nms_response(plan, name), edges)
        Ir, cr, _ = S.azimuthal_average_cartesian(ref[name], g[4], edges)
        assert np.array_equal(cg, cr)
        assert iq_rel_error(Ig, Ir) <= IQ_TOL


@pytest.mark.parametrize("ny,nz,n", [(33, 65, 1), (1, 1, 31), (97, 130, 1001), (200, 7, 4129)])
def test_tc_ragged_shapes(ny, nz, n):
    f = I.small_random_field(n, seed=ny + nz + n, extent=12.0)
    kw = dict(kind="cartesian", n0=ny, n1=nz, lo0=-1.7, hi0=1.3, lo1=-0.6, hi1=2.1)
    plan = run(f, kw)
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    err = amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f))
    assert np.all(err <= AMP_TOL), err


@pytest.mark.parametrize("kc", [0, 64, 128, 192])
def test_tc_coherent_q0_pixel(kc):
    # all-positive constant weights, pixels at and near q = 0: the partial sums
    # in the FP32 tensor accumulators are as coherent as they can be
    f = I.box_field(40, 40, 40, a=1.0, n_modes=4, seed=2, pores=False)
    kw = dict(kind="cartesian", n0=9, n1=9, lo0=-0.02, hi0=0.02, lo1=-0.02, hi1=0.02)
    plan = run(f, kw, kc_cells=kc)
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    err = amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f))
    assert np.all(err <= AMP_TOL), err


def test_tc_objects_and_rotation():
    f = I.small_random_field(1500, seed=5, extent=5.0, n_objects=6)
    kw = dict(kind="cartesian", n0=40, n1=36, lo0=-1.0, hi0=1.2, lo1=-1.1, hi1=0.9)
    Rs = I.random_rotations(2, seed=4)
    plan = run(f, kw, rot=Rs, want_dilute=1)
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


def test_tc_matches_direct_path():
    f = I.box_field(48, 40, 24, a=2.0, n_modes=8, n_pores=5, seed=6)
    kw = dict(kind="cartesian", n0=96, n1=80, lo0=-2.0, hi0=2.0, lo1=-2.0, hi1=2.0)
    F_tc = nms.nms_get_amplitudes(run(f, kw))
    g = nms.make_grid(**kw)
    pd = nms.plan_from_field(f, g, nms.nms_options_default(precision=nms.PREC_FP32_DIRECT))
    nms.nms_amplitudes(pd)
    F_d = nms.nms_get_amplitudes(pd)
    err = amp_error(F_tc, F_d, weight_sums(f))
    assert np.all(err <= 2 * AMP_TOL), err


def test_tc_full_box_sampled_pixels():
    # the default benchmark workload at full size (4.19M cells, 512^2 pixels),
    # checked on a random sample of pixels the oracle evaluates one by one
    f = I.box_field(256, 256, 64, a=2.0, n_modes=64, kmax=0.2, n_pores=200, seed=1)
    kw = dict(kind="cartesian", n0=512, n1=512, lo0=-2.0, hi0=2.0, lo1=-2.0, hi1=2.0)
    plan = run(f, kw)
    F = nms.nms_get_amplitudes(plan)
    g = og(kw)
    rng = np.random.default_rng(0)
    centre = [255 * 512 + 255, 255 * 512 + 256, 256 * 512 + 255, 256 * 512 + 256]   # most coherent pixels
    idx = np.unique(np.concatenate([rng.choice(512 * 512, 24, replace=False), centre]))
    w = S.cell_weights(f.vol, f.nuc, f.mag, np.eye(3))
    F_ref = S.dsft(f.pos[:, 1], f.pos[:, 2], w, g[0][idx], g[1][idx])
    err = amp_error(F[:, idx], F_ref, np.abs(w).sum(1))
    assert np.all(err <= AMP_TOL), err


def test_tc_full_box_iq_bins():
    # the same full-size workload through the unpolarized and spin-flip images
    # and their 128-bin I(q) (bins of width 2/128 up to |q| = 2): pixel counts
    # and mean |q| of every bin against the oracle's binning, and I(q) of
    # seven whole bins -- the four innermost (most coherent), 16, 63 and the
    # outermost (largest phases) -- from the oracle's amplitudes of every
    # pixel in them (5,352 of 262,144)
    f = I.box_field(256, 256, 64, a=2.0, n_modes=64, kmax=0.2, n_pores=200, seed=1)
    kw = dict(kind="cartesian", n0=512, n1=512, lo0=-2.0, hi0=2.0, lo1=-2.0, hi1=2.0)
    plan = run(f, kw)
    edges = np.linspace(0.0, 2.0, 129)
    g = og(kw)
    _, cr, qr = S.azimuthal_average_cartesian(np.zeros(512 * 512), g[4], edges)
    bins = np.array([0, 1, 2, 3, 16, 63, 127])
    sel = np.flatnonzero(np.isin(np.searchsorted(edges, g[4], side="right") - 1, bins))
    assert sel.size == cr[bins].sum() == 5352
    w = S.cell_weights(f.vol, f.nuc, f.mag, np.eye(3))
    F_ref = S.dsft(f.pos[:, 1], f.pos[:, 2], w, g[0][sel], g[1][sel])
    ref = S.responses(F_ref, g[2][sel], g[3][sel])
    for name in ("UNPOL", "SF"):
        Ig, cg, qg = nms.nms_azimuthal_average(plan, nms.nms_response(plan, name), edges)
        assert np.array_equal(cg, cr)
        np.testing.assert_allclose(qg[cg > 0], qr[cr > 0], rtol=1e-13)
        Ir, cs, _ = S.azimuthal_average_cartesian(ref[name], g[4][sel], edges)
        assert np.array_equal(cs[bins], cr[bins])
        assert np.all(Ir[bins] > 1e-8 * Ir[0])           # every chosen bin is under the 1e-5 bar
        rel = np.abs(Ig[bins] - Ir[bins]) / np.abs(Ir[bins])
        assert np.all(rel <= IQ_TOL), (name, rel)


def test_tc_ensemble_many_chunks_dilute_interference():
    # ~1500 small spheres, table workspace forced small so objects are cut
    # into pieces across many table chunks; dilute, total and interference
    f = I.sphere_ensemble(n_spheres=1500, median=2.5, sigma=0.35, clip=(1.5, 4.0), a=1.0, cube=300.0, seed=7)
    kw = dict(kind="cartesian", n0=40, n1=56, lo0=-1.5, hi0=1.5, lo1=-1.5, hi1=1.5)
    plan = run(f, kw, want_dilute=1, workspace_bytes=8 << 20)
    g = og(kw)
    ids = ("N", "M", "SF", "CHI", "NM", "UNPOL")
    parts = S.response_parts(f, np.eye(3), g, ids=ids)
    tol = 2 * resp_tol(f)
    # the dilute part scales with the number of objects, not with (sum |w|)^2
    wk = [np.abs(S.cell_weights(f.vol[a:b], f.nuc[a:b], f.mag[a:b], np.eye(3))).sum(1)
          for a, b in zip(f.offsets[:-1], f.offsets[1:])]
    tol_dil = 4e-6 * sum((w[0] + w[1] + w[2] + w[3]) ** 2 for w in wk)
    for k in ids:
        assert np.max(np.abs(nms.nms_response(plan, k, nms.PART_TOTAL) - parts[k][0])) <= tol, k
        assert np.max(np.abs(nms.nms_response(plan, k, nms.PART_DILUTE) - parts[k][1])) <= tol_dil, k
        assert np.max(np.abs(nms.nms_response(plan, k, nms.PART_INTERFERENCE) - parts[k][2])) <= tol + tol_dil, k


def test_tc_mixed_object_sizes_direct_and_split_outputs():
    # one large object (its tiles are split over many work items and reduced)
    # beside many small ones (one item per tile, written straight into F), in
    # the same table chunk; plus a two-rotation batch so outputs of both kinds
    # interleave across rotation slots
    rng = np.random.default_rng(21)
    sizes = np.concatenate([[20000], rng.integers(1, 300, size=60)])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    pos = rng.uniform(-6.0, 6.0, size=(n, 3))
    f = I.Field(pos, rng.uniform(0.5, 1.5, n), rng.normal(size=n), rng.normal(size=(n, 3)), offsets=off,
                centers=rng.uniform(-40.0, 40.0, size=(len(sizes), 3)), name="mixed_objects")
    kw = dict(kind="cartesian", n0=40, n1=56, lo0=-1.5, hi0=1.5, lo1=-1.5, hi1=1.5)
    Rs = I.random_rotations(2, seed=8)
    plan = run(f, kw, rot=Rs, want_dilute=1)
    g = og(kw)
    ids = ("N", "M", "SF", "UNPOL")
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


@pytest.mark.parametrize("n_obj, n_rot", [(3, 1), (300, 2)])
def test_tc_dilute_pass_whole_q_y_rows(n_obj, n_rot):
    # q_y rows of 256 pixels (two blocks of 128) and an even q_z count: the
    # dilute/shift pass stages each block's slice of F_b with bulk copies.
    # Fewer outputs than ring slots; several hundred outputs whose rotation
    # changes inside a batch
    if n_obj == 3:
        f = I.small_random_field(900, seed=41, extent=5.0, n_objects=3)
    else:
        f = I.sphere_ensemble(n_spheres=n_obj, median=2.5, sigma=0.35, clip=(1.5, 4.0), a=1.0, cube=200.0, seed=43)
    kw = dict(kind="cartesian", n0=256, n1=14, lo0=-1.5, hi0=1.5, lo1=-1.2, hi1=1.4)
    Rs = I.random_rotations(n_rot, seed=44)
    plan = run(f, kw, rot=Rs, want_dilute=1)
    g = og(kw)
    ids = ("N", "M", "SF", "UNPOL")
    acc = {k: [0, 0, 0] for k in ids}
    for R in Rs:
        parts = S.response_parts(f, R, g, ids=ids)
        for k in ids:
            for i in range(3):
                acc[k][i] = acc[k][i] + parts[k][i] / len(Rs)
    tol = 2 * resp_tol(f, rotations=Rs)
    # the dilute part is bounded by the sum over objects of each one's (sum |w|)^2
    tol_dil = 0.0
    for R in Rs:
        wk = [np.abs(S.cell_weights(f.vol[a:b], f.nuc[a:b], f.mag[a:b], R)).sum(1)
              for a, b in zip(f.offsets[:-1], f.offsets[1:])]
        tol_dil = max(tol_dil, 4e-6 * sum((w[0] + w[1] + w[2] + w[3]) ** 2 for w in wk))
    for k in ids:
        assert np.max(np.abs(nms.nms_response(plan, k, nms.PART_TOTAL) - acc[k][0])) <= tol, k
        assert np.max(np.abs(nms.nms_response(plan, k, nms.PART_DILUTE) - acc[k][1])) <= tol_dil, k
        assert np.max(np.abs(nms.nms_response(plan, k, nms.PART_INTERFERENCE) - acc[k][2])) <= tol + tol_dil, k


@pytest.mark.parametrize("mode", [0, 2])
def test_tc_gemm_forms_agree_with_oracle(mode, monkeypatch):
    # the two GEMM forms (one CTA per tile; the two-SM MMA over A-tile pairs)
    # on a grid with an even number of A tiles, with split-and-reduced items
    # (one large object) and direct items (small ones)
    monkeypatch.setenv("NMS_GEMM_MODE", str(mode))
    rng = np.random.default_rng(30 + mode)
    sizes = np.concatenate([[12000], rng.integers(1, 200, size=20)])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    f = I.Field(rng.uniform(-5.0, 5.0, size=(n, 3)), rng.uniform(0.5, 1.5, n), rng.normal(size=n),
                rng.normal(size=(n, 3)), offsets=off, centers=rng.uniform(-30.0, 30.0, size=(len(sizes), 3)),
                name="mixed_objects")
    kw = dict(kind="cartesian", n0=61, n1=117, lo0=-1.5, hi0=1.4, lo1=-1.3, hi1=1.5)   # 4 A tiles, 2 B tiles
    plan = run(f, kw, want_dilute=1)
    g = og(kw)
    ids = ("N", "M", "UNPOL")
    parts = S.response_parts(f, np.eye(3), g, ids=ids)
    tol = 2 * resp_tol(f)
    for k in ids:
        for i, part in enumerate((nms.PART_TOTAL, nms.PART_DILUTE, nms.PART_INTERFERENCE)):
            assert np.max(np.abs(nms.nms_response(plan, k, part) - parts[k][i])) <= tol, (k, part)
    # one object alone: amplitudes against the oracle element by element
    f1 = I.Field(f.pos[:12000], f.vol[:12000], f.nuc[:12000], f.mag[:12000], name="large_object")
    plan1 = run(f1, kw)
    F_ref = S.amplitudes(f1, np.eye(3), g[0], g[1])
    err = amp_error(nms.nms_get_amplitudes(plan1), F_ref, weight_sums(f1))
    assert np.all(err <= AMP_TOL), err


def test_tc_rotation_batches_full_and_remainder():
    # 70 rotations: one batch of 64 prepared rotations and a remainder of 6
    f = I.ellipsoid_uniform((8.0, 5.0, 5.0), a=1.0, seed=2)
    Rs = I.random_rotations(70, seed=13)
    kw = dict(kind="cartesian", n0=24, n1=20, lo0=-1.0, hi0=1.0, lo1=-1.0, hi1=1.0)
    plan = run(f, kw, rot=Rs)
    g = og(kw)
    acc = None
    for R in Rs:
        r = S.responses(S.amplitudes(f, R, g[0], g[1]), g[2], g[3])
        acc = r if acc is None else {k: acc[k] + r[k] for k in acc}
    for name in ("UNPOL", "SF", "M", "P", "CHI"):
        assert np.max(np.abs(nms.nms_response(plan, name) - acc[name] / len(Rs))) <= resp_tol(f, rotations=Rs), name
    F_ref = S.amplitudes(f, Rs[-1], g[0], g[1])
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f, Rs[-1])) <= AMP_TOL)


def test_tc_amplitudes_capture_in_cuda_graph():
    torch = pytest.importorskip("torch")
    f = I.small_random_field(3000, seed=31, extent=8.0, n_objects=5)
    kw = dict(kind="cartesian", n0=48, n1=40, lo0=-1.0, hi0=1.0, lo1=-1.0, hi1=1.0)
    side = torch.cuda.Stream()
    opt = nms.nms_options_default(precision=TC, want_dilute=1)
    plan = nms.plan_from_field(f, nms.make_grid(**kw), opt, rot=I.random_rotations(3, seed=2),
                               stream=side.cuda_stream)
    nms.nms_amplitudes(plan)                     # first call outside capture
    ref = nms.nms_response(plan, "UNPOL", nms.PART_INTERFERENCE).copy()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        graph.capture_begin()
        nms.nms_amplitudes(plan)
        graph.capture_end()
    for _ in range(2):
        with torch.cuda.stream(side):
            graph.replay()                       # replays on the capturing stream
        torch.cuda.synchronize()
        got = nms.nms_response(plan, "UNPOL", nms.PART_INTERFERENCE)
        assert np.array_equal(got, ref)


def test_tc_ensemble_graph_replay_matches_oracle():
    # An ensemble of 1500 small spheres captured once in a CUDA graph and
    # replayed: a point-symmetric detector with 128-pixel q_y rows (half-plane
    # amplitudes, the bulk-copy dilute pass split into output slices), a
    # table workspace small enough for many chunks.  Every replay must give
    # the eager result bit for bit, and the eager result must match the
    # oracle's total, dilute and interference parts.
    torch = pytest.importorskip("torch")
    f = I.sphere_ensemble(n_spheres=1500, median=2.5, sigma=0.35, clip=(1.5, 4.0), a=1.0, cube=300.0, seed=17)
    kw = dict(kind="cartesian", n0=128, n1=64, lo0=-1.5, hi0=1.5, lo1=-1.2, hi1=1.2)
    side = torch.cuda.Stream()
    opt = nms.nms_options_default(precision=TC, want_dilute=1, workspace_bytes=8 << 20)
    plan = nms.plan_from_field(f, nms.make_grid(**kw), opt, stream=side.cuda_stream)
    assert nms.nms_plan_info(plan)["mirror"] == (1, 1)
    ids = ("N", "M", "SF", "UNPOL")
    parts_of = (nms.PART_TOTAL, nms.PART_DILUTE, nms.PART_INTERFERENCE)
    nms.nms_amplitudes(plan)                     # eager, outside capture
    eager = {(k, pt): nms.nms_response(plan, k, pt).copy() for k in ids for pt in parts_of}
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(side):
        graph.capture_begin()
        nms.nms_amplitudes(plan)
        graph.capture_end()
    for _ in range(2):
        with torch.cuda.stream(side):
            graph.replay()
        torch.cuda.synchronize()
        for k in ids:
            for pt in parts_of:
                assert np.array_equal(nms.nms_response(plan, k, pt), eager[(k, pt)]), (k, pt)
    g = og(kw)
    ref = S.response_parts(f, np.eye(3), g, ids=ids)
    tol = 2 * resp_tol(f)
    wk = [np.abs(S.cell_weights(f.vol[a:b], f.nuc[a:b], f.mag[a:b], np.eye(3))).sum(1)
          for a, b in zip(f.offsets[:-1], f.offsets[1:])]
    tol_dil = 4e-6 * sum((w[0] + w[1] + w[2] + w[3]) ** 2 for w in wk)
    for k in ids:
        assert np.max(np.abs(eager[(k, nms.PART_TOTAL)] - ref[k][0])) <= tol, k
        assert np.max(np.abs(eager[(k, nms.PART_DILUTE)] - ref[k][1])) <= tol_dil, k
        assert np.max(np.abs(eager[(k, nms.PART_INTERFERENCE)] - ref[k][2])) <= tol + tol_dil, k


def test_tc_autotune_picks_valid_config_and_caches(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("NMS_AUTOTUNE_CACHE", str(cache))
    f = I.box_field(40, 40, 40, a=1.0, n_modes=4, seed=2, pores=False)     # coherent: a hard probe
    kw = dict(kind="cartesian", n0=36, n1=40, lo0=-0.3, hi0=0.3, lo1=-0.3, hi1=0.3)
    plan = run(f, kw, autotune=1)
    info = nms.nms_plan_info(plan)
    assert info["precision"] == TC and info["kc_cells"] in (64, 128, 192, 256) and info["items_per_sm"] in (4, 8, 16)
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f)) <= AMP_TOL)
    # a second plan of the same shape reuses the tuned choice
    plan2 = run(f, kw, autotune=1)
    assert nms.nms_plan_info(plan2) == info


# Detector axes symmetric about q = 0 (lo = -hi) are computed on their q >= 0
# half and written for both signs (cos even, sin odd in q); an odd node count
# has a q = 0 node that is its own mirror.  Every combination of symmetric and
# asymmetric axes, even and odd node counts, against the oracle: amplitudes
# element by element, and the dilute / total / interference parts of objects
# whose outputs are written straight from the GEMM (one piece), assembled
# from several pieces (small table workspace) and reduced from split items.
# On a grid symmetric in both axes only the q_z >= 0 half of the per-object
# amplitudes is stored and the dilute pass writes the other half by
# conjugation; the last grid takes the pass that copies whole 128-pixel q_y
# rows, with an odd q_z count (a q_z = 0 row that is its own mirror).
SYM_GRIDS = [
    dict(n0=64, n1=48, lo0=-1.2, hi0=1.2, lo1=-0.9, hi1=0.9),     # both symmetric, even
    dict(n0=63, n1=49, lo0=-1.2, hi0=1.2, lo1=-0.9, hi1=0.9),     # both symmetric, odd (q = 0 nodes)
    dict(n0=37, n1=40, lo0=-1.0, hi0=1.0, lo1=-0.7, hi1=1.3),     # q_y symmetric (odd), q_z not
    dict(n0=52, n1=41, lo0=-0.8, hi0=1.1, lo1=-1.4, hi1=1.4),     # q_z symmetric (odd), q_y not
    dict(n0=200, n1=2, lo0=-2.0, hi0=2.0, lo1=-0.5, hi1=0.5),     # several A tiles; two q_z nodes
    dict(n0=3, n1=300, lo0=-0.3, hi0=0.3, lo1=-2.0, hi1=2.0),     # three q_y nodes; several B tiles
    dict(n0=128, n1=33, lo0=-1.0, hi0=1.0, lo1=-0.8, hi1=0.8),    # both symmetric; q_y rows of 128 pixels
]


@pytest.mark.parametrize("gi", range(len(SYM_GRIDS)))
def test_tc_symmetric_axes_amplitudes(gi):
    kw = dict(kind="cartesian", **SYM_GRIDS[gi])
    f = I.small_random_field(5000, seed=60 + gi, extent=15.0)
    plan = run(f, kw)
    g = og(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    err = amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f))
    assert np.all(err <= AMP_TOL), err


@pytest.mark.parametrize("gi", [0, 1, 2, 3, 6])
@pytest.mark.parametrize("ws", [0, 4 << 20])
def test_tc_symmetric_axes_objects(gi, ws):
    kw = dict(kind="cartesian", **SYM_GRIDS[gi])
    rng = np.random.default_rng(70 + gi)
    sizes = np.concatenate([[9000], rng.integers(1, 400, size=40)])
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(off[-1])
    f = I.Field(rng.uniform(-6.0, 6.0, size=(n, 3)), rng.uniform(0.5, 1.5, n), rng.normal(size=n),
                rng.normal(size=(n, 3)), offsets=off, centers=rng.uniform(-40.0, 40.0, size=(len(sizes), 3)),
                name="mixed_objects")
    Rs = I.random_rotations(2, seed=71 + gi)
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

