"""GPU parity of the direct-sum path (FP32, compensated phase) against the oracle.

Element-by-element comparison on seeded inputs through the C ABI: amplitudes,
every response id, azimuthal averages, correlation functions, objects with the
dilute/interference split, rotation averages, polar and list grids, and the
degenerate cases (one cell, empty objects, absent channels, q = 0).
"""
import numpy as np
import pytest

from oracle import sans as S
from paper_2601_18444_gb300 import inputs as I
from paper_2601_18444_gb300 import nms
from parity_util import AMP_TOL, IQ_TOL, amp_error, iq_rel_error, resp_tol, weight_sums

pytestmark = pytest.mark.gpu

DIRECT = nms.PREC_FP32_DIRECT


def run_plan(field, grid_kw, prec=DIRECT, rot=None, **optkw):
    g = nms.make_grid(**grid_kw)
    opt = nms.nms_options_default(precision=prec, **optkw)
    plan = nms.plan_from_field(field, g, opt, rot=rot)
    nms.nms_amplitudes(plan)
    return plan


def oracle_grid(grid_kw):
    kw = dict(grid_kw)
    kind = kw.pop("kind")
    return S.q_grid(kind, **kw)


CFG1 = dict(kind="cartesian", n0=128, n1=128, lo0=-1.0, hi0=1.0, lo1=-1.0, hi1=1.0)


@pytest.fixture(scope="module")
def sphere1():
    return I.sphere_vortex(16.0, 2.0, seed=0)


def test_config1_amplitudes_and_responses(sphere1):
    f = sphere1
    plan = run_plan(f, CFG1)
    g = oracle_grid(CFG1)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    F = nms.nms_get_amplitudes(plan)
    err = amp_error(F, F_ref, weight_sums(f))
    assert np.all(err <= AMP_TOL), err
    ref = S.responses(F_ref, g[2], g[3])
    tol = resp_tol(f)
    for name in nms.RESPONSE_NAMES:
        got = nms.nms_response(plan, name)
        assert np.max(np.abs(got - ref[name])) <= tol, name


def test_config1_azimuthal_and_correlation(sphere1):
    f = sphere1
    plan = run_plan(f, CFG1)
    g = oracle_grid(CFG1)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    ref = S.responses(F_ref, g[2], g[3])
    edges = np.linspace(0.0, 1.0, 65)
    r = np.linspace(0.0, 40.0, 64)
    for name in ("UNPOL", "SF"):
        img = nms.nms_response(plan, name)
        Ig, cg, qg = nms.nms_azimuthal_average(plan, img, edges)
        Ir, cr, qr = S.azimuthal_average_cartesian(ref[name], g[4], edges)
        assert np.array_equal(cg, cr)                       # integer work: bit-exact
        assert np.array_equal(np.isnan(Ig), np.isnan(Ir))
        assert iq_rel_error(Ig, Ir) <= IQ_TOL
        np.testing.assert_allclose(qg[cg > 0], qr[cr > 0], rtol=1e-13)
        # correlation through the library from the library's I(q)
        c, p = nms.nms_correlation(qg, Ig, r)
        c_ref, p_ref = S.correlation(qr, Ir, r)
        np.testing.assert_allclose(c, c_ref, rtol=1e-5, atol=1e-5 * np.max(np.abs(c_ref)))
        np.testing.assert_allclose(p, p_ref, rtol=1e-5, atol=1e-5 * np.max(np.abs(p_ref)))


def test_correlation_kernel_exact_inputs():
    rng = np.random.default_rng(3)
    q = np.sort(rng.uniform(0, 2, 301))
    Iq = np.exp(-q * 3) + 0.1
    Iq[[5, 77]] = np.nan           # empty bins are skipped
    r = np.linspace(0, 30, 97)
    c, p = nms.nms_correlation(q, Iq, r, prefactor=0.0)
    c_ref, p_ref = S.correlation(q, Iq, r)
    np.testing.assert_allclose(c, c_ref, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(p, p_ref, rtol=1e-12, atol=1e-12)
    c1, _ = nms.nms_correlation(q, Iq, r, prefactor=1.0)
    np.testing.assert_allclose(c1, c_ref * 2 * np.pi ** 2, rtol=1e-12, atol=1e-13)


def test_polar_grid_and_average():
    f = I.linear_vortex_sphere(10.0, 1.0, M0=1.0, N0=0.7)
    kw = dict(kind="polar", n0=33, n1=48, lo0=0.0, hi0=1.2)
    plan = run_plan(f, kw)
    g = oracle_grid(kw)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f)) <= AMP_TOL)
    ref = S.responses(F_ref, g[2], g[3])
    for name in ("M", "CHI", "NM", "SANSPOL_P"):
        img = nms.nms_response(plan, name)
        assert np.max(np.abs(img - ref[name])) <= resp_tol(f)
        Ig, cg, qg = nms.nms_azimuthal_average(plan, img, nbins=33)
        Ir = S.azimuthal_average_polar(ref[name], 33, 48)
        assert np.all(cg == 48)
        if name != "CHI":
            assert iq_rel_error(Ig, Ir) <= IQ_TOL
        else:
            assert np.max(np.abs(Ig)) <= resp_tol(f)


def test_list_grid_large_phase():
    # arbitrary q points with |q.r| up to ~ 2000 rad: the compensated phase matters
    f = I.box_field(32, 48, 40, a=2.0, n_modes=16, n_pores=10, seed=5)
    rng = np.random.default_rng(9)
    ql = rng.uniform(-40.0, 40.0, size=(301, 2))
    kw = dict(kind="list", n0=301, qlist=ql)
    plan = run_plan(f, kw)
    g = S.q_grid("list", qlist=ql)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    F = nms.nms_get_amplitudes(plan)
    err = amp_error(F, F_ref, weight_sums(f))
    assert np.all(err <= AMP_TOL), err
    # the naive FP32 phase is visibly worse at these phases
    plan_n = run_plan(f, kw, prec=nms.PREC_FP32_NAIVE)
    err_n = amp_error(nms.nms_get_amplitudes(plan_n), F_ref, weight_sums(f))
    assert np.max(err_n) > 10 * np.max(err)


def test_objects_dilute_and_interference():
    f = I.small_random_field(900, seed=21, extent=6.0, n_objects=7)
    # one empty object and one single-cell object
    off = f.offsets.copy()
    off = np.concatenate([off[:3], [off[2]], [off[2] + 1], off[3:]])
    cen = np.vstack([f.centers[:2], [[5.0, -3.0, 2.0]], [[1.0, 1.0, 1.0]], f.centers[2:]])
    f = I.Field(f.pos, f.vol, f.nuc, f.mag, offsets=off, centers=cen)
    kw = dict(kind="cartesian", n0=37, n1=29, lo0=-1.3, hi0=1.1, lo1=-0.9, hi1=1.4)
    R = S.sample_rotation(25.0, 140.0)
    plan = run_plan(f, kw, rot=R[None], want_dilute=1, volume_V=3.5, b_H=0.8, P=(0.3, 0.1, 0.9))
    g = oracle_grid(kw)
    P = np.array([0.3, 0.1, 0.9]) / np.linalg.norm([0.3, 0.1, 0.9])
    ids = ("N", "M", "P", "NM", "CHI", "SANSPOL_M", "UNPOL", "G_XY_IM")
    parts = S.response_parts(f, R, g, ids=ids, P=P, b_H=0.8, V=3.5)
    tol = resp_tol(f, b=0.8, V=3.5, rotations=[R]) * 2
    for name in ids:
        for k, part in enumerate((nms.PART_TOTAL, nms.PART_DILUTE, nms.PART_INTERFERENCE)):
            got = nms.nms_response(plan, name, part)
            assert np.max(np.abs(got - parts[name][k])) <= tol, (name, part)


def test_rotation_average():
    f = I.ellipsoid_uniform((8.0, 5.0, 5.0), a=1.0, seed=2)
    Rs = I.random_rotations(5, seed=11)
    kw = dict(kind="cartesian", n0=24, n1=20, lo0=-1.0, hi0=1.0, lo1=-1.0, hi1=1.0)
    plan = run_plan(f, kw, rot=Rs)
    g = oracle_grid(kw)
    acc = None
    for R in Rs:
        r = S.responses(S.amplitudes(f, R, g[0], g[1]), g[2], g[3])
        acc = r if acc is None else {k: acc[k] + r[k] for k in acc}
    for name in ("UNPOL", "SF", "CHI", "M"):
        got = nms.nms_response(plan, name)
        assert np.max(np.abs(got - acc[name] / 5)) <= resp_tol(f, rotations=Rs)
    # the last rotation's amplitude is kept
    F_ref = S.amplitudes(f, Rs[-1], g[0], g[1])
    assert np.all(amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(f, Rs[-1])) <= AMP_TOL)


@pytest.mark.parametrize("n", [1, 7, 513, 4099])
def test_ragged_sizes_and_channels(n):
    f = I.small_random_field(n, seed=n, extent=4.0)
    kw = dict(kind="cartesian", n0=3, n1=515, lo0=-0.5, hi0=0.7, lo1=-2.0, hi1=2.0)
    for nuc, mag in ((f.nuc, None), (None, f.mag), (f.nuc, f.mag)):
        ff = I.Field(f.pos, f.vol, nuc, mag)
        plan = run_plan(ff, kw)
        g = oracle_grid(kw)
        F_ref = S.amplitudes(ff, np.eye(3), g[0], g[1])
        F = nms.nms_get_amplitudes(plan)
        ws = weight_sums(ff)
        assert np.all(amp_error(F, F_ref, ws) <= AMP_TOL)
        for c in range(4):
            if ws[c] == 0:
                assert np.all(F[c] == 0)


def test_q_zero_pixel_is_weight_sum():
    f = I.sphere_vortex(6.0, 1.0, seed=4)
    kw = dict(kind="cartesian", n0=5, n1=5, lo0=-1.0, hi0=1.0, lo1=-1.0, hi1=1.0)   # centre pixel q = 0
    plan = run_plan(f, kw)
    F = nms.nms_get_amplitudes(plan)
    w = S.cell_weights(f.vol, f.nuc, f.mag, np.eye(3))
    np.testing.assert_allclose(F[:, 12].real, w.sum(1), rtol=0, atol=1e-6 * np.abs(w).sum(1).max())
    assert np.max(np.abs(F[:, 12].imag)) <= 1e-6 * np.abs(w).sum(1).max()


def test_device_output_pointers():
    torch = pytest.importorskip("torch")
    f = I.sphere_vortex(8.0, 2.0, seed=1)
    plan = run_plan(f, CFG1)
    host = nms.nms_response(plan, "SF")
    dev = torch.empty(plan.npix, dtype=torch.float64, device="cuda")
    nms.nms_response(plan, "SF", out=dev)
    assert np.array_equal(dev.cpu().numpy(), host)
    Fd = torch.empty(8 * plan.npix, dtype=torch.float64, device="cuda")
    nms.nms_get_amplitudes(plan, Fd)
    Fh = nms.nms_get_amplitudes(plan)
    b = Fd.cpu().numpy().reshape(4, -1, 2)
    assert np.array_equal(b[..., 0] + 1j * b[..., 1], Fh)


def test_errors_reported_on_bad_calls():
    f = I.sphere_vortex(4.0, 2.0, seed=1)
    g = nms.make_grid("cartesian", 4, 4, -1, 1, -1, 1)
    plan = nms.plan_from_field(f, g, nms.nms_options_default(precision=DIRECT))
    with pytest.raises(nms.NmsError) as e:
        nms.nms_response(plan, "N")                  # before nms_amplitudes
    assert e.value.status == 6
    nms.nms_amplitudes(plan)
    with pytest.raises(nms.NmsError) as e:
        nms.nms_response(plan, "N", nms.PART_DILUTE)  # want_dilute not set
    assert e.value.status == 4
    with pytest.raises(nms.NmsError) as e:
        nms.nms_response(plan, 99)
    assert e.value.status == 1
    with pytest.raises(nms.NmsError) as e:      # the tensor path takes CARTESIAN and POLAR grids only
        nms.nms_plan_create(f.pos, grid=nms.make_grid("list", 3, qlist=np.zeros((3, 2))),
                            opt=nms.nms_options_default(precision=nms.PREC_TC_F16X3))
    assert e.value.status == 1


def test_stage_timing_counts_launches():
    f = I.sphere_vortex(8.0, 2.0, seed=1)
    plan = run_plan(f, CFG1, timing=1)
    st = nms.nms_plan_stage_ms(plan)
    assert st["direct"][1] == 1 and st["direct"][0] > 0
    assert st["prep"][1] == 1 and st["gacc"][1] == 1
