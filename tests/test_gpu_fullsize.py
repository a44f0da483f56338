"""Full-size parity of the batched workloads against the FP64 oracle.

Sec. "Summation approach" splits the scattering of many objects into the
sum of their own form factors (dilute part), the full sum with every object
at its position (total) and their difference (interparticle interference).
These tests run the two batched workloads at the sizes they are benchmarked
at and check them where the oracle can follow:

- the 10^4-sphere ensemble (3.67e7 cells, 256^2 detector): the three parts of
  N, M, SF and UNPOL on a seeded sample of pixels (plus the four most
  coherent ones), each against the oracle's per-object and total sums, and
  the per-object unpolarized I(q) of a few objects element by element;
- the ellipsoid under 4096 orientations (204,401 cells, 256^2 detector):
  the amplitude of the last orientation on sampled pixels, the
  orientation-averaged responses on a few pixels over all 4096 orientations,
  and the 128-bin logarithmic I(q) (equal counts, relative error <= 1e-5
  where I > 1e-8 I(q_0)) over a shorter orientation list run by both sides,
  on every eighth non-empty bin.

Bounds: amplitudes max |dF| / sum_j |w_cj| <= 1e-6; a response part within
the bound that implies, 4e-6 (sum |w|)^2, summed over objects for the dilute
part; I(q) relative 1e-5.
"""
import numpy as np
import pytest

from oracle import sans as S
from paper_2601_18444_gb300 import inputs as I
from paper_2601_18444_gb300 import nms
from parity_util import AMP_TOL, IQ_TOL, amp_error, weight_sums

pytestmark = pytest.mark.gpu

TC = nms.PREC_TC_F16X3
IDS = ("N", "M", "SF", "UNPOL")


def _grid(n, lo, hi):
    return dict(kind="cartesian", n0=n, n1=n, lo0=lo, hi0=hi, lo1=lo, hi1=hi)


def _sub(g, idx):
    return tuple(a[idx] for a in g)


def _sample(npix, n, seed, extra=()):
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([rng.choice(npix, n, replace=False), np.asarray(extra, dtype=np.int64)]))


def _centre_pixels(n):
    h = n // 2
    return [(h - 1) * n + h - 1, (h - 1) * n + h, h * n + h - 1, h * n + h]


def test_ensemble_config3_full_size():
    f = I.sphere_ensemble(n_spheres=10000, median=8.0, sigma=0.35, clip=(5.0, 20.0), a=1.0, cube=2000.0, seed=3)
    assert 3.0e7 < f.n < 4.5e7
    kw = _grid(256, -1.0, 1.0)
    plan = nms.plan_from_field(f, nms.make_grid(**kw), nms.nms_options_default(precision=TC, want_dilute=1))
    edges = np.linspace(0.0, 1.0, 129)
    nms.nms_plan_object_iq(plan, "UNPOL", edges)
    nms.nms_amplitudes(plan)
    info = nms.nms_plan_info(plan)
    assert info["precision"] == TC and info["mirror"] == (1, 1)
    g = S.q_grid("cartesian", 256, 256, -1.0, 1.0, -1.0, 1.0)
    idx = _sample(256 * 256, 40, 31, _centre_pixels(256))
    parts = S.response_parts(f, np.eye(3), _sub(g, idx), ids=IDS)
    wk = [np.abs(S.cell_weights(f.vol[a:b], f.nuc[a:b], f.mag[a:b], np.eye(3))).sum(1)
          for a, b in zip(f.offsets[:-1], f.offsets[1:])]
    wt = weight_sums(f)
    tol_tot = 4e-6 * (wt[0] + wt[1] + wt[2] + wt[3]) ** 2
    tol_dil = 4e-6 * sum((w[0] + w[1] + w[2] + w[3]) ** 2 for w in wk)
    for k in IDS:
        for i, (part, tol) in enumerate(((nms.PART_TOTAL, tol_tot), (nms.PART_DILUTE, tol_dil),
                                         (nms.PART_INTERFERENCE, tol_tot + tol_dil))):
            got = nms.nms_response(plan, k, part)[idx]
            assert np.max(np.abs(got - parts[k][i])) <= tol, (k, part)
    # per-object I(q) of a few objects (their own cells, full detector)
    Iobj, counts, _ = nms.nms_get_object_iq(plan, 10000)
    for k in (0, 4321, 9999):
        a, b = f.offsets[k], f.offsets[k + 1]
        fk = I.Field(f.pos[a:b], f.vol[a:b], f.nuc[a:b], f.mag[a:b])
        img = S.responses(S.amplitudes(fk, np.eye(3), g[0], g[1]), g[2], g[3])["UNPOL"]
        Ir, cr, _ = S.azimuthal_average_cartesian(img, g[4], edges)
        assert np.array_equal(counts, cr)
        ok = np.isfinite(Ir)
        np.testing.assert_allclose(Iobj[k][ok], Ir[ok], rtol=IQ_TOL, atol=1e-8 * np.nanmax(Ir))


def test_rotations_config4_full_size():
    f = I.ellipsoid_uniform((40.0, 25.0, 25.0), a=0.8, seed=4)
    assert 2.0e5 < f.n < 2.1e5
    Rs = I.random_rotations(4096, seed=5)
    kw = _grid(256, -2.0, 2.0)
    g = S.q_grid("cartesian", 256, 256, -2.0, 2.0, -2.0, 2.0)
    plan = nms.plan_from_field(f, nms.make_grid(**kw), nms.nms_options_default(precision=TC), rot=Rs)
    nms.nms_amplitudes(plan)
    # amplitude of the last orientation on sampled pixels
    idx = _sample(256 * 256, 60, 41, _centre_pixels(256))
    F_ref = S.amplitudes(f, Rs[-1], g[0][idx], g[1][idx])
    err = amp_error(nms.nms_get_amplitudes(plan)[:, idx], F_ref, weight_sums(f, Rs[-1]))
    assert np.all(err <= AMP_TOL), err
    # orientation-averaged responses over all 4096 orientations on a few pixels
    few = _sample(256 * 256, 4, 42, _centre_pixels(256)[:1])
    gf = _sub(g, few)
    acc = {k: 0.0 for k in IDS}
    for R in Rs:
        r = S.responses(S.amplitudes(f, R, gf[0], gf[1]), gf[2], gf[3])
        for k in IDS:
            acc[k] = acc[k] + r[k]
    # sum_c sum_j |w_cj| <= sum_j V_j (|N_j| + sqrt(3) |M_j|) under every rotation
    wmax = np.sum(f.vol * np.abs(f.nuc)) + np.sqrt(3.0) * np.sum(f.vol * np.linalg.norm(f.mag, axis=1))
    tol = 2 * 4e-6 * wmax ** 2
    for k in IDS:
        got = nms.nms_response(plan, k)[few]
        assert np.max(np.abs(got - acc[k] / len(Rs))) <= tol, k
    plan.close()
    # I(q) on 128 log bins over a shorter orientation list run by both sides
    Rsub = Rs[:8]
    edges = np.geomspace(0.01, 2.0, 129)
    plan = nms.plan_from_field(f, nms.make_grid(**kw), nms.nms_options_default(precision=TC), rot=Rsub)
    nms.nms_amplitudes(plan)
    Ig, cg, _ = nms.nms_azimuthal_average(plan, nms.nms_response(plan, "UNPOL"), edges)
    _, cr, _ = S.azimuthal_average_cartesian(np.zeros(256 * 256), g[4], edges)
    assert np.array_equal(cg, cr)
    nonempty = np.flatnonzero(cr > 0)
    chosen = nonempty[::8]
    sel = np.zeros(256 * 256, dtype=bool)
    for b in chosen:
        sel |= (g[4] >= edges[b]) & (g[4] < edges[b + 1])
    pix = np.flatnonzero(sel)
    gs = _sub(g, pix)
    img = np.zeros(len(pix))
    for R in Rsub:
        img += S.responses(S.amplitudes(f, R, gs[0], gs[1]), gs[2], gs[3])["UNPOL"] / len(Rsub)
    full = np.full(256 * 256, np.nan)
    full[pix] = img
    ref0 = None
    for b in chosen:
        m = (g[4] >= edges[b]) & (g[4] < edges[b + 1])
        Ir = full[m].mean()
        ref0 = Ir if ref0 is None else ref0
        if abs(Ir) > 1e-8 * abs(ref0):
            assert abs(Ig[b] - Ir) <= IQ_TOL * abs(Ir), (b, Ig[b], Ir)
