"""GPU parity of loop mode (weight sets): S magnetization states of one
geometry computed in one plan -- stacked along the GEMM rows on the tensor
path, one pass per set on the direct path -- each against the oracle run on
that state alone (paper, Sec. "Program description": loop modes over field-,
temperature- or time-dependent data sets)."""
import numpy as np
import pytest

from oracle import sans as S
from paper_2601_18444_gb300 import inputs as I
from paper_2601_18444_gb300 import nms
from parity_util import AMP_TOL, amp_error, resp_tol, weight_sums

pytestmark = pytest.mark.gpu


def og(grid_kw):
    kw = dict(grid_kw)
    kind = kw.pop("kind")
    return S.q_grid(kind, **kw)


def state(field, nuc, mag, s):
    return I.Field(field.pos, field.vol, nuc[s], mag[s], offsets=field.offsets, centers=field.centers,
                   name=f"state{s}")


@pytest.mark.parametrize("prec,n_states", [(nms.PREC_TC_F16X3, 3), (nms.PREC_TC_F16X3, 8),
                                           (nms.PREC_FP32_DIRECT, 3)])
def test_weight_sets_match_oracle_per_state(prec, n_states):
    f = I.box_field(24, 20, 16, a=2.0, n_modes=6, n_pores=4, seed=9)
    nuc, mag = I.field_sweep(f, np.linspace(0.0, 2.5, n_states))
    kw = dict(kind="cartesian", n0=40, n1=56, lo0=-1.2, hi0=1.0, lo1=-1.1, hi1=1.3)
    g = nms.make_grid(**kw)
    opt = nms.nms_options_default(precision=prec, n_sets=n_states)
    plan = nms.nms_plan_create(f.pos, f.vol, nuc, mag, grid=g, opt=opt)
    nms.nms_amplitudes(plan)
    q = og(kw)
    for s in range(n_states):
        fs = state(f, nuc, mag, s)
        nms.nms_select_set(plan, s)
        F_ref = S.amplitudes(fs, np.eye(3), q[0], q[1])
        err = amp_error(nms.nms_get_amplitudes(plan), F_ref, weight_sums(fs))
        assert np.all(err <= AMP_TOL), (s, err)
        ref = S.responses(F_ref, q[2], q[3])
        for name in ("UNPOL", "SF", "CHI"):
            assert np.max(np.abs(nms.nms_response(plan, name) - ref[name])) <= resp_tol(fs), (s, name)


def test_weight_sets_with_objects_and_rotations():
    # 3 states x 6 objects (dilute, total, interference) x 2 orientations
    f = I.small_random_field(1500, seed=5, extent=5.0, n_objects=6)
    nuc, mag = I.field_sweep(f, [0.0, 0.7, 4.0])
    kw = dict(kind="cartesian", n0=36, n1=40, lo0=-1.0, hi0=1.2, lo1=-1.1, hi1=0.9)
    Rs = I.random_rotations(2, seed=4)
    opt = nms.nms_options_default(precision=nms.PREC_TC_F16X3, want_dilute=1, n_sets=3)
    plan = nms.nms_plan_create(f.pos, f.vol, nuc, mag, f.offsets, f.centers, Rs, grid=nms.make_grid(**kw), opt=opt)
    nms.nms_amplitudes(plan)
    q = og(kw)
    ids = ("N", "M", "SF", "UNPOL")
    for s in (2, 0, 1):
        fs = state(f, nuc, mag, s)
        acc = {k: [0, 0, 0] for k in ids}
        for R in Rs:
            parts = S.response_parts(fs, R, q, ids=ids)
            for k in ids:
                for i in range(3):
                    acc[k][i] = acc[k][i] + parts[k][i] / len(Rs)
        tol = 2 * resp_tol(fs, rotations=Rs)
        nms.nms_select_set(plan, s)
        for k in ids:
            for i, part in enumerate((nms.PART_TOTAL, nms.PART_DILUTE, nms.PART_INTERFERENCE)):
                assert np.max(np.abs(nms.nms_response(plan, k, part) - acc[k][i])) <= tol, (s, k, part)


def test_single_set_plan_unchanged_by_stacking():
    # the same state as set 2 of a 5-set plan and as a plan of its own agree
    f = I.sphere_vortex(12.0, 2.0, seed=1)
    nuc, mag = I.field_sweep(f, [0.0, 0.3, 0.9, 2.0, 5.0])
    kw = dict(kind="cartesian", n0=64, n1=64, lo0=-1.0, hi0=1.0, lo1=-1.0, hi1=1.0)
    g = nms.make_grid(**kw)
    p5 = nms.nms_plan_create(f.pos, f.vol, nuc, mag, grid=g,
                             opt=nms.nms_options_default(precision=nms.PREC_TC_F16X3, n_sets=5))
    nms.nms_amplitudes(p5)
    nms.nms_select_set(p5, 2)
    p1 = nms.nms_plan_create(f.pos, f.vol, nuc[2], mag[2], grid=g,
                             opt=nms.nms_options_default(precision=nms.PREC_TC_F16X3))
    nms.nms_amplitudes(p1)
    err = amp_error(nms.nms_get_amplitudes(p5), nms.nms_get_amplitudes(p1), weight_sums(state(f, nuc, mag, 2)))
    assert np.all(err <= 2 * AMP_TOL), err


def test_weight_set_errors():
    f = I.small_random_field(50, seed=2, n_objects=2)
    nuc, mag = I.field_sweep(f, [0.0, 1.0])
    g = nms.make_grid("cartesian", 16, 16, -1, 1, -1, 1)
    plan = nms.nms_plan_create(f.pos, f.vol, nuc, mag, f.offsets, None, grid=g,
                               opt=nms.nms_options_default(precision=nms.PREC_TC_F16X3, n_sets=2, want_dilute=1))
    with pytest.raises(nms.NmsError) as e:
        nms.nms_select_set(plan, 2)
    assert e.value.status == 1
    with pytest.raises(nms.NmsError) as e:
        nms.nms_plan_object_iq(plan, "UNPOL", np.linspace(0, 1, 5))
    assert e.value.status == 4
    n33 = np.tile(f.nuc, (33, 1))
    m33 = np.tile(f.mag, (33, 1, 1))
    with pytest.raises(nms.NmsError) as e:
        nms.nms_plan_create(f.pos, f.vol, n33, m33, grid=g,
                            opt=nms.nms_options_default(precision=nms.PREC_TC_F16X3, n_sets=33))
    assert e.value.status == 1
    with pytest.raises(ValueError):
        nms.nms_plan_create(f.pos, f.vol, nuc, mag[:1], grid=g, opt=nms.nms_options_default(n_sets=2))
