"""Failure handling on the GPU without a fault: a device wait that nothing
satisfies gives up after its limit, the kernel returns an error status the
host reads (NMS_ERR_TIMEOUT), and the CUDA context keeps working."""
import time

import numpy as np
import pytest

from oracle import sans as S
from paper_2601_18444_gb300 import inputs as I
from paper_2601_18444_gb300 import nms

pytestmark = pytest.mark.gpu


def test_bounded_wait_runs_out_and_context_stays_usable():
    t0 = time.perf_counter()
    with pytest.raises(nms.NmsError) as e:
        nms.nms_selftest_bounded_wait(20000)          # 20 ms on a barrier nothing arrives on
    dt = time.perf_counter() - t0
    assert e.value.status == 5, e.value
    assert 0.02 <= dt < 5.0, dt
    # the hot path still runs and is still right
    f = I.sphere_vortex(6.0, 2.0, seed=3)
    kw = dict(kind="cartesian", n0=16, n1=16, lo0=-1.0, hi0=1.0, lo1=-1.0, hi1=1.0)
    plan = nms.plan_from_field(f, nms.make_grid(**kw), nms.nms_options_default())
    nms.nms_amplitudes(plan)
    g = S.q_grid("cartesian", 16, 16, -1.0, 1.0, -1.0, 1.0)
    F_ref = S.amplitudes(f, np.eye(3), g[0], g[1])
    ws = np.abs(S.cell_weights(f.vol, f.nuc, f.mag, np.eye(3))).sum(1)
    F = nms.nms_get_amplitudes(plan)
    assert max(np.max(np.abs(F[c] - F_ref[c])) / ws[c] for c in range(4)) <= 1e-6


def test_selftest_argument_errors():
    with pytest.raises(nms.NmsError) as e:
        nms.nms_selftest_bounded_wait(0)
    assert e.value.status == 1
