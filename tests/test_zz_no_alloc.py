"""The no-allocation entry point against the plan API's direct path.

nms_dsft_direct_noalloc serves callers that cannot let the library allocate
device memory (their allocator owns the device memory, or a cudaMalloc in a
latency-critical loop would stall the device).  It must give the same sums
as a plan with identity rotation, a LIST grid and the FP32_DIRECT path,
within the amplitude bar of the other tests, on consecutive calls that share
its static scratch array.  This file sorts last so that a run stopping at the
first failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2601_18444_gb300 import inputs as I
from paper_2601_18444_gb300 import nms
from parity_util import AMP_TOL

pytestmark = pytest.mark.gpu


def _case(n_cells, n_q, seed):
    f = I.small_random_field(n_cells, seed=seed, extent=30.0)
    rng = np.random.default_rng(seed + 1)
    ql = rng.uniform(-3.0, 3.0, size=(n_q, 2))
    w = np.stack([f.vol * f.nuc, f.vol * f.mag[:, 0], f.vol * f.mag[:, 1], f.vol * f.mag[:, 2]])
    return f, ql, w


def _plan_reference(f, ql):
    g = nms.make_grid("list", len(ql), qlist=ql)
    plan = nms.plan_from_field(f, g, nms.nms_options_default(precision=nms.PREC_FP32_DIRECT))
    nms.nms_amplitudes(plan)
    F = nms.nms_get_amplitudes(plan)
    plan.close()
    return F


def test_noalloc_matches_plan_direct_on_consecutive_calls():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    dev = "cuda"
    # two calls in a row with different sizes: the second reuses the scratch
    for n_cells, n_q, seed in ((5000, 3001, 11), (1234, 777, 12)):
        f, ql, w = _case(n_cells, n_q, seed)
        Y = torch.tensor(f.pos[:, 1], dtype=torch.float64, device=dev)
        Z = torch.tensor(f.pos[:, 2], dtype=torch.float64, device=dev)
        W = torch.tensor(w, dtype=torch.float64, device=dev).contiguous()
        qy = torch.tensor(ql[:, 0], dtype=torch.float64, device=dev)
        qz = torch.tensor(ql[:, 1], dtype=torch.float64, device=dev)
        F = torch.full((4, n_q, 2), float("nan"), dtype=torch.float64, device=dev)
        nms.nms_dsft_direct_noalloc(Y, Z, W, qy, qz, F, stream=torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        got = F.cpu().numpy()
        got = got[..., 0] + 1j * got[..., 1]
        ref = _plan_reference(f, ql)
        wsum = np.abs(w).sum(axis=1)
        err = np.max(np.abs(got - ref), axis=1) / wsum
        assert np.all(err <= AMP_TOL), err


def test_noalloc_rejects_oversized_grid():
    torch = pytest.importorskip("torch")
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = torch.zeros(262145, dtype=torch.float64, device="cuda")
    with pytest.raises(nms.NmsError) as e:
        nms.nms_dsft_direct_noalloc(z, z, torch.zeros(4, dtype=torch.float64, device="cuda"), big, big,
                                    torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert e.value.status == 1 and "scratch capacity" in str(e.value)
