"""The no-allocation entry point against the FP64 oracle.

nms_dsft_direct_noalloc serves callers that cannot let the library allocate
device memory (their allocator owns the device memory, or a cudaMalloc in a
latency-critical loop would stall the device).  It must give the oracle's
direct sums F[c][p] = sum_j w[c][j] exp(-i (qy_p Y_j + qz_p Z_j)) within the
amplitude bar of the other tests, on consecutive calls that share its static
scratch array, allocate no device memory doing so (the free device memory is
unchanged across a call after the first), and handle the edge sizes: the
largest grid the scratch admits (n_q = 262144, one split), no cells (zeros)
and no q-points (nothing written).  This file sorts last so that a run
stopping at the first failure has already run every other test.
"""
import numpy as np
import pytest

from oracle import sans as S
from paper_2601_18444_gb300 import inputs as I
from paper_2601_18444_gb300 import nms
from parity_util import AMP_TOL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MAX_Q = 262144


def _case(n_cells, n_q, seed):
    f = I.small_random_field(n_cells, seed=seed, extent=30.0)
    rng = np.random.default_rng(seed + 1)
    ql = rng.uniform(-3.0, 3.0, size=(n_q, 2))
    w = S.cell_weights(f.vol, f.nuc, f.mag, np.eye(3))
    return f, ql, w


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _call(f, ql, w, F=None):
    n_q = len(ql)
    if F is None:
        F = torch.full((4, n_q, 2), float("nan"), dtype=torch.float64, device="cuda")
    nms.nms_dsft_direct_noalloc(_dev(f.pos[:, 1]), _dev(f.pos[:, 2]), _dev(w), _dev(ql[:, 0]), _dev(ql[:, 1]), F,
                                stream=torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    got = F.cpu().numpy()
    return got[..., 0] + 1j * got[..., 1]


def _check_against_oracle(f, ql, w, got):
    ref = S.dsft(f.pos[:, 1], f.pos[:, 2], w, ql[:, 0], ql[:, 1])
    wsum = np.abs(w).sum(axis=1)
    err = np.max(np.abs(got - ref), axis=1) / wsum
    assert np.all(err <= AMP_TOL), err


def test_noalloc_matches_oracle_on_consecutive_calls():
    assert torch.cuda.is_available()
    # two calls in a row with different sizes: the second reuses the scratch
    for n_cells, n_q, seed in ((5000, 3001, 11), (1234, 777, 12)):
        f, ql, w = _case(n_cells, n_q, seed)
        _check_against_oracle(f, ql, w, _call(f, ql, w))


def test_noalloc_allocates_no_device_memory():
    f, ql, w = _case(3000, 2048, 21)
    args = [_dev(f.pos[:, 1]), _dev(f.pos[:, 2]), _dev(w), _dev(ql[:, 0]), _dev(ql[:, 1])]
    F = torch.empty((4, len(ql), 2), dtype=torch.float64, device="cuda")
    nms.nms_dsft_direct_noalloc(*args, F)          # first call: symbol lookup, module loaded
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        nms.nms_dsft_direct_noalloc(*args, F)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    got = F.cpu().numpy()
    _check_against_oracle(f, ql, w, got[..., 0] + 1j * got[..., 1])


def test_noalloc_largest_grid_single_split():
    f, ql, w = _case(600, MAX_Q, 31)
    _check_against_oracle(f, ql, w, _call(f, ql, w))


def test_noalloc_no_cells_gives_zeros_and_no_q_points_is_a_no_op():
    _, ql, _ = _case(1, 500, 41)
    empty = torch.zeros(0, dtype=torch.float64, device="cuda")
    F = torch.full((4, 500, 2), float("nan"), dtype=torch.float64, device="cuda")
    nms.nms_dsft_direct_noalloc(empty, empty, torch.zeros((4, 0), dtype=torch.float64, device="cuda"),
                                _dev(ql[:, 0]), _dev(ql[:, 1]), F)
    torch.cuda.synchronize()
    assert torch.count_nonzero(F).item() == 0
    f, _, w = _case(100, 1, 42)
    G = torch.full((4, 0, 2), 0.0, dtype=torch.float64, device="cuda")
    nms.nms_dsft_direct_noalloc(_dev(f.pos[:, 1]), _dev(f.pos[:, 2]), _dev(w), empty, empty, G)
    torch.cuda.synchronize()


def test_noalloc_rejects_oversized_grid():
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    big = torch.zeros(MAX_Q + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(nms.NmsError) as e:
        nms.nms_dsft_direct_noalloc(z, z, torch.zeros(4, dtype=torch.float64, device="cuda"), big, big,
                                    torch.zeros(8 * (MAX_Q + 1), dtype=torch.float64, device="cuda"))
    assert e.value.status == 1 and "scratch capacity" in str(e.value)
