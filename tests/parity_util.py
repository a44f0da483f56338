"""Shared helpers of the GPU parity tests: oracle evaluation and error metrics.

The error metrics are those the tensor-core/FP32 comparison is stated in:
  amplitude: max over pixels of |F_gpu - F_oracle| / sum_j |w_cj|, per channel c
             (bar 1e-6);
  I(q):      relative error of the azimuthal average where I > 1e-8 I(q_0)
             (bar 1e-5).
Responses (quadratic in F) are compared with the bound that the amplitude bar
implies: |d resp| <= 4e-6 s (sum|w_N| + b sum|w_M|)^2 (s = 1/V), plus the
same relative slack.
"""
import numpy as np

from oracle import sans as S

AMP_TOL = 1e-6
IQ_TOL = 1e-5


def grid_arrays(kind, n0, n1=1, lo0=0.0, hi0=0.0, lo1=0.0, hi1=0.0, qlist=None):
    return S.q_grid(kind, n0, n1, lo0, hi0, lo1, hi1, qlist)


def weight_sums(field, R=np.eye(3)):
    w = S.cell_weights(field.vol, field.nuc, field.mag, R)
    return np.abs(w).sum(axis=1)


def amp_error(F_gpu, F_ref, wsum):
    """Per channel: max_p |dF| / sum_j |w_cj| (channels with zero weight skipped)."""
    err = np.zeros(4)
    for c in range(4):
        if wsum[c] > 0:
            err[c] = np.max(np.abs(F_gpu[c] - F_ref[c])) / wsum[c]
    return err


def resp_tol(field, b=1.0, V=1.0, rotations=None):
    ws = []
    for R in (rotations if rotations is not None else [np.eye(3)]):
        w = weight_sums(field, R)
        ws.append(w[0] + b * (w[1] + w[2] + w[3]))
    return 4e-6 * max(ws) ** 2 / V


def iq_rel_error(I_gpu, I_ref):
    ok = np.isfinite(I_ref)
    ref0 = I_ref[ok][0]
    sel = ok & (np.abs(I_ref) > 1e-8 * abs(ref0))
    return np.max(np.abs(I_gpu[sel] - I_ref[sel]) / np.abs(I_ref[sel]))
