"""Surrogate workflow: training curves from the batched transform, then the MLP.

The orientation-averaged, azimuthally averaged unpolarized cross section of
every member of the vortex-particle family is computed in ONE plan: each
member is an object of a dilute sample, all members see the same set of
orientations, and nms_plan_object_iq bins each object's own |F_k|-based
response inside the tensor-core engine.  The surrogate (nms_surrogate_*)
then learns log10 I(q) from the six family parameters.  This module only
arranges arrays and calls the C ABI.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs as I
from . import nms


def family_field(params, a=2.0):
    """All members as objects of one dilute field (no centres)."""
    members = [I.vortex_family_member(p, a) for p in params]
    off = np.zeros(len(members) + 1, dtype=np.int64)
    off[1:] = np.cumsum([m.n for m in members])
    return I.Field(np.concatenate([m.pos for m in members]), np.concatenate([m.vol for m in members]),
                   np.concatenate([m.nuc for m in members]), np.concatenate([m.mag for m in members]),
                   offsets=off, name=f"vortex_family_x{len(members)}")


def default_grid(q_max=1.2, n=128):
    return dict(kind="cartesian", n0=n, n1=n, lo0=-q_max, hi0=q_max, lo1=-q_max, hi1=q_max)


def generate_curves(params, edges, a=2.0, n_rot=16, grid=None, rot_seed=11, response="UNPOL", stream=None):
    """Exact orientation-averaged I(q) [n, nbins] of every parameter row.

    Returns (I, qmean, seconds, terms): wall time of the transform (plan
    creation included) and the number of cell x q-point terms it evaluated.
    """
    grid = grid or default_grid()
    f = family_field(params, a)
    rot = I.random_rotations(n_rot, seed=rot_seed)
    g = nms.make_grid(**grid)
    opt = nms.nms_options_default(precision=nms.PREC_TC_F16X3, want_dilute=1)
    t0 = time.perf_counter()
    plan = nms.plan_from_field(f, g, opt, rot=rot, stream=stream)
    nms.nms_plan_object_iq(plan, response, edges)
    nms.nms_amplitudes(plan)
    Iq, counts, qmean = nms.nms_get_object_iq(plan, len(params))
    dt = time.perf_counter() - t0
    plan.close()
    terms = float(f.n) * plan.npix * n_rot
    return Iq, qmean, dt, terms


def log_targets(Iq, floor=1e-30):
    return np.ascontiguousarray(np.log10(np.maximum(Iq, floor)), dtype=np.float32)
