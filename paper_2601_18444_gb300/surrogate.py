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

import multiprocessing as mp
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


def _member_arrays(args):
    """Worker: the concatenated arrays of a slice of family members."""
    rows, a = args
    members = [I.vortex_family_member(p, a) for p in rows]
    n = np.array([m.n for m in members], dtype=np.int64)
    return (np.concatenate([m.pos for m in members]), np.concatenate([m.vol for m in members]),
            np.concatenate([m.nuc for m in members]), np.concatenate([m.mag for m in members]), n)


def _family_async(pool, rows, a, parts=64):
    """Start building one chunk's family field on the worker pool."""
    slices = [x for x in np.array_split(rows, min(parts, len(rows))) if len(x)]
    return pool.map_async(_member_arrays, [(x, a) for x in slices])


def _family_assemble(res, n_members):
    n = np.concatenate([r[4] for r in res])
    off = np.zeros(len(n) + 1, dtype=np.int64)
    off[1:] = np.cumsum(n)
    return I.Field(np.concatenate([r[0] for r in res]), np.concatenate([r[1] for r in res]),
                   np.concatenate([r[2] for r in res]), np.concatenate([r[3] for r in res]), offsets=off,
                   name=f"vortex_family_x{n_members}")


def generate_curves_chunked(params, edges, a=2.5, n_rot=256, grid=None, rot_seed=11, chunk=8000, workers=16,
                            response="UNPOL", stream=None):
    """generate_curves for a large family: members in chunks of ``chunk`` per
    plan (every chunk sees the same orientations); the member lattices of the
    next chunk are built by ``workers`` spawned processes while the GPU works
    on the current one.  Returns (I [n, nbins], qmean, transform seconds,
    terms, host seconds spent waiting for member arrays)."""
    grid = grid or default_grid()
    rot = I.random_rotations(n_rot, seed=rot_seed)
    g = nms.make_grid(**grid)
    opt = nms.nms_options_default(precision=nms.PREC_TC_F16X3, want_dilute=1)
    chunks = [params[i:i + chunk] for i in range(0, len(params), chunk)]
    out, qmean = [], None
    t_gpu, t_host, terms = 0.0, 0.0, 0.0
    with mp.get_context("spawn").Pool(workers) as pool:
        pending = _family_async(pool, chunks[0], a)
        for ci, rows in enumerate(chunks):
            t0 = time.perf_counter()
            f = _family_assemble(pending.get(), len(rows))
            t_host += time.perf_counter() - t0
            if ci + 1 < len(chunks):
                pending = _family_async(pool, chunks[ci + 1], a)
            t0 = time.perf_counter()
            plan = nms.plan_from_field(f, g, opt, rot=rot, stream=stream)
            nms.nms_plan_object_iq(plan, response, edges)
            nms.nms_amplitudes(plan)
            Iq, counts, qmean = nms.nms_get_object_iq(plan, len(rows))
            terms += float(f.n) * plan.npix * n_rot
            plan.close()
            t_gpu += time.perf_counter() - t0
            out.append(Iq)
            del f
    return np.concatenate(out), qmean, t_gpu, terms, t_host
