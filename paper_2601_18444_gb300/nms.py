"""Python binding of libnms (ctypes): the C ABI of include/nms.h, same names.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Host arrays are numpy float64; device arrays are torch CUDA tensors
(passed by ``data_ptr()``).  There is no CPU fallback: if libnms.so is not
built or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

NMS_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "OUT_OF_MEMORY", 3: "CUDA", 4: "UNSUPPORTED", 5: "TIMEOUT",
          6: "BAD_STATE"}

QGRID_CARTESIAN, QGRID_POLAR, QGRID_LIST = 0, 1, 2
PREC_AUTO, PREC_TC_F16X3, PREC_FP32_DIRECT, PREC_FP32_NAIVE = 0, 1, 2, 3
PART_TOTAL, PART_DILUTE, PART_INTERFERENCE = 0, 1, 2

RESPONSE_NAMES = ["N", "M", "P", "NM", "CHI", "SF", "PM", "MP", "PP", "MM", "SANSPOL_P", "SANSPOL_M", "UNPOL"] + \
    [f"G_{a}{b}_{p}" for a in "XYZ" for b in "XYZ" for p in ("RE", "IM")] + ["QX2", "QY2", "QZ2"]
RESPONSE_ID = {n: i for i, n in enumerate(RESPONSE_NAMES)}

STAGES = ["prep", "tables", "gemm", "direct", "reduce", "gacc", "s6", "s7"]


class NmsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"nms {STATUS.get(status, status)}: {msg}")
        self.status = status


class nms_qgrid(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n0", ctypes.c_int32), ("n1", ctypes.c_int32),
                ("lo0", ctypes.c_double), ("hi0", ctypes.c_double), ("lo1", ctypes.c_double),
                ("hi1", ctypes.c_double), ("qlist", ctypes.POINTER(ctypes.c_double))]


class nms_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("want_dilute", ctypes.c_int32), ("volume_V", ctypes.c_double),
                ("b_H", ctypes.c_double), ("P", ctypes.c_double * 3), ("kc_cells", ctypes.c_int32),
                ("split_k", ctypes.c_int32), ("max_spin", ctypes.c_int64), ("workspace_bytes", ctypes.c_int64),
                ("timing", ctypes.c_int32), ("autotune", ctypes.c_int32), ("n_sets", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 5)]


_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I64 = ctypes.POINTER(ctypes.c_int64)
_V = ctypes.c_void_p

# name -> (restype, argtypes); the full C ABI of include/nms.h
SIGNATURES = {
    "nms_options_default": (ctypes.c_int, [ctypes.POINTER(nms_options)]),
    "nms_plan_create": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_int64, _D, _D, _D, _D, ctypes.c_int64, _I64, _D,
                                       ctypes.c_int32, _D, ctypes.POINTER(nms_qgrid), ctypes.POINTER(nms_options),
                                       _V]),
    "nms_amplitudes": (ctypes.c_int, [_V]),
    "nms_get_amplitudes": (ctypes.c_int, [_V, _V, ctypes.c_int32]),
    "nms_response": (ctypes.c_int, [_V, ctypes.c_int32, ctypes.c_int32, _V, ctypes.c_int32]),
    "nms_azimuthal_average": (ctypes.c_int, [_V, _V, ctypes.c_int32, ctypes.c_int32, _D, _V, _V, _V,
                                             ctypes.c_int32]),
    "nms_angular_spectrum": (ctypes.c_int, [_V, _V, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, _D, _V, _V, _V,
                                            _V, _V, _V, ctypes.c_int32]),
    "nms_correlation_2d": (ctypes.c_int, [_V, _V, ctypes.c_int32, ctypes.c_int32, _D, ctypes.c_int32, _D, _V, _V,
                                          ctypes.c_int32]),
    "nms_correlation": (ctypes.c_int, [ctypes.c_int32, _V, _V, ctypes.c_int32, _V, ctypes.c_double, _V, _V,
                                       ctypes.c_int32, _V]),
    "nms_plan_stage_ms": (ctypes.c_int, [_V, _D, _I64, ctypes.c_int32]),
    "nms_plan_object_iq": (ctypes.c_int, [_V, ctypes.c_int32, ctypes.c_int32, _D]),
    "nms_get_object_iq": (ctypes.c_int, [_V, _V, _V, _V, ctypes.c_int32]),
    "nms_surrogate_create": (ctypes.c_int, [ctypes.POINTER(_V), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                            _F, _F, ctypes.c_uint64, _V]),
    "nms_surrogate_set_target_stats": (ctypes.c_int, [_V, _F, _F]),
    "nms_surrogate_train": (ctypes.c_int, [_V, _V, _V, ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                           ctypes.c_uint64, _F]),
    "nms_surrogate_gradients": (ctypes.c_int, [_V, _V, _V, ctypes.c_int32, _F, _D]),
    "nms_surrogate_infer": (ctypes.c_int, [_V, _V, ctypes.c_int64, _V]),
    "nms_surrogate_get_params": (ctypes.c_int, [_V, _F, _I64]),
    "nms_surrogate_set_params": (ctypes.c_int, [_V, _F, ctypes.c_int64]),
    "nms_surrogate_save": (ctypes.c_int, [_V, ctypes.c_char_p]),
    "nms_surrogate_load": (ctypes.c_int, [_V, ctypes.c_char_p]),
    "nms_surrogate_destroy": (ctypes.c_int, [_V]),
    "nms_dsft_direct_noalloc": (ctypes.c_int, [ctypes.c_int64, _V, _V, _V, ctypes.c_int64, _V, _V, _V, _V]),
    "nms_plan_info": (ctypes.c_int, [_V] + [ctypes.POINTER(ctypes.c_int32)] * 6),
    "nms_select_set": (ctypes.c_int, [_V, ctypes.c_int32]),
    "nms_selftest_bounded_wait": (ctypes.c_int, [ctypes.c_int64, _V]),
    "nms_selftest_sincos": (ctypes.c_int, [ctypes.c_int64, _V, _V, _V]),
    "nms_plan_destroy": (ctypes.c_int, [_V]),
    "nms_last_error": (ctypes.c_char_p, []),
    "nms_version": (ctypes.c_char_p, []),
}


def lib_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libnms.so (building it in-tree if needed); raises if it cannot."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing and _build.needs_build():
        _build.build()
    if not os.path.exists(path):
        raise NmsError(3, f"libnms.so not built at {path}")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def _check(st):
    if st != NMS_OK:
        raise NmsError(st, nms_last_error())


def nms_last_error():
    return load().nms_last_error().decode()


def nms_version():
    return load().nms_version().decode()


def _host(a, shape_last=None):
    if a is None:
        return None, None
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_D)


def _is_dev(t):
    return hasattr(t, "is_cuda") and t.is_cuda


def _ptr(t):
    """Raw address of a row-major buffer; strided views are refused (the C ABI
    takes plain row-major arrays)."""
    if _is_dev(t):
        if not t.is_contiguous():
            raise ValueError("device tensor must be contiguous (row-major)")
        return ctypes.c_void_p(t.data_ptr())
    if not t.flags.c_contiguous:
        raise ValueError("host array must be C-contiguous")
    return ctypes.c_void_p(t.ctypes.data)


def _dev_in(t):
    """Device input as a row-major tensor (copies a strided view)."""
    return t.contiguous() if _is_dev(t) else t


def nms_options_default(**kw):
    o = nms_options()
    _check(load().nms_options_default(ctypes.byref(o)))
    for k, v in kw.items():
        if k == "P":
            for i in range(3):
                o.P[i] = float(v[i])
        else:
            setattr(o, k, v)
    return o


def make_grid(kind, n0, n1=1, lo0=0.0, hi0=0.0, lo1=0.0, hi1=0.0, qlist=None):
    g = nms_qgrid()
    g.kind = {"cartesian": 0, "polar": 1, "list": 2}.get(kind, kind)
    g.n0, g.n1 = int(n0), int(n1)
    g.lo0, g.hi0, g.lo1, g.hi1 = float(lo0), float(hi0), float(lo1), float(hi1)
    keep = None
    if qlist is not None:
        keep = np.ascontiguousarray(qlist, dtype=np.float64).reshape(-1)
        g.qlist = keep.ctypes.data_as(_D)
    g._keep = keep
    return g


class Plan:
    """Owning wrapper of an nms_plan_t (destroyed on close/garbage collection)."""

    def __init__(self, handle, npix, grid):
        self.handle = handle
        self.npix = npix
        self.grid = grid

    def close(self):
        if self.handle:
            load().nms_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def nms_plan_create(pos, cell_vol=None, nuc=None, mag=None, object_offsets=None, object_centers=None, rot=None,
                    grid=None, opt=None, stream=None):
    lib = load()
    pos, p_pos = _host(pos)
    n = pos.shape[0]
    vol, p_vol = _host(cell_vol)
    nuc, p_nuc = _host(nuc)
    mag, p_mag = _host(mag)
    cen, p_cen = _host(object_centers)
    # loop mode: nuc [S][n] and mag [S][n][3]; the library trusts the sizes
    S = max(1, int(opt.n_sets)) if opt is not None else 1
    if nuc is not None and nuc.size != S * n:
        raise ValueError(f"nuc must hold n_sets x n_cells = {S} x {n} values")
    if mag is not None and mag.size != 3 * S * n:
        raise ValueError(f"mag must hold n_sets x n_cells x 3 = {S} x {n} x 3 values")
    off = None
    p_off = None
    K = 1
    if object_offsets is not None:
        off = np.ascontiguousarray(object_offsets, dtype=np.int64)
        p_off = off.ctypes.data_as(_I64)
        K = len(off) - 1
    nrot = 1
    R, p_R = None, None
    if rot is not None:
        R = np.ascontiguousarray(rot, dtype=np.float64).reshape(-1, 9)
        nrot = R.shape[0]
        p_R = R.ctypes.data_as(_D)
    h = ctypes.c_void_p()
    _check(lib.nms_plan_create(ctypes.byref(h), n, p_pos, p_vol, p_nuc, p_mag, K, p_off, p_cen, nrot, p_R,
                               ctypes.byref(grid), ctypes.byref(opt) if opt is not None else None,
                               ctypes.c_void_p(stream or 0)))
    npix = grid.n0 * grid.n1 if grid.kind != QGRID_LIST else grid.n0
    return Plan(h, npix, grid)


def nms_amplitudes(plan):
    _check(load().nms_amplitudes(plan.handle))


def nms_get_amplitudes(plan, out=None):
    """Total amplitudes of the last rotation: complex128 [4, npix] (host) or into a device tensor."""
    if out is None:
        buf = np.empty(8 * plan.npix, dtype=np.float64)
        _check(load().nms_get_amplitudes(plan.handle, _ptr(buf), 0))
        b = buf.reshape(4, plan.npix, 2)
        return b[..., 0] + 1j * b[..., 1]
    _check(load().nms_get_amplitudes(plan.handle, _ptr(out), 1 if _is_dev(out) else 0))
    return out


def nms_response(plan, response, part=PART_TOTAL, out=None):
    rid = RESPONSE_ID[response] if isinstance(response, str) else int(response)
    if out is None:
        out = np.empty(plan.npix, dtype=np.float64)
    _check(load().nms_response(plan.handle, rid, part, _ptr(out), 1 if _is_dev(out) else 0))
    return out


def nms_azimuthal_average(plan, img, bin_edges=None, nbins=None):
    """Returns (I, counts, qmean) as host numpy arrays."""
    if bin_edges is not None:
        edges = np.ascontiguousarray(bin_edges, dtype=np.float64)
        nb = len(edges) - 1
        p_e = edges.ctypes.data_as(_D)
    else:
        edges, p_e, nb = None, None, int(nbins)
    img = _dev_in(img) if _is_dev(img) else np.ascontiguousarray(img, dtype=np.float64)
    I = np.empty(nb, dtype=np.float64)
    c = np.empty(nb, dtype=np.int64)
    qm = np.empty(nb, dtype=np.float64)
    _check(load().nms_azimuthal_average(plan.handle, _ptr(img), 1 if _is_dev(img) else 0, nb, p_e, _ptr(I),
                                        _ptr(c), _ptr(qm), 0))
    return I, c, qm


def nms_angular_spectrum(plan, img, kmax, bin_edges=None, nbins=None):
    """Returns dict(Ic, Is [kmax+1][nbins], counts, qmean, Ac, As) as host numpy arrays."""
    if bin_edges is not None:
        edges = np.ascontiguousarray(bin_edges, dtype=np.float64)
        nb = len(edges) - 1
        p_e = edges.ctypes.data_as(_D)
    else:
        edges, p_e, nb = None, None, int(nbins)
    img = _dev_in(img) if _is_dev(img) else np.ascontiguousarray(img, dtype=np.float64)
    K = int(kmax) + 1
    Ic = np.empty((K, nb), dtype=np.float64)
    Is = np.empty((K, nb), dtype=np.float64)
    c = np.empty(nb, dtype=np.int64)
    qm = np.empty(nb, dtype=np.float64)
    Ac = np.empty(K, dtype=np.float64)
    As = np.empty(K, dtype=np.float64)
    _check(load().nms_angular_spectrum(plan.handle, _ptr(img), 1 if _is_dev(img) else 0, int(kmax), nb, p_e,
                                       _ptr(Ic), _ptr(Is), _ptr(c), _ptr(qm), _ptr(Ac), _ptr(As), 0))
    return {"Ic": Ic, "Is": Is, "counts": c, "qmean": qm, "Ac": Ac, "As": As}


def nms_correlation_2d(plan, img, rho, alpha, out=None):
    """C(rho, alpha) of Eq. crav2d.  Returns (C complex [n_rho][n_alpha] host
    array, scale = sum |W f|); with out (a device float64 [n_rho][n_alpha][2]
    tensor) the result stays on the device and (out, scale) is returned."""
    rho = np.ascontiguousarray(rho, dtype=np.float64).ravel()
    alpha = np.ascontiguousarray(alpha, dtype=np.float64).ravel()
    img = _dev_in(img) if _is_dev(img) else np.ascontiguousarray(img, dtype=np.float64)
    lib = load()
    if out is not None:
        import torch
        sc = torch.empty(1, dtype=torch.float64, device=out.device)
        _check(lib.nms_correlation_2d(plan.handle, _ptr(img), 1 if _is_dev(img) else 0, len(rho),
                                      rho.ctypes.data_as(_D), len(alpha), alpha.ctypes.data_as(_D), _ptr(out),
                                      _ptr(sc), 1))
        return out, sc
    C = np.empty((len(rho), len(alpha), 2), dtype=np.float64)
    sc = np.empty(1, dtype=np.float64)
    _check(lib.nms_correlation_2d(plan.handle, _ptr(img), 1 if _is_dev(img) else 0, len(rho),
                                  rho.ctypes.data_as(_D), len(alpha), alpha.ctypes.data_as(_D), _ptr(C), _ptr(sc),
                                  0))
    return C[..., 0] + 1j * C[..., 1], float(sc[0])


def nms_correlation(q, Iq, r, prefactor=0.0, stream=None):
    """c(r), p(r) by the library's trapezoid kernel; host numpy in and out."""
    q = np.ascontiguousarray(q, dtype=np.float64)
    Iq = np.ascontiguousarray(Iq, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    c = np.empty(len(r))
    p = np.empty(len(r))
    _check(load().nms_correlation(len(q), _ptr(q), _ptr(Iq), len(r), _ptr(r), float(prefactor), _ptr(c), _ptr(p),
                                  0, ctypes.c_void_p(stream or 0)))
    return c, p


def nms_correlation_device(q, Iq, r, c, p, prefactor=0.0, stream=None):
    """Device variant: all five arguments are CUDA tensors (float64)."""
    _check(load().nms_correlation(q.numel(), _ptr(q), _ptr(Iq), r.numel(), _ptr(r), float(prefactor), _ptr(c),
                                  _ptr(p), 1, ctypes.c_void_p(stream or 0)))


def nms_plan_stage_ms(plan, reset=False):
    ms = (ctypes.c_double * 8)()
    ln = (ctypes.c_int64 * 8)()
    _check(load().nms_plan_stage_ms(plan.handle, ms, ln, 1 if reset else 0))
    return {STAGES[i]: (ms[i], ln[i]) for i in range(8)}


class Surrogate:
    """Owning wrapper of an nms_surrogate_t."""

    def __init__(self, handle, n_in, n_hidden, n_out):
        self.handle, self.n_in, self.n_hidden, self.n_out = handle, n_in, n_hidden, n_out

    def close(self):
        if self.handle:
            load().nms_surrogate_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _fp(a):
    return a.ctypes.data_as(_F)


def nms_surrogate_create(n_in, n_hidden, n_out, x_lo, x_hi, seed=0, stream=None):
    lo = np.ascontiguousarray(x_lo, dtype=np.float32)
    hi = np.ascontiguousarray(x_hi, dtype=np.float32)
    h = ctypes.c_void_p()
    _check(load().nms_surrogate_create(ctypes.byref(h), n_in, n_hidden, n_out, _fp(lo), _fp(hi), seed,
                                       ctypes.c_void_p(stream or 0)))
    return Surrogate(h, n_in, n_hidden, n_out)


def nms_surrogate_set_target_stats(s, y_mean, y_std):
    m = np.ascontiguousarray(y_mean, dtype=np.float32)
    d = np.ascontiguousarray(y_std, dtype=np.float32)
    _check(load().nms_surrogate_set_target_stats(s.handle, _fp(m), _fp(d)))


def nms_surrogate_train(s, X, Y, batch, epochs, lr, seed=0):
    """X, Y: float32 CUDA tensors [n, n_in], [n, n_out]; returns the last epoch's loss."""
    X, Y = _dev_in(X), _dev_in(Y)
    loss = ctypes.c_float(0.0)
    _check(load().nms_surrogate_train(s.handle, _ptr(X), _ptr(Y), X.shape[0], batch, epochs, lr, seed,
                                      ctypes.byref(loss)))
    return loss.value


def nms_surrogate_gradients(s, X, Y):
    X, Y = _dev_in(X), _dev_in(Y)
    g = np.empty(nms_surrogate_get_params(s, count_only=True), dtype=np.float32)
    loss = ctypes.c_double(0.0)
    _check(load().nms_surrogate_gradients(s.handle, _ptr(X), _ptr(Y), X.shape[0], _fp(g), ctypes.byref(loss)))
    return g, loss.value


def nms_surrogate_infer(s, X, Y):
    X = _dev_in(X)
    _check(load().nms_surrogate_infer(s.handle, _ptr(X), X.shape[0], _ptr(Y)))
    return Y


def nms_surrogate_get_params(s, count_only=False):
    n = ctypes.c_int64(0)
    _check(load().nms_surrogate_get_params(s.handle, None, ctypes.byref(n)))
    if count_only:
        return n.value
    w = np.empty(n.value, dtype=np.float32)
    _check(load().nms_surrogate_get_params(s.handle, _fp(w), ctypes.byref(n)))
    return w


def nms_surrogate_set_params(s, w):
    w = np.ascontiguousarray(w, dtype=np.float32)
    _check(load().nms_surrogate_set_params(s.handle, _fp(w), w.size))


def nms_surrogate_save(s, path):
    _check(load().nms_surrogate_save(s.handle, str(path).encode()))


def nms_surrogate_load(s, path):
    _check(load().nms_surrogate_load(s.handle, str(path).encode()))


def nms_surrogate_destroy(s):
    s.close()


def nms_plan_object_iq(plan, response, bin_edges):
    rid = RESPONSE_ID[response] if isinstance(response, str) else int(response)
    edges = np.ascontiguousarray(bin_edges, dtype=np.float64)
    _check(load().nms_plan_object_iq(plan.handle, rid, len(edges) - 1, edges.ctypes.data_as(_D)))
    plan._oiq_nbins = len(edges) - 1


def nms_get_object_iq(plan, n_objects):
    """(Iq [n_objects, nbins], counts [nbins], qmean [nbins]) as host arrays."""
    nb = plan._oiq_nbins
    I = np.empty((n_objects, nb), dtype=np.float64)
    c = np.empty(nb, dtype=np.int64)
    q = np.empty(nb, dtype=np.float64)
    _check(load().nms_get_object_iq(plan.handle, _ptr(I), _ptr(c), _ptr(q), 0))
    return I, c, q


def _noalloc_args(Y, Z, w, qy, qz, F):
    """Checks of nms_dsft_direct_noalloc's buffers before any device access:
    float64 torch tensors, sizes consistent with n_cells = Y.numel() and
    n_q = qy.numel(), F contiguous, and (last) every tensor on the GPU.
    Raises ValueError on the first mismatch."""
    names = ("Y", "Z", "w", "qy", "qz", "F")
    bufs = (Y, Z, w, qy, qz, F)
    for nm, t in zip(names, bufs):
        if not (hasattr(t, "dtype") and hasattr(t, "numel") and hasattr(t, "is_cuda")):
            raise ValueError(f"{nm} must be a torch tensor")
        if str(t.dtype) != "torch.float64":
            raise ValueError(f"{nm} must be float64, got {t.dtype}")
    n, nq = Y.numel(), qy.numel()
    if Z.numel() != n:
        raise ValueError(f"Z has {Z.numel()} elements, Y has {n}")
    if w.numel() != 4 * n:
        raise ValueError(f"w must hold [4][n_cells] = {4 * n} weights, has {w.numel()}")
    if qz.numel() != nq:
        raise ValueError(f"qz has {qz.numel()} elements, qy has {nq}")
    if F.numel() < 8 * nq:
        raise ValueError(f"F must hold [4][n_q][2] = {8 * nq} values, has {F.numel()}")
    if not F.is_contiguous():
        raise ValueError("F must be contiguous (it is written in place)")
    for nm, t in zip(names, bufs):
        if not t.is_cuda:
            raise ValueError(f"{nm} must be a CUDA tensor (the entry point reads and writes device memory)")
    devs = {t.device for t in bufs}
    if len(devs) != 1:
        raise ValueError(f"all buffers must be on one device, got {sorted(str(d) for d in devs)}")


def nms_dsft_direct_noalloc(Y, Z, w, qy, qz, F, stream=None):
    """Direct sums into a caller-owned device tensor F [4, n_q, 2] without any
    device allocation by the library (all arguments are float64 CUDA tensors
    on one device; checked here before the call)."""
    _noalloc_args(Y, Z, w, qy, qz, F)
    Y, Z, w, qy, qz = (_dev_in(t) for t in (Y, Z, w, qy, qz))
    _check(load().nms_dsft_direct_noalloc(Y.numel(), _ptr(Y), _ptr(Z), _ptr(w), qy.numel(), _ptr(qy), _ptr(qz),
                                          _ptr(F), ctypes.c_void_p(stream or 0)))
    return F


def nms_plan_info(plan):
    """dict(precision, kc_cells, items_per_sm, gemm_form, mirror=(y, z)) the plan settled on."""
    v = [ctypes.c_int32() for _ in range(6)]
    _check(load().nms_plan_info(plan.handle, *[ctypes.byref(x) for x in v]))
    return {"precision": v[0].value, "kc_cells": v[1].value, "items_per_sm": v[2].value, "gemm_form": v[3].value,
            "mirror": (v[4].value, v[5].value)}


def nms_plan_destroy(plan):
    plan.close()


def nms_select_set(plan, s):
    """Loop mode: later nms_get_amplitudes / nms_response calls report weight set s."""
    _check(load().nms_select_set(plan.handle, int(s)))


def nms_selftest_bounded_wait(limit_us, stream=None):
    """Run the bounded-wait self-test; raises NmsError (status TIMEOUT) when the
    device wait gave up, which is the expected outcome."""
    _check(load().nms_selftest_bounded_wait(int(limit_us), ctypes.c_void_p(stream or 0)))


def nms_selftest_sincos(t, stream=None):
    """(n, 4) float32: sin, cos of 2 pi t by the fused ray form's routine, then by sincospif."""
    t = np.ascontiguousarray(t, dtype=np.float32).ravel()
    out = np.empty((t.size, 4), dtype=np.float32)
    _check(load().nms_selftest_sincos(t.size, t.ctypes.data_as(_V), out.ctypes.data_as(_V),
                                      ctypes.c_void_p(stream or 0)))
    return out


def plan_from_field(field, grid, opt=None, rot=None, stream=None):
    """Convenience: nms_plan_create from an inputs.Field."""
    return nms_plan_create(field.pos, field.vol, field.nuc, field.mag, field.offsets, field.centers, rot, grid, opt,
                           stream)
