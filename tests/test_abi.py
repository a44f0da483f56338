"""The C-ABI library builds, loads and exports every symbol include/nms.h declares.

CPU-only: no compute call is made except those that must fail cleanly
without a GPU (no CPU fallback exists).
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2601_18444_gb300 import nms

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "nms.h")


def declared_functions():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(nms_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_abi():
    names = declared_functions()
    for n in ["nms_plan_create", "nms_amplitudes", "nms_response", "nms_azimuthal_average", "nms_correlation",
              "nms_plan_destroy", "nms_last_error", "nms_get_amplitudes", "nms_options_default"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    path = nms.lib_path()
    nms.load()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (nms_[a-z_0-9]+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert sorted(nms.SIGNATURES) == declared_functions()


def test_struct_layouts_match_c(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "nms.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu\\n", sizeof(nms_options), sizeof(nms_qgrid),'
                   ' offsetof(nms_options, timing), offsetof(nms_qgrid, qlist));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    a, b, c, d = map(int, subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split())
    assert a == ctypes.sizeof(nms.nms_options)
    assert b == ctypes.sizeof(nms.nms_qgrid)
    assert c == nms.nms_options.timing.offset
    assert d == nms.nms_qgrid.qlist.offset


def test_response_ids_match_header():
    txt = open(HEADER).read()
    body = txt[txt.index("NMS_RESP_N = 0"):txt.index("NMS_RESP_COUNT")]
    ids = [m.replace("NMS_RESP_", "") for m in re.findall(r"NMS_RESP_[A-Z_0-9]+", body)]
    assert ids == nms.RESPONSE_NAMES


def test_defaults_and_version():
    o = nms.nms_options_default()
    assert o.precision == nms.PREC_AUTO and o.volume_V == 1.0 and o.b_H == 1.0 and tuple(o.P) == (0.0, 0.0, 1.0)
    assert "sm_103a" in nms.nms_version()


def test_invalid_arguments_are_reported_without_gpu():
    g = nms.make_grid("cartesian", 4, 4, -1, 1, -1, 1)
    with pytest.raises(nms.NmsError) as e:
        nms.nms_plan_create(np.zeros((0, 3)), grid=g)
    assert e.value.status == 1
    # with valid arguments and no GPU the library refuses: no CPU fallback
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:
        with pytest.raises(nms.NmsError) as e:
            nms.nms_plan_create(np.zeros((3, 3)), grid=g)
        assert e.value.status == 3
        with pytest.raises(nms.NmsError):
            nms.nms_correlation([0.0, 1.0], [1.0, 1.0], [1.0])


def test_sincos_selftest_checks_arguments_before_the_device():
    lib = nms.load()
    assert lib.nms_selftest_sincos(-1, None, None, None) == 1            # INVALID_ARG
    assert lib.nms_selftest_sincos(3, None, None, None) == 1             # NULL arrays with n > 0
    assert lib.nms_selftest_sincos(0, None, None, None) == 0             # nothing to do
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:
        has_gpu = False
    if not has_gpu:   # valid arguments, no device: refused, no CPU fallback
        with pytest.raises(nms.NmsError) as e:
            nms.nms_selftest_sincos(np.zeros(4, dtype=np.float32))
        assert e.value.status == 3


def test_plan_create_argument_checks_come_before_the_device():
    # the host-side checks of nms_plan_create run before any CUDA call, so each
    # bad argument gives INVALID_ARG (1), not CUDA (3), with or without a GPU
    lib = nms.load()
    g = nms.make_grid("cartesian", 4, 4, -1, 1, -1, 1)
    pos = np.zeros((3, 3))
    p_pos = pos.ctypes.data_as(nms._D)
    rot = np.eye(3).reshape(1, 9).repeat(2, axis=0)
    h = ctypes.c_void_p()

    def create(n, p, K, off, nrot, R, grid=ctypes.byref(g)):
        h.value = 0x1234                                                     # cleared by every failed create
        st = lib.nms_plan_create(ctypes.byref(h), n, p, None, None, None, K, off, None, nrot, R, grid, None, None)
        assert h.value is None
        return st

    assert create(0, p_pos, 1, None, 1, None) == 1                           # no cells
    assert create(3, None, 1, None, 1, None) == 1                            # no positions
    assert create(3, p_pos, 0, None, 1, None) == 1                           # no objects
    assert create(3, p_pos, 2, None, 1, None) == 1                           # K > 1 without offsets
    assert create(3, p_pos, 1, None, 0, None) == 1                           # no orientations
    assert create(3, p_pos, 1, None, 2, None) == 1                           # identity needs n_rot == 1
    assert create(3, p_pos, 1, None, 2, rot.ctypes.data_as(nms._D), grid=None) == 1   # no grid
    assert lib.nms_plan_create(None, 3, p_pos, None, None, None, 1, None, None, 1, None, ctypes.byref(g), None,
                               None) == 1                                     # no output handle
    assert nms.nms_last_error() == "out is NULL"


def test_binding_refuses_strided_buffers():
    a = np.zeros((4, 6))[:, ::2]
    with pytest.raises(ValueError):
        nms._ptr(a)
    f = np.asfortranarray(np.zeros((3, 5)))
    with pytest.raises(ValueError):
        nms._ptr(f)
    assert nms._ptr(np.zeros((3, 5))).value is not None


def test_noalloc_binding_checks_buffers_before_the_call():
    # every malformed buffer is refused by the binding before the library is
    # called: wrong dtype, inconsistent sizes, a short or strided output, and
    # host (CPU) tensors; no GPU is needed to see the refusals
    torch = pytest.importorskip("torch")
    d = torch.float64
    n, nq = 10, 7
    ok = dict(Y=torch.zeros(n, dtype=d), Z=torch.zeros(n, dtype=d), w=torch.zeros(4, n, dtype=d),
              qy=torch.zeros(nq, dtype=d), qz=torch.zeros(nq, dtype=d), F=torch.zeros(4, nq, 2, dtype=d))
    bad = [("Y", torch.zeros(n, dtype=torch.float32), "float64"),
           ("w", torch.zeros(1, n, dtype=d), "[4][n_cells]"),
           ("Z", torch.zeros(n + 1, dtype=d), "Z has"),
           ("qz", torch.zeros(nq - 1, dtype=d), "qz has"),
           ("F", torch.zeros(4, nq, 1, dtype=d), "[4][n_q][2]"),
           ("F", torch.zeros(4, 2, nq, dtype=d).transpose(1, 2), "contiguous"),
           ("qy", np.zeros(nq), "torch tensor")]
    for name, val, msg in bad:
        kw = dict(ok)
        kw[name] = val
        with pytest.raises(ValueError, match=re.escape(msg)):
            nms.nms_dsft_direct_noalloc(**kw)
    with pytest.raises(ValueError, match="CUDA tensor"):
        nms.nms_dsft_direct_noalloc(**ok)
