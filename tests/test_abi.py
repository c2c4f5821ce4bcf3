"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/rpnn.h declares (no compute calls: no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "rpnn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rpnn_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1709_05418_gb300 import build
    return build.build()


def test_header_declares_the_named_entry_points():
    names = declared()
    for must in ("rpnn_load_volume", "rpnn_build_mips", "rpnn_set_weights", "rpnn_render",
                 "rpnn_train_step"):
        assert must in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (rpnn_[a-z_0-9]+)\b", out))
    missing = [n for n in declared() if n not in exported]
    assert not missing, missing


def test_library_loads_and_resolves(libpath):
    import torch  # noqa: F401  (shares the CUDA runtime with the library)
    L = ctypes.CDLL(libpath)
    for n in declared():
        assert getattr(L, n)
    L.rpnn_last_error.restype = ctypes.c_char_p
    assert isinstance(L.rpnn_last_error(), bytes)   # other tests may have left a message
    # argument checks that need no device
    L.rpnn_create.argtypes = [ctypes.c_void_p]
    assert L.rpnn_create(None) == -1


def test_argument_checks_without_a_device(libpath):
    """Entry points reject a null context before touching the device."""
    import torch  # noqa: F401
    L = ctypes.CDLL(libpath)
    L.rpnn_set_train_precision.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    L.rpnn_set_autotune.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    L.rpnn_get_autotune.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    L.rpnn_render_env.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                  ctypes.c_void_p]
    for rc in (L.rpnn_set_train_precision(None, 2), L.rpnn_set_autotune(None, 1),
               L.rpnn_get_autotune(None, None, 0, None),
               L.rpnn_render_env(None, 0, None, None, None, 1, None, None, None)):
        assert rc == -2    # RPNN_ERR_HANDLE


def test_phase_and_stencil_entry_points_check_arguments_without_a_device(libpath):
    """The Lorenz-Mie option and the stencil-size entry points reject a null context, and
    the stencil widths and parameter counts follow their definitions (host-only calls)."""
    import torch  # noqa: F401
    L = ctypes.CDLL(libpath)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.rpnn_set_phase_function.argtypes = [vp, i32, i32]
    L.rpnn_stencil_param_count.argtypes = [i32]
    L.rpnn_stencil_param_count.restype = i64
    L.rpnn_stencil_descriptors.argtypes = [vp, i32, i32, vp, vp, vp, i32, i64, vp, vp]
    L.rpnn_stencil_forward.argtypes = [vp, i32, vp, vp, i64, vp, vp]
    L.rpnn_stencil_backward.argtypes = [vp, i32, vp, vp, i64, vp, vp, vp]
    L.rpnn_stencil_train_step.argtypes = [vp, i32, vp, vp, i32, vp, i64, vp, vp, vp, vp, vp]
    for rc in (L.rpnn_set_phase_function(None, 0, 1),
               L.rpnn_stencil_descriptors(None, 0, 3, None, None, None, 0, 1, None, None),
               L.rpnn_stencil_forward(None, 3, None, None, 1, None, None),
               L.rpnn_stencil_backward(None, 3, None, None, 1, None, None, None),
               L.rpnn_stencil_train_step(None, 3, None, None, 1, None, 1, None, None, None, None, None)):
        assert rc == -2    # RPNN_ERR_HANDLE
    for n in range(2, 10):
        din = n * n * (2 * n - 1) + 1
        expect = 10 * (200 * din + 200 + 200 * 200 + 200) + 9 * 200 * 200 + 2 * (200 * 200 + 200) + 201
        assert L.rpnn_stencil_param_count(n) == expect
    assert L.rpnn_stencil_param_count(5) == 1296601
    assert L.rpnn_stencil_param_count(1) == -1 and L.rpnn_stencil_param_count(10) == -1
