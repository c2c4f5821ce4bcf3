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
