"""The C-ABI library builds, loads and exports every entry point that include/unocg.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "unocg.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(unocg_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2508_02681_gb300 import _lib, build
    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.LIB_PATH


def test_header_declares_the_solver_calls():
    names = declared_symbols()
    for required in ["unocg_create", "unocg_set_microstructure", "unocg_set_phase_properties",
                     "unocg_set_macro_load", "unocg_set_uno_weights", "unocg_solve",
                     "unocg_get_fluctuation", "unocg_get_effective_tensor", "unocg_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (unocg_[A-Za-z_0-9]+)\b", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(libpath)
    for s in declared_symbols():
        getattr(lib, s)


def test_binding_signatures_cover_header(libpath):
    from paper_2508_02681_gb300 import _lib
    assert set(_lib.SIGNATURES) == set(declared_symbols())
    _lib.load(libpath)


def test_create_rejects_bad_grids(libpath):
    # argument validation happens before any device call
    from paper_2508_02681_gb300 import _lib
    lib = _lib.load(libpath)
    h = ctypes.c_void_p()
    assert lib.unocg_create(ctypes.byref(h), 1, 1, 7, 8, 8, 1.0) == _lib.ERR_INVALID_ARG
    assert lib.unocg_create(ctypes.byref(h), 1, 1, 8, 8, 9, 1.0) == _lib.ERR_INVALID_ARG
    assert lib.unocg_create(ctypes.byref(h), 2, 1, 8, 8, 8, 1.0) == _lib.ERR_INVALID_ARG
    assert lib.unocg_create(ctypes.byref(h), 1, 0, 8, 8, 8, 1.0) == _lib.ERR_INVALID_ARG


def test_device_pointer_bindings_check_their_tensors():
    """The device-pointer entry points refuse tensors the library would read or write out of
    bounds (host memory, another dtype, a strided view, another size), before any library call."""
    import torch
    from paper_2508_02681_gb300 import api
    ctx = ctypes.c_void_p(12345)
    api._FIELD_VALUES[ctx.value] = 8
    try:
        for bad in (torch.zeros(8, dtype=torch.float64),):  # host tensor
            with pytest.raises(ValueError, match="CUDA"):
                api._device_field(ctx, bad, "r_dev")
    finally:
        api._FIELD_VALUES.pop(ctx.value, None)
