"""The C ABI boundary, host side only (no GPU needed).

* liblsas.so builds, loads and exports every function include/lsas.h declares.
* The host-only entry points validate configurations and report frame sizes
  as documented, and a plan cannot be created without a GPU (LSAS_ERR_CUDA,
  not a crash).
"""

import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1901_07499_gb300.build import build
    build()
    import paper_1901_07499_gb300.lsas as lsas
    return lsas


def declared_functions():
    with open(os.path.join(ROOT, "include", "lsas.h")) as fh:
        text = fh.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lsas_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_function(L):
    names = declared_functions()
    assert "lsas_run_frame" in names and len(names) >= 14
    lib = C.CDLL(L.LIB)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(L.EXPORTED) == names


def test_status_strings(L):
    for code in range(8):
        assert L.lsas_status_str(code).startswith(b"LSAS_")
    assert L.lsas_status_str(99) == b"LSAS_ERR_UNKNOWN"


@pytest.mark.parametrize("args,ok", [
    ((64, 1024, 128, 14, 0, 16), True),
    ((1, 64, 0, 2, 1, 2), True),
    ((256, 2048, 2047, 64, 63, 256), True),
    ((0, 1024, 128, 14, 0, 16), False),
    ((257, 1024, 128, 14, 0, 16), False),
    ((64, 1000, 128, 14, 0, 16), False),
    ((64, 32, 8, 14, 0, 16), False),
    ((64, 4096, 128, 14, 0, 16), False),
    ((64, 1024, 1024, 14, 0, 16), False),
    ((64, 1024, -1, 14, 0, 16), False),
    ((64, 1024, 128, 1, 0, 16), False),
    ((64, 1024, 128, 65, 0, 16), False),
    ((64, 1024, 128, 14, 14, 16), False),
    ((64, 1024, 128, 14, -1, 16), False),
    ((64, 1024, 128, 14, 0, 8), False),
    ((64, 1024, 128, 14, 0, 32), False),
])
def test_check_config(L, args, ok):
    assert (L.lsas_check_config(*args) == L.LSAS_OK) == ok


def test_frame_bytes(L):
    # 64 antennas, N=1024, CP=128, 14 symbols, 16-QAM, sc16
    assert L.frame_bytes(64, 1024, 128, 14, 16, "sc16") == (4128768, 524288, 6656, 106496)
    assert L.frame_bytes(8, 64, 16, 15, 4, "fc32") == (76800, 4096, 224, 7168)
    out = (C.c_size_t * 4)()
    assert L.lsas_frame_bytes(8, 64, 16, 15, 4, 5, out) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_frame_bytes(8, 64, 16, 15, 4, 0, None) == L.LSAS_ERR_INVALID_ARG


def test_null_plan_is_rejected(L):
    assert L.lsas_run_frame(None, None, 1, None, None, None, None) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_plan_sync(None, None) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_plan_destroy(None) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_plan_create(8, 64, 16, 4, 0, 4, None) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_plan_set_profile(None, 1) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_plan_profile(None, None, 0, None) == L.LSAS_ERR_INVALID_ARG


def test_plan_create_without_gpu_fails_cleanly(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    assert L.lsas_plan_create(8, 64, 16, 4, 0, 4, C.byref(h)) == L.LSAS_ERR_CUDA
    assert h.value is None
    # invalid arguments are rejected before CUDA is touched
    assert L.lsas_plan_create(8, 63, 16, 4, 0, 4, C.byref(h)) == L.LSAS_ERR_INVALID_ARG


def test_server_needs_a_gpu_and_valid_arguments(L):
    import torch
    h = C.c_void_p()
    assert L.lsas_server_create(1 << 30, 0, 10.0, C.byref(h)) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_server_create(1 << 30, 8, -1.0, C.byref(h)) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_server_wait(None, 1, 1.0, None) == L.LSAS_ERR_INVALID_ARG
    assert L.lsas_server_destroy(None) == L.LSAS_ERR_INVALID_ARG
    if not torch.cuda.is_available():
        assert L.lsas_server_create(1 << 30, 8, 10.0, C.byref(h)) == L.LSAS_ERR_CUDA
        assert h.value is None
