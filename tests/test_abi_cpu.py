"""Host-side checks that need no GPU: the library loads and exports every entry
point the header declares, host-only logic matches the oracle, and arguments
are rejected before any CUDA call."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04979_gb300 import binding as B
from paper_1505_04979_gb300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "polarbp.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return B.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(polarbp_\w+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("polarbp_construct", "polarbp_destroy", "polarbp_encode", "polarbp_decode",
                     "polarbp_get_frozen_mask", "polarbp_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)


def test_library_is_built_for_sm_103a(lib):
    assert "sm_103a" in B.polarbp_version()


@pytest.mark.parametrize("N,K", [(2, 1), (8, 4), (64, 32), (128, 64), (256, 64), (256, 128), (256, 192),
                                 (1024, 256), (1024, 512), (1024, 768), (4096, 1024), (4096, 2048),
                                 (4096, 3072), (8192, 4096), (16384, 8192), (32768, 16384), (16, 0), (16, 16),
                                 (64, 1), (1024, 1023), (8192, 0), (8192, 1), (8192, 8191), (8192, 8192)])
def test_frozen_set_matches_oracle(lib, N, K):
    """Sec. II construction: the library's host recursion and the oracle agree exactly."""
    assert np.array_equal(B.polarbp_frozen_set(N, K, 0.5), O.bec_frozen(N, K, 0.5))


@pytest.mark.parametrize("args", [(3, 1, 0.5), (0, 0, 0.5), (65536, 10, 0.5), (8, 9, 0.5), (8, -1, 0.5),
                                  (8, 4, 0.0), (8, 4, 1.0)])
def test_frozen_set_rejects_bad_arguments(lib, args):
    out = np.zeros(max(args[0], 1), np.uint8)
    rc = lib.polarbp_frozen_set(args[0], args[1], args[2], out.ctypes.data_as(ctypes.c_void_p))
    assert rc == B.POLARBP_ERR_ARG
    assert lib.polarbp_last_error().decode()


def test_construct_rejects_bad_arguments_before_touching_cuda(lib):
    h = ctypes.c_void_p()
    assert lib.polarbp_construct(12, 4, None, 0.5, ctypes.byref(h)) == B.POLARBP_ERR_ARG
    assert lib.polarbp_construct(16, 17, None, 0.5, ctypes.byref(h)) == B.POLARBP_ERR_ARG
    assert lib.polarbp_construct(16, 8, None, 1.5, ctypes.byref(h)) == B.POLARBP_ERR_ARG
    bad = np.ones(16, np.uint8)  # popcount 16 != N - K
    assert lib.polarbp_construct(16, 8, bad.ctypes.data_as(ctypes.c_void_p), 0.5, ctypes.byref(h)) == B.POLARBP_ERR_ARG
    two = np.full(16, 2, np.uint8)
    assert lib.polarbp_construct(16, 0, two.ctypes.data_as(ctypes.c_void_p), 0.5, ctypes.byref(h)) == B.POLARBP_ERR_ARG
    assert lib.polarbp_construct(16, 8, None, 0.5, None) == B.POLARBP_ERR_ARG
    assert not h.value


def test_calls_on_a_null_handle_fail_cleanly(lib):
    assert lib.polarbp_decode(None, None, 1, 1, 1.0, 0, 0, None, None, None, None) == B.POLARBP_ERR_ARG
    assert lib.polarbp_encode(None, None, None, 1, None) == B.POLARBP_ERR_ARG
    assert lib.polarbp_code_info(None, None, None, None) == B.POLARBP_ERR_ARG
    assert lib.polarbp_get_status(None, None) == B.POLARBP_ERR_ARG
    lib.polarbp_destroy(None)


@pytest.mark.parametrize("name", ["polarbp_decode_segments", "polarbp_decode_mixed"])
def test_mixed_stream_entry_points_reject_bad_arguments_before_touching_cuda(lib, name):
    f = getattr(lib, name)
    ws = ctypes.c_void_p(16)  # never dereferenced: every call below fails its argument checks first
    assert f(None, -1, 10, ctypes.c_float(0.9), 1, 1, ws, ctypes.c_size_t(256), None) == B.POLARBP_ERR_ARG
    assert f(None, 1, 10, ctypes.c_float(0.9), 1, 1, ws, ctypes.c_size_t(256), None) == B.POLARBP_ERR_ARG
    assert f(None, 0, 0, ctypes.c_float(0.9), 1, 1, ws, ctypes.c_size_t(256), None) == B.POLARBP_ERR_ARG
    assert f(None, 0, 10, ctypes.c_float(0.0), 1, 1, ws, ctypes.c_size_t(256), None) == B.POLARBP_ERR_ARG
    assert f(None, 0, 10, ctypes.c_float(float("nan")), 1, 1, ws, ctypes.c_size_t(256), None) == B.POLARBP_ERR_ARG
    assert f(None, 0, 10, ctypes.c_float(0.9), 2, 1, ws, ctypes.c_size_t(256), None) == B.POLARBP_ERR_ARG
    assert f(None, 0, 10, ctypes.c_float(0.9), 1, 3, ws, ctypes.c_size_t(256), None) == B.POLARBP_ERR_ARG
    assert f(None, 0, 10, ctypes.c_float(0.9), 1, 1, None, ctypes.c_size_t(256), None) == B.POLARBP_ERR_ARG
    assert f(None, 0, 10, ctypes.c_float(0.9), 1, 1, ws, ctypes.c_size_t(4), None) == B.POLARBP_ERR_ARG
    assert lib.polarbp_last_error().decode()


def test_thread_mapping_calls_reject_bad_arguments(lib):
    v = ctypes.c_int()
    assert lib.polarbp_set_thread_mapping(None, B.POLARBP_MAP_BLOCK) == B.POLARBP_ERR_ARG
    assert lib.polarbp_get_thread_mapping(None, ctypes.byref(v)) == B.POLARBP_ERR_ARG
