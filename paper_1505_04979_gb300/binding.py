"""Thin ctypes binding of the C ABI in include/polarbp.h.

Argument marshalling only: tensors are passed as ``data_ptr()`` together with
torch's current CUDA stream; every step of decoding runs in the CUDA library.
There is no CPU fallback: if ``libpolarbp.so`` is missing or fails to load, the
calls raise.  The environment variable POLARBP_LIBRARY, when set, names another
build of the library to load instead (the checked build, libpolarbp_checked.so).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("POLARBP_LIBRARY") or os.path.join(_HERE, "libpolarbp.so")

POLARBP_OK = 0
POLARBP_ERR_ARG = 1
POLARBP_ERR_NONFINITE = 2
POLARBP_ERR_CUDA = 3
POLARBP_ERR_TIMEOUT = 4
POLARBP_ERR_NOMEM = 5
POLARBP_ERR_UNSUPPORTED = 6
POLARBP_ERR_CHECK = 7
POLARBP_STOP_NONE = 0
POLARBP_STOP_GMATRIX = 1
POLARBP_FREEZE_OFF = 0
POLARBP_FREEZE_CSFG = 1
POLARBP_FREEZE_CSFG_MULTI = 2
POLARBP_MAP_PIPELINED = 0
POLARBP_MAP_BLOCK = 1

_lock = threading.Lock()
_lib = None


class PolarBPError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


_VP = ctypes.c_void_p
_SIGS = {
    "polarbp_construct": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _VP, ctypes.c_double, ctypes.POINTER(_VP)]),
    "polarbp_frozen_set": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, _VP]),
    "polarbp_destroy": (None, [_VP]),
    "polarbp_code_info": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
    "polarbp_get_frozen_mask": (ctypes.c_int, [_VP, _VP]),
    "polarbp_set_bit_reversed": (ctypes.c_int, [_VP, ctypes.c_int]),
    "polarbp_get_bit_reversed": (ctypes.c_int, [_VP, _VP]),
    "polarbp_encode": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int, _VP]),
    "polarbp_decode": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                      ctypes.c_int, _VP, _VP, _VP, _VP]),
    "polarbp_decode_trace": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                            ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
    "polarbp_decode_flooding": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                               _VP, _VP, _VP, _VP, _VP, _VP]),
    "polarbp_decode_quantized": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, _VP, _VP, _VP, _VP, _VP, _VP]),
    "polarbp_decode_host_workspace": (ctypes.c_size_t, [_VP, ctypes.c_int]),
    "polarbp_decode_host": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                           ctypes.c_int, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP]),
    "polarbp_decode_host_noalloc": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                                   ctypes.c_int, _VP, _VP, _VP, _VP]),
    "polarbp_awgn": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, ctypes.c_float, _VP, _VP,
                                    _VP]),
    "polarbp_awgn_ebn0": (ctypes.c_int, [_VP, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _VP, _VP, _VP, _VP]),
    "polarbp_decode_segments_workspace": (ctypes.c_size_t, []),
    "polarbp_decode_segments": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                               ctypes.c_int, _VP, ctypes.c_size_t, _VP]),
    "polarbp_decode_mixed": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_float, ctypes.c_int,
                                            ctypes.c_int, _VP, ctypes.c_size_t, _VP]),
    "polarbp_set_codewords_per_block": (ctypes.c_int, [_VP, ctypes.c_int]),
    "polarbp_get_codewords_per_block": (ctypes.c_int, [_VP, _VP]),
    "polarbp_set_thread_mapping": (ctypes.c_int, [_VP, ctypes.c_int]),
    "polarbp_get_thread_mapping": (ctypes.c_int, [_VP, _VP]),
    "polarbp_autotune": (ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_float, ctypes.c_int, ctypes.c_int, _VP]),
    "polarbp_wms_workspace": (ctypes.c_size_t, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "polarbp_wms_forward": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP,
                                           ctypes.c_size_t, _VP]),
    "polarbp_wms_backward": (ctypes.c_int, [_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, _VP, _VP, _VP,
                                            _VP, ctypes.c_size_t, _VP]),
    "polarbp_get_status": (ctypes.c_int, [_VP, _VP]),
    "polarbp_last_error": (ctypes.c_char_p, []),
    "polarbp_version": (ctypes.c_char_p, []),
}


def lib():
    """Load libpolarbp.so (built in-tree by ``paper_1505_04979_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(f"{LIB_PATH} is missing: run paper_1505_04979_gb300.build.build() first")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
        return _lib


def _check(rc: int, where: str) -> None:
    if rc != POLARBP_OK:
        raise PolarBPError(rc, where, lib().polarbp_last_error().decode())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _need(t, dtype, shape, name):
    if t.dtype != dtype or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of shape {tuple(shape)}")


def polarbp_version() -> str:
    return lib().polarbp_version().decode()


def polarbp_frozen_set(N: int, K: int, z0: float = 0.5) -> np.ndarray:
    out = np.zeros(N, np.uint8)
    _check(lib().polarbp_frozen_set(N, K, z0, out.ctypes.data_as(ctypes.c_void_p)), "polarbp_frozen_set")
    return out


class PolarCode:
    """Owning wrapper of a polarbp_code handle."""

    def __init__(self, N: int, K: int, frozen_mask=None, z0: float = 0.5):
        h = ctypes.c_void_p()
        mask = None
        if frozen_mask is not None:
            mask = np.ascontiguousarray(frozen_mask, dtype=np.uint8)
        _check(lib().polarbp_construct(N, K, None if mask is None else mask.ctypes.data_as(ctypes.c_void_p), z0,
                                       ctypes.byref(h)), "polarbp_construct")
        self.handle = h
        self.N, self.K = N, K
        self.m = N.bit_length() - 1

    def set_bit_reversed(self, on: bool) -> None:
        """Codeword positions in bit-reversed channel order (polarbp_set_bit_reversed)."""
        _check(lib().polarbp_set_bit_reversed(self.handle, 1 if on else 0), "polarbp_set_bit_reversed")

    def bit_reversed(self) -> bool:
        v = ctypes.c_int()
        _check(lib().polarbp_get_bit_reversed(self.handle, ctypes.byref(v)), "polarbp_get_bit_reversed")
        return bool(v.value)

    def frozen_mask(self) -> np.ndarray:
        out = np.zeros(self.N, np.uint8)
        _check(lib().polarbp_get_frozen_mask(self.handle, out.ctypes.data_as(ctypes.c_void_p)), "get_frozen_mask")
        return out

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            lib().polarbp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def polarbp_construct(N: int, K: int, frozen_mask=None, z0: float = 0.5) -> PolarCode:
    return PolarCode(N, K, frozen_mask, z0)


def polarbp_encode(code: PolarCode, u, x=None, stream=None):
    import torch
    B = u.shape[0]
    _need(u, torch.uint8, (B, code.N), "u")
    if x is None:
        x = torch.empty_like(u)
    _need(x, torch.uint8, (B, code.N), "x")
    _check(lib().polarbp_encode(code.handle, _ptr(u), _ptr(x), B, _stream(stream)), "polarbp_encode")
    return x


def polarbp_awgn(code: PolarCode, seed: int, first_codeword: int, batch: int, ebn0_db: float, u=None, llr=None,
                 with_u: bool = True, stream=None):
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    if llr is None:
        llr = torch.empty((batch, code.N), dtype=torch.float32, device=dev)
    if with_u and u is None:
        u = torch.empty((batch, code.N), dtype=torch.uint8, device=dev)
    _need(llr, torch.float32, (batch, code.N), "llr")
    if u is not None:
        _need(u, torch.uint8, (batch, code.N), "u")
    _check(lib().polarbp_awgn(code.handle, seed, first_codeword, batch, ebn0_db, _ptr(u), _ptr(llr),
                              _stream(stream)), "polarbp_awgn")
    return u, llr


def polarbp_awgn_ebn0(code: PolarCode, seed: int, first_codeword: int, ebn0_db, u=None, llr=None,
                      with_u: bool = True, stream=None):
    """Device channel input with one Eb/N0 per codeword (``ebn0_db``: CUDA float32 [batch])."""
    import torch
    batch = ebn0_db.shape[0]
    _need(ebn0_db, torch.float32, (batch,), "ebn0_db")
    dev = ebn0_db.device
    if llr is None:
        llr = torch.empty((batch, code.N), dtype=torch.float32, device=dev)
    if with_u and u is None:
        u = torch.empty((batch, code.N), dtype=torch.uint8, device=dev)
    _need(llr, torch.float32, (batch, code.N), "llr")
    if u is not None:
        _need(u, torch.uint8, (batch, code.N), "u")
    _check(lib().polarbp_awgn_ebn0(code.handle, seed, first_codeword, batch, _ptr(ebn0_db), _ptr(u), _ptr(llr),
                                   _stream(stream)), "polarbp_awgn_ebn0")
    return u, llr


class _Segment(ctypes.Structure):
    _fields_ = [("code", ctypes.c_void_p), ("llr", ctypes.c_void_p), ("u_hat", ctypes.c_void_p),
                ("iterations", ctypes.c_void_p), ("pe_updates", ctypes.c_void_p), ("count", ctypes.c_int)]


def polarbp_decode_segments_workspace() -> int:
    return int(lib().polarbp_decode_segments_workspace())


def _segment_array(segments):
    import torch
    arr = (_Segment * max(1, len(segments)))()
    for k, (code, llr, u_hat, it, pe) in enumerate(segments):
        n = llr.shape[0]
        _need(llr, torch.float32, (n, code.N), "llr")
        _need(u_hat, torch.uint8, (n, code.N), "u_hat")
        if it is not None:
            _need(it, torch.int32, (n,), "iterations")
        if pe is not None:
            _need(pe, torch.int64, (n,), "pe_updates")
        arr[k] = _Segment(code.handle.value, llr.data_ptr(), u_hat.data_ptr(), None if it is None else it.data_ptr(),
                          None if pe is None else pe.data_ptr(), n)
    return arr


def polarbp_decode_segments(segments, max_iter: int, scale: float = 0.9375, stop_mode: int = 0,
                            freeze_mode: int = 0, workspace=None, stream=None):
    """Decode runs of codewords [(code, llr, u_hat, iterations, pe_updates), ...] with one
    persistent launch per code length.  ``workspace``: CUDA uint8 tensor (allocated if None)."""
    import torch
    arr = _segment_array(segments)
    if workspace is None:
        workspace = torch.empty(polarbp_decode_segments_workspace(), dtype=torch.uint8, device="cuda")
    _check(lib().polarbp_decode_segments(ctypes.cast(arr, ctypes.c_void_p), len(segments), max_iter, scale,
                                         stop_mode, freeze_mode, _ptr(workspace), workspace.numel(),
                                         _stream(stream)), "polarbp_decode_segments")
    return workspace


def polarbp_decode_mixed(segments, max_iter: int, scale: float = 0.9375, stop_mode: int = 0,
                         freeze_mode: int = 0, workspace=None, stream=None):
    """Decode runs of codewords [(code, llr, u_hat, iterations, pe_updates), ...] of mixed
    lengths with ONE persistent launch.  ``workspace``: CUDA uint8 tensor (allocated if None)."""
    import torch
    arr = _segment_array(segments)
    if workspace is None:
        workspace = torch.empty(polarbp_decode_segments_workspace(), dtype=torch.uint8, device="cuda")
    _check(lib().polarbp_decode_mixed(ctypes.cast(arr, ctypes.c_void_p), len(segments), max_iter, scale,
                                      stop_mode, freeze_mode, _ptr(workspace), workspace.numel(),
                                      _stream(stream)), "polarbp_decode_mixed")
    return workspace


def polarbp_set_codewords_per_block(code: PolarCode, cpc: int) -> None:
    _check(lib().polarbp_set_codewords_per_block(code.handle, cpc), "polarbp_set_codewords_per_block")


def polarbp_get_codewords_per_block(code: PolarCode) -> int:
    v = ctypes.c_int()
    _check(lib().polarbp_get_codewords_per_block(code.handle, ctypes.byref(v)), "polarbp_get_codewords_per_block")
    return v.value


def polarbp_set_thread_mapping(code: PolarCode, mapping: int) -> None:
    _check(lib().polarbp_set_thread_mapping(code.handle, mapping), "polarbp_set_thread_mapping")


def polarbp_get_thread_mapping(code: PolarCode) -> int:
    v = ctypes.c_int()
    _check(lib().polarbp_get_thread_mapping(code.handle, ctypes.byref(v)), "polarbp_get_thread_mapping")
    return v.value


def polarbp_autotune(code: PolarCode, max_iter: int, scale: float = 0.9375, stop_mode: int = 1,
                     freeze_mode: int = 1, stream=None) -> int:
    """Time every admissible (thread mapping, codewords per block) pair and keep the fastest
    in the handle; returns the codewords per block (polarbp_get_thread_mapping gives the
    mapping)."""
    _check(lib().polarbp_autotune(code.handle, max_iter, scale, stop_mode, freeze_mode, _stream(stream)),
           "polarbp_autotune")
    return polarbp_get_codewords_per_block(code)


def polarbp_decode(code: PolarCode, llr, max_iter: int, scale: float = 0.9375, stop_mode: int = 0,
                   freeze_mode: int = 0, u_hat=None, iterations=None, pe_updates=None, stream=None):
    import torch
    B = llr.shape[0]
    _need(llr, torch.float32, (B, code.N), "llr")
    if u_hat is None:
        u_hat = torch.empty((B, code.N), dtype=torch.uint8, device=llr.device)
    if iterations is None:
        iterations = torch.empty(B, dtype=torch.int32, device=llr.device)
    if pe_updates is None:
        pe_updates = torch.empty(B, dtype=torch.int64, device=llr.device)
    _need(u_hat, torch.uint8, (B, code.N), "u_hat")
    _need(iterations, torch.int32, (B,), "iterations")
    _need(pe_updates, torch.int64, (B,), "pe_updates")
    _check(lib().polarbp_decode(code.handle, _ptr(llr), B, max_iter, scale, stop_mode, freeze_mode, _ptr(u_hat),
                                _ptr(iterations), _ptr(pe_updates), _stream(stream)), "polarbp_decode")
    return u_hat, iterations, pe_updates


def polarbp_decode_trace(code: PolarCode, llr, max_iter: int, scale: float = 0.9375, stop_mode: int = 0,
                         freeze_mode: int = 0, stream=None):
    """Decode and return (u_hat, iterations, pe_updates, trace_L, trace_R, trace_P)."""
    import torch
    B = llr.shape[0]
    _need(llr, torch.float32, (B, code.N), "llr")
    dev = llr.device
    u_hat = torch.empty((B, code.N), dtype=torch.uint8, device=dev)
    iterations = torch.empty(B, dtype=torch.int32, device=dev)
    pe_updates = torch.empty(B, dtype=torch.int64, device=dev)
    shape = (B, max_iter, code.m + 1, code.N)
    tL = torch.full(shape, float("nan"), dtype=torch.float32, device=dev)
    tR = torch.full(shape, float("nan"), dtype=torch.float32, device=dev)
    tP = torch.full((B, max_iter), -1, dtype=torch.int32, device=dev)
    _check(lib().polarbp_decode_trace(code.handle, _ptr(llr), B, max_iter, scale, stop_mode, freeze_mode, _ptr(u_hat),
                                      _ptr(iterations), _ptr(pe_updates), _ptr(tL), _ptr(tR), _ptr(tP),
                                      _stream(stream)), "polarbp_decode_trace")
    return u_hat, iterations, pe_updates, tL, tR, tP


def polarbp_decode_flooding(code: PolarCode, llr, max_iter: int, scale: float = 0.9375, stop_mode: int = 0,
                            u_hat=None, iterations=None, pe_updates=None, trace: bool = False, stream=None):
    """Flooding-schedule decode; returns (u_hat, iterations, pe_updates) or, with ``trace``,
    (u_hat, iterations, pe_updates, trace_L, trace_R) with planes [batch, max_iter, m+1, N]."""
    import torch
    B = llr.shape[0]
    _need(llr, torch.float32, (B, code.N), "llr")
    if u_hat is None:
        u_hat = torch.empty((B, code.N), dtype=torch.uint8, device=llr.device)
    if iterations is None:
        iterations = torch.empty(B, dtype=torch.int32, device=llr.device)
    if pe_updates is None:
        pe_updates = torch.empty(B, dtype=torch.int64, device=llr.device)
    _need(u_hat, torch.uint8, (B, code.N), "u_hat")
    _need(iterations, torch.int32, (B,), "iterations")
    _need(pe_updates, torch.int64, (B,), "pe_updates")
    tl = tr = None
    if trace:
        m = code.N.bit_length() - 1
        tl = torch.full((B, max_iter, m + 1, code.N), float("nan"), dtype=torch.float32, device=llr.device)
        tr = torch.full_like(tl, float("nan"))
    _check(lib().polarbp_decode_flooding(code.handle, _ptr(llr), B, max_iter, scale, stop_mode, _ptr(u_hat),
                                         _ptr(iterations), _ptr(pe_updates), _ptr(tl), _ptr(tr), _stream(stream)),
           "polarbp_decode_flooding")
    return (u_hat, iterations, pe_updates, tl, tr) if trace else (u_hat, iterations, pe_updates)


def polarbp_decode_quantized(code: PolarCode, llr, max_iter: int, alpha_16: int = 15, frac_bits: int = 3,
                             stop_mode: int = 0, u_hat=None, iterations=None, pe_updates=None, trace: bool = False,
                             stream=None):
    """Quantised-message decode; returns (u_hat, iterations, pe_updates) or, with ``trace``,
    (u_hat, iterations, pe_updates, trace_L, trace_R) with int16 planes [batch, max_iter, m+1, N]."""
    import torch
    B = llr.shape[0]
    _need(llr, torch.float32, (B, code.N), "llr")
    if u_hat is None:
        u_hat = torch.empty((B, code.N), dtype=torch.uint8, device=llr.device)
    if iterations is None:
        iterations = torch.empty(B, dtype=torch.int32, device=llr.device)
    if pe_updates is None:
        pe_updates = torch.empty(B, dtype=torch.int64, device=llr.device)
    _need(u_hat, torch.uint8, (B, code.N), "u_hat")
    _need(iterations, torch.int32, (B,), "iterations")
    _need(pe_updates, torch.int64, (B,), "pe_updates")
    tl = tr = None
    if trace:
        m = code.N.bit_length() - 1
        tl = torch.zeros((B, max_iter, m + 1, code.N), dtype=torch.int16, device=llr.device)
        tr = torch.zeros_like(tl)
    _check(lib().polarbp_decode_quantized(code.handle, _ptr(llr), B, max_iter, alpha_16, frac_bits, stop_mode,
                                          _ptr(u_hat), _ptr(iterations), _ptr(pe_updates), _ptr(tl), _ptr(tr),
                                          _stream(stream)), "polarbp_decode_quantized")
    return (u_hat, iterations, pe_updates, tl, tr) if trace else (u_hat, iterations, pe_updates)


def polarbp_decode_host_workspace(code: PolarCode, batch: int) -> int:
    return int(lib().polarbp_decode_host_workspace(code.handle, batch))


def polarbp_decode_host(code: PolarCode, llr_host, max_iter: int, scale: float, stop_mode: int, freeze_mode: int,
                        u_hat_host, iterations_host, pe_host, workspace, stream=None) -> None:
    """Host buffers in and out (CPU tensors, pinned for overlap); ``workspace`` is a CUDA uint8 tensor."""
    B = llr_host.shape[0]
    for t, name in ((llr_host, "llr"), (u_hat_host, "u_hat")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous host tensor")
    _check(lib().polarbp_decode_host(code.handle, _ptr(llr_host), B, max_iter, scale, stop_mode, freeze_mode,
                                     _ptr(u_hat_host), _ptr(iterations_host), _ptr(pe_host), _ptr(workspace),
                                     workspace.numel(), _stream(stream)), "polarbp_decode_host")


def polarbp_decode_host_noalloc(code: PolarCode, llr_host, max_iter: int, scale: float, stop_mode: int,
                                freeze_mode: int, u_hat_host, iterations_host, pe_host, stream=None) -> None:
    """polarbp_decode_host staging through the library's built-in device array (no allocation)."""
    B = llr_host.shape[0]
    for t, name in ((llr_host, "llr"), (u_hat_host, "u_hat")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous host tensor")
    _check(lib().polarbp_decode_host_noalloc(code.handle, _ptr(llr_host), B, max_iter, scale, stop_mode, freeze_mode,
                                             _ptr(u_hat_host), _ptr(iterations_host), _ptr(pe_host),
                                             _stream(stream)), "polarbp_decode_host_noalloc")


def polarbp_get_status(code: PolarCode, stream=None) -> int:
    """POLARBP_OK, or POLARBP_ERR_NONFINITE when a decode saw a non-finite LLR (clears the flag).
    A redzone store seen by the checked build raises PolarBPError with code POLARBP_ERR_CHECK."""
    rc = lib().polarbp_get_status(code.handle, _stream(stream))
    if rc not in (POLARBP_OK, POLARBP_ERR_NONFINITE):
        _check(rc, "polarbp_get_status")
    return rc


def polarbp_wms_workspace(code: PolarCode, batch: int, iterations: int, checkpoint_every: int = 1) -> int:
    return int(lib().polarbp_wms_workspace(code.handle, batch, iterations, checkpoint_every))


def polarbp_wms_forward(code: PolarCode, llr, weights, workspace, out=None, stream=None, checkpoint_every: int = 1):
    import torch
    B = llr.shape[0]
    T = weights.shape[0]
    _need(llr, torch.float32, (B, code.N), "llr")
    _need(weights, torch.float32, (T, code.m, code.N // 2), "weights")
    if out is None:
        out = torch.empty((B, code.N), dtype=torch.float32, device=llr.device)
    _check(lib().polarbp_wms_forward(code.handle, _ptr(llr), B, T, checkpoint_every, _ptr(weights), _ptr(out),
                                     _ptr(workspace), workspace.numel(), _stream(stream)), "polarbp_wms_forward")
    return out


def polarbp_wms_backward(code: PolarCode, llr, weights, dout, workspace, stream=None, checkpoint_every: int = 1):
    import torch
    B = llr.shape[0]
    T = weights.shape[0]
    dout = dout.contiguous()
    _need(dout, torch.float32, (B, code.N), "dout")
    dw = torch.empty_like(weights)
    dl = torch.empty_like(llr)
    _check(lib().polarbp_wms_backward(code.handle, _ptr(llr), B, T, checkpoint_every, _ptr(weights), _ptr(dout),
                                      _ptr(dw), _ptr(dl), _ptr(workspace), workspace.numel(), _stream(stream)),
           "polarbp_wms_backward")
    return dw, dl


def weighted_min_sum(code: PolarCode, llr, weights, checkpoint_every: int = 1):
    """Differentiable weighted min-sum decoder: soft outputs [batch, N] as a function of
    (llr, weights); gradients come from the library's adjoint kernel.  ``checkpoint_every``:
    the forward keeps the message state of every k-th iteration, the adjoint recomputes
    the rest (the gradients do not depend on k)."""
    import torch

    class _WMS(torch.autograd.Function):
        @staticmethod
        def forward(ctx, llr_t, w_t):
            llr_c = llr_t.detach().contiguous()
            w_c = w_t.detach().contiguous()
            ws = torch.empty(polarbp_wms_workspace(code, llr_c.shape[0], w_c.shape[0], checkpoint_every),
                             dtype=torch.uint8, device=llr_c.device)
            out = polarbp_wms_forward(code, llr_c, w_c, ws, checkpoint_every=checkpoint_every)
            ctx.save_for_backward(llr_c, w_c, ws)
            return out

        @staticmethod
        def backward(ctx, dout):
            llr_c, w_c, ws = ctx.saved_tensors
            dw, dl = polarbp_wms_backward(code, llr_c, w_c, dout.to(torch.float32), ws,
                                          checkpoint_every=checkpoint_every)
            return dl, dw

    return _WMS.apply(llr, weights)
