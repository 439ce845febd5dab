"""ctypes wrapper around the plain C oracle in ``polar_oracle.c``.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg are the only callers.  The product path never
imports this module, and this module imports nothing from the product package.

Paper: arXiv 1505.04979.  The C file cites the section / equation each
function follows (Sec. II code construction and encoder, Eq. (1) PE update,
Eqs. (2)-(4) CSFG check, Sec. IV computation count).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polar_oracle.c")
_LIB = os.path.join(_HERE, "libpolar_oracle.so")
_lock = threading.Lock()
_lib = None

STOP_NONE = 0
STOP_GMATRIX = 1
FREEZE_OFF = 0
FREEZE_CSFG = 1
FREEZE_CSFG_MULTI = 2  # reading B: checks continue along a level while they pass (a variant)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP over codewords, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        f32p = ctypes.POINTER(ctypes.c_float)
        f64p = ctypes.POINTER(ctypes.c_double)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        ci, cd = ctypes.c_int, ctypes.c_double
        lib.orc_bec_lnz.argtypes = [ci, cd, f64p, f64p]
        lib.orc_bec_frozen.argtypes = [ci, ci, cd, u8p]
        lib.orc_encode.argtypes = [ci, u8p, u8p]
        lib.orc_csfg_check_ext.argtypes = [ci, f64p, u8p, u8p, u8p]
        lib.orc_decode.argtypes = [ci, u8p, f32p, ci, cd, ci, ci, ci, u8p, i32p, i64p, f64p, i32p,
                                   f64p, f64p, i32p, i64p]
        lib.orc_decode_batch.argtypes = [ci, u8p, f32p, ci, ci, cd, ci, ci, ci, ci, u8p, i32p, i64p,
                                         f64p, i32p]
        lib.orc_decode_flood.argtypes = [ci, u8p, f32p, ci, cd, ci, ci, u8p, i32p, i64p, f64p, f64p, f64p]
        lib.orc_decode_flood_batch.argtypes = [ci, u8p, f32p, ci, ci, cd, ci, ci, ci, u8p, i32p, i64p, f64p]
        lib.orc_sc_decode.argtypes = [ci, u8p, f32p, ci, u8p]
        lib.orc_sc_decode_batch.argtypes = [ci, u8p, f32p, ci, ci, ci, u8p]
        lib.orc_decode_q.argtypes = [ci, u8p, f32p, ci, ci, ci, ci, u8p, i32p, i64p, i32p, i32p]
        lib.orc_decode_q_batch.argtypes = [ci, u8p, f32p, ci, ci, ci, ci, ci, ci, u8p, i32p, i64p]
        lib.orc_max_threads.argtypes = []
        lib.orc_decode_rule_batch.argtypes = [ci, u8p, f32p, ci, ci, cd, ci, ci, cd, ci, ci, u8p, i32p, i64p]
        lib.orc_wms_forward.argtypes = [ci, u8p, f32p, ci, f64p, ci, f64p, f64p, f64p]
        lib.orc_wms_backward.argtypes = [ci, u8p, f32p, ci, f64p, f64p, ci, f64p, f64p]
        for fn in ("orc_bec_lnz", "orc_bec_frozen", "orc_encode", "orc_csfg_check_ext", "orc_decode",
                   "orc_decode_batch", "orc_decode_flood", "orc_decode_flood_batch", "orc_sc_decode",
                   "orc_sc_decode_batch", "orc_decode_q", "orc_decode_q_batch", "orc_max_threads",
                   "orc_wms_forward", "orc_wms_backward", "orc_decode_rule_batch"):
            getattr(lib, fn).restype = ci
        _lib = lib
        return lib


def _p(arr, ctype):
    if arr is None:
        return None
    return arr.ctypes.data_as(ctypes.POINTER(ctype))


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def max_threads() -> int:
    return int(_load().orc_max_threads())


def bec_lnz(N: int, z0: float = 0.5):
    """(ln z, ln(1-z)) of the N synthetic channels of a BEC(z0) (Sec. II)."""
    a = np.zeros(N, np.float64)
    b = np.zeros(N, np.float64)
    _check(_load().orc_bec_lnz(N, z0, _p(a, ctypes.c_double), _p(b, ctypes.c_double)), "bec_lnz")
    return a, b


def bec_frozen(N: int, K: int, z0: float = 0.5) -> np.ndarray:
    """Frozen mask (1 = frozen) of the (N, K) code: the N-K largest z (Sec. II)."""
    out = np.zeros(N, np.uint8)
    _check(_load().orc_bec_frozen(N, K, z0, _p(out, ctypes.c_uint8)), "bec_frozen")
    return out


def encode(u: np.ndarray) -> np.ndarray:
    """x = u F^{(x)m} over GF(2) (Sec. II); u is [N] or [batch, N]."""
    u = np.ascontiguousarray(u, dtype=np.uint8)
    flat = u.reshape(-1, u.shape[-1])
    N = flat.shape[1]
    out = np.zeros_like(flat)
    lib = _load()
    for r in range(flat.shape[0]):
        row_in = np.ascontiguousarray(flat[r])
        row_out = np.zeros(N, np.uint8)
        _check(lib.orc_encode(N, _p(row_in, ctypes.c_uint8), _p(row_out, ctypes.c_uint8)), "encode")
        out[r] = row_out
    return out.reshape(u.shape)


def csfg_check(R: np.ndarray, frozen_sub: np.ndarray):
    """Eqs. (2)-(4) on one CSFG: returns (passes, x_hat, u_hat)."""
    R = np.ascontiguousarray(R, dtype=np.float64)
    fz = np.ascontiguousarray(frozen_sub, dtype=np.uint8)
    S = R.shape[0]
    xh = np.zeros(S, np.uint8)
    uh = np.zeros(S, np.uint8)
    rc = _load().orc_csfg_check_ext(S, _p(R, ctypes.c_double), _p(fz, ctypes.c_uint8),
                                     _p(xh, ctypes.c_uint8), _p(uh, ctypes.c_uint8))
    if rc < 0:
        _check(rc, "csfg_check")
    return bool(rc), xh, uh


def decode(frozen, llr, max_iter: int, alpha: float = 0.9375, stop: int = STOP_NONE,
           freeze: int = FREEZE_OFF, fp32: bool = False, trace: bool = False) -> dict:
    """Decode one codeword (Eq. (1) sweep, G-matrix stop, CSFG freezing).

    Returns a dict with u_hat, iters, pe, margin and, when ``trace`` is set,
    the per-iteration L / R planes ([iters, m+1, N]), covered-prefix lengths P
    and per-iteration PE counts.
    """
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    N = frozen.shape[0]
    m = N.bit_length() - 1
    u_hat = np.zeros(N, np.uint8)
    iters = np.zeros(1, np.int32)
    pe = np.zeros(1, np.int64)
    margin = np.zeros(1, np.float64)
    cover = np.zeros(1, np.int32)
    tl = tr = tp = tpe = None
    if trace:
        tl = np.full((max_iter, m + 1, N), np.nan, np.float64)
        tr = np.full((max_iter, m + 1, N), np.nan, np.float64)
        tp = np.full(max_iter, -1, np.int32)
        tpe = np.zeros(max_iter, np.int64)
    rc = _load().orc_decode(N, _p(frozen, ctypes.c_uint8), _p(llr, ctypes.c_float), max_iter, alpha, stop,
                            freeze, 1 if fp32 else 0, _p(u_hat, ctypes.c_uint8), _p(iters, ctypes.c_int32),
                            _p(pe, ctypes.c_int64), _p(margin, ctypes.c_double), _p(cover, ctypes.c_int32),
                            _p(tl, ctypes.c_double), _p(tr, ctypes.c_double), _p(tp, ctypes.c_int32),
                            _p(tpe, ctypes.c_int64))
    _check(rc, "decode")
    out = {"u_hat": u_hat, "iters": int(iters[0]), "pe": int(pe[0]), "margin": float(margin[0]),
           "cover": int(cover[0])}
    if trace:
        n = out["iters"]
        out.update(L=tl[:n], R=tr[:n], P=tp[:n], pe_iter=tpe[:n])
    return out


def decode_batch(frozen, llr, max_iter: int, alpha: float = 0.9375, stop: int = STOP_NONE,
                 freeze: int = FREEZE_OFF, fp32: bool = False, nthreads: int = 0, cover: bool = False):
    """Decode a [batch, N] LLR array; returns (u_hat, iters, pe, margin), plus the final
    covered-prefix lengths when ``cover`` is set."""
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    B, N = llr.shape
    u_hat = np.zeros((B, N), np.uint8)
    iters = np.zeros(B, np.int32)
    pe = np.zeros(B, np.int64)
    margin = np.zeros(B, np.float64)
    cv = np.zeros(B, np.int32) if cover else None
    rc = _load().orc_decode_batch(N, _p(frozen, ctypes.c_uint8), _p(llr, ctypes.c_float), B, max_iter, alpha,
                                  stop, freeze, 1 if fp32 else 0, nthreads, _p(u_hat, ctypes.c_uint8),
                                  _p(iters, ctypes.c_int32), _p(pe, ctypes.c_int64), _p(margin, ctypes.c_double),
                                  _p(cv, ctypes.c_int32))
    _check(rc, "decode_batch")
    return (u_hat, iters, pe, margin, cv) if cover else (u_hat, iters, pe, margin)


def decode_flood(frozen, llr, max_iter: int, alpha: float = 0.9375, stop: int = STOP_NONE, fp32: bool = False,
                 trace: bool = False) -> dict:
    """Decode one codeword under the true flooding schedule (every PE of every stage
    from iteration t-1's messages; no freezing).  Returns u_hat, iters, pe, margin and,
    with ``trace``, the L / R planes after each iteration ([iters, m+1, N])."""
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    N = frozen.shape[0]
    m = N.bit_length() - 1
    u_hat = np.zeros(N, np.uint8)
    iters = np.zeros(1, np.int32)
    pe = np.zeros(1, np.int64)
    margin = np.zeros(1, np.float64)
    tl = tr = None
    if trace:
        tl = np.full((max_iter, m + 1, N), np.nan, np.float64)
        tr = np.full((max_iter, m + 1, N), np.nan, np.float64)
    rc = _load().orc_decode_flood(N, _p(frozen, ctypes.c_uint8), _p(llr, ctypes.c_float), max_iter, alpha, stop,
                                  1 if fp32 else 0, _p(u_hat, ctypes.c_uint8), _p(iters, ctypes.c_int32),
                                  _p(pe, ctypes.c_int64), _p(margin, ctypes.c_double), _p(tl, ctypes.c_double),
                                  _p(tr, ctypes.c_double))
    _check(rc, "decode_flood")
    out = {"u_hat": u_hat, "iters": int(iters[0]), "pe": int(pe[0]), "margin": float(margin[0])}
    if trace:
        n = out["iters"]
        out.update(L=tl[:n], R=tr[:n])
    return out


def decode_flood_batch(frozen, llr, max_iter: int, alpha: float = 0.9375, stop: int = STOP_NONE,
                       fp32: bool = False, nthreads: int = 0):
    """Flooding-schedule decode of a [batch, N] LLR array; returns (u_hat, iters, pe, margin)."""
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    B, N = llr.shape
    u_hat = np.zeros((B, N), np.uint8)
    iters = np.zeros(B, np.int32)
    pe = np.zeros(B, np.int64)
    margin = np.zeros(B, np.float64)
    rc = _load().orc_decode_flood_batch(N, _p(frozen, ctypes.c_uint8), _p(llr, ctypes.c_float), B, max_iter,
                                        alpha, stop, 1 if fp32 else 0, nthreads, _p(u_hat, ctypes.c_uint8),
                                        _p(iters, ctypes.c_int32), _p(pe, ctypes.c_int64),
                                        _p(margin, ctypes.c_double))
    _check(rc, "decode_flood_batch")
    return u_hat, iters, pe, margin


def sc_decode(frozen, llr, exact: bool = True) -> np.ndarray:
    """Successive-cancellation decision (N,) for one codeword; exact box-plus f or min-sum."""
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    u_hat = np.zeros(frozen.shape[0], np.uint8)
    _check(_load().orc_sc_decode(frozen.shape[0], _p(frozen, ctypes.c_uint8), _p(llr, ctypes.c_float),
                                 1 if exact else 0, _p(u_hat, ctypes.c_uint8)), "sc_decode")
    return u_hat


def sc_decode_batch(frozen, llr, exact: bool = True, nthreads: int = 0) -> np.ndarray:
    """Successive-cancellation decisions [batch, N] for a [batch, N] LLR array."""
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    B, N = llr.shape
    u_hat = np.zeros((B, N), np.uint8)
    _check(_load().orc_sc_decode_batch(N, _p(frozen, ctypes.c_uint8), _p(llr, ctypes.c_float), B,
                                       1 if exact else 0, nthreads, _p(u_hat, ctypes.c_uint8)), "sc_decode_batch")
    return u_hat


def decode_q(frozen, llr, max_iter: int, A: int = 15, F: int = 2, stop: int = STOP_NONE, trace: bool = False) -> dict:
    """Quantised-message decode of one codeword (16-bit saturating integers, alpha = A/16, F
    fractional bits of the channel LLRs).  Returns u_hat, iters, pe and, with ``trace``, the
    integer planes after each iteration ([iters, m+1, N])."""
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    N = frozen.shape[0]
    m = N.bit_length() - 1
    u_hat = np.zeros(N, np.uint8)
    iters = np.zeros(1, np.int32)
    pe = np.zeros(1, np.int64)
    tl = tr = None
    if trace:
        tl = np.zeros((max_iter, m + 1, N), np.int32)
        tr = np.zeros((max_iter, m + 1, N), np.int32)
    _check(_load().orc_decode_q(N, _p(frozen, ctypes.c_uint8), _p(llr, ctypes.c_float), max_iter, A, F, stop,
                                _p(u_hat, ctypes.c_uint8), _p(iters, ctypes.c_int32), _p(pe, ctypes.c_int64),
                                _p(tl, ctypes.c_int32), _p(tr, ctypes.c_int32)), "decode_q")
    out = {"u_hat": u_hat, "iters": int(iters[0]), "pe": int(pe[0])}
    if trace:
        n = out["iters"]
        out.update(L=tl[:n], R=tr[:n])
    return out


def decode_q_batch(frozen, llr, max_iter: int, A: int = 15, F: int = 2, stop: int = STOP_NONE, nthreads: int = 0):
    """Quantised-message decode of a [batch, N] LLR array; returns (u_hat, iters, pe)."""
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    B, N = llr.shape
    u_hat = np.zeros((B, N), np.uint8)
    iters = np.zeros(B, np.int32)
    pe = np.zeros(B, np.int64)
    _check(_load().orc_decode_q_batch(N, _p(frozen, ctypes.c_uint8), _p(llr, ctypes.c_float), B, max_iter, A, F,
                                      stop, nthreads, _p(u_hat, ctypes.c_uint8), _p(iters, ctypes.c_int32),
                                      _p(pe, ctypes.c_int64)), "decode_q_batch")
    return u_hat, iters, pe


def wms_forward(frozen, llr, weights, fp32: bool = False, trace: bool = False):
    """Weighted min-sum soft outputs (N,) after T iterations; weights [T, m, N/2]."""
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    N = frozen.shape[0]
    m = N.bit_length() - 1
    T = w.shape[0]
    out = np.zeros(N, np.float64)
    tl = tr = None
    if trace:
        tl = np.zeros((T, m + 1, N), np.float64)
        tr = np.zeros((T, m + 1, N), np.float64)
    _check(_load().orc_wms_forward(N, _p(frozen, ctypes.c_uint8), _p(llr, ctypes.c_float), T, _p(w, ctypes.c_double),
                                   1 if fp32 else 0, _p(out, ctypes.c_double), _p(tl, ctypes.c_double),
                                   _p(tr, ctypes.c_double)), "wms_forward")
    return (out, tl, tr) if trace else out


def wms_backward(frozen, llr, weights, dout, fp32: bool = False):
    """(dweights [T, m, N/2], dllr [N]) of sum(dout * out) through wms_forward: FP64, or with
    fp32 the binary32 forward and every adjoint operation rounded to binary32."""
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    d = np.ascontiguousarray(dout, dtype=np.float64)
    N = frozen.shape[0]
    dw = np.zeros_like(w)
    dl = np.zeros(N, np.float64)
    _check(_load().orc_wms_backward(N, _p(frozen, ctypes.c_uint8), _p(llr, ctypes.c_float), w.shape[0],
                                    _p(w, ctypes.c_double), _p(d, ctypes.c_double), 1 if fp32 else 0,
                                    _p(dw, ctypes.c_double),
                                    _p(dl, ctypes.c_double)), "wms_backward")
    return dw, dl


RULE_R, RULE_R_PLUS_L, RULE_THRESHOLD = 0, 1, 2


def decode_rule_batch(frozen, llr, max_iter: int, alpha: float = 0.9375, stop: int = STOP_NONE, rule: int = RULE_R,
                      theta: float = 0.0, fp32: bool = False, nthreads: int = 0):
    """Reading-A freezing with a variant of the CSFG check (rule 0: Eqs. (2)-(4) on R; 1: on R + L;
    2: on R, only when every |R| of the CSFG is >= theta); returns (u_hat, iters, pe)."""
    frozen = np.ascontiguousarray(frozen, dtype=np.uint8)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    B, N = llr.shape
    u_hat = np.zeros((B, N), np.uint8)
    iters = np.zeros(B, np.int32)
    pe = np.zeros(B, np.int64)
    _check(_load().orc_decode_rule_batch(N, _p(frozen, ctypes.c_uint8), _p(llr, ctypes.c_float), B, max_iter, alpha,
                                         stop, rule, theta, 1 if fp32 else 0, nthreads, _p(u_hat, ctypes.c_uint8),
                                         _p(iters, ctypes.c_int32), _p(pe, ctypes.c_int64)), "decode_rule_batch")
    return u_hat, iters, pe


def bit_reverse_permutation(N: int) -> np.ndarray:
    """rev[i] = the m-bit reversal of i (N = 2^m): Arikan's B_N as an index map."""
    m = N.bit_length() - 1
    i = np.arange(N)
    r = np.zeros(N, np.int64)
    for b in range(m):
        r |= ((i >> b) & 1) << (m - 1 - b)
    return r


def encode_bit_reversed(u: np.ndarray) -> np.ndarray:
    """x = u B_N F^{(x)m} (Sec. II with Arikan's bit-reversal): channel position i carries
    position rev(i) of the natural encoding u F^{(x)m}, as B_N F^{(x)m} = F^{(x)m} B_N."""
    x = encode(u)
    return np.ascontiguousarray(x[..., bit_reverse_permutation(x.shape[-1])])


def natural_order_llr(llr_channel: np.ndarray) -> np.ndarray:
    """LLRs received in bit-reversed channel order, put back in code-position order (B_N is an
    involution): decoding a bit-reversed codeword is the natural decode of these."""
    llr_channel = np.ascontiguousarray(llr_channel)
    return np.ascontiguousarray(llr_channel[..., bit_reverse_permutation(llr_channel.shape[-1])])
