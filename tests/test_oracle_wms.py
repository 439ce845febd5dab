"""Pins of the oracle's weighted min-sum (Eq. (1) with per-(iteration, stage, PE)
weights) and its analytic gradient."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04979_gb300 import inputs as I


def setup(N, T, seed, ebn0=2.0):
    K = N // 2
    m = N.bit_length() - 1
    fz = O.bec_frozen(N, K)
    u = I.info_bits(seed, np.arange(1), fz)
    llr = I.channel_llr(O.encode(u), I.gaussian(seed, np.arange(1), N), I.sigma(ebn0, K / N))[0]
    w = np.random.default_rng(seed).uniform(0.6, 1.3, (T, m, N // 2))
    return fz, llr, w


@pytest.mark.parametrize("N,T", [(16, 3), (16, 10), (64, 6)])
def test_constant_weights_reproduce_scaled_min_sum(N, T):
    """All weights = alpha gives the planes of the scaled min-sum decoder, fixed iterations."""
    fz, llr, _ = setup(N, T, 1)
    m = N.bit_length() - 1
    w = np.full((T, m, N // 2), 0.9375)
    out, tl, tr = O.wms_forward(fz, llr, w, trace=True)
    r = O.decode(fz, llr, T, 0.9375, trace=True)
    assert np.array_equal(tl, r["L"]) and np.array_equal(tr, r["R"])
    assert np.array_equal(out, r["R"][-1][m] + r["L"][-1][m])


@pytest.mark.parametrize("s", [0, 1, 2, 3])
def test_weight_layout_addresses_one_pe(s):
    """Changing weight (t=0, s, p) changes iteration 1's stage-s outputs exactly at the two
    positions (a, a + 2^(m-1-s)) of PE p, p = (a >> (m-s)) * 2^(m-1-s) + a mod 2^(m-1-s)."""
    N, T = 16, 1
    m = 4
    fz, llr, w = setup(N, T, 3)
    h = 1 << (m - 1 - s)
    for p in range(N // 2):
        w2 = w.copy()
        w2[0, s, p] *= 1.5
        _, tl1, tr1 = O.wms_forward(fz, llr, w, trace=True)
        _, tl2, tr2 = O.wms_forward(fz, llr, w2, trace=True)
        changed = np.nonzero((tr1[0][s + 1] != tr2[0][s + 1]) | (tl1[0][s] != tl2[0][s]))[0]
        a = (p // h) * 2 * h + p % h
        assert set(changed.tolist()) <= {a, a + h} and len(changed) > 0


@pytest.mark.parametrize("N,T,seed", [(16, 4, 5), (16, 10, 6), (8, 7, 7)])
def test_gradient_matches_central_differences(N, T, seed):
    """Analytic adjoint vs central finite differences (h = 1e-6) of L = sum(c * out)."""
    fz, llr, w = setup(N, T, seed)
    c = np.random.default_rng(seed + 100).normal(0, 1, N)
    c[fz == 1] = 0.0  # the loss sees the information positions (frozen outputs are the +inf prior)
    info = fz == 0
    F = lambda ww, ll: float(c[info] @ O.wms_forward(fz, ll, ww)[info])
    dw, dl = O.wms_backward(fz, llr, w, c)
    rng = np.random.default_rng(seed + 200)
    hstep = 1e-6
    flat = w.reshape(-1)
    picks = rng.choice(flat.size, min(120, flat.size), replace=False)
    checked = 0
    for k in picks:
        wp = flat.copy(); wp[k] += hstep
        wm = flat.copy(); wm[k] -= hstep
        fd = (F(wp.reshape(w.shape), llr) - F(wm.reshape(w.shape), llr)) / (2 * hstep)
        an = dw.reshape(-1)[k]
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (k, fd, an)
        checked += abs(an) > 0
    assert checked > 10
    # channel LLRs (binary32 inputs: step in double through a double copy of the input)
    for i in range(N):
        lp = llr.astype(np.float64).copy(); lm = lp.copy()
        lp[i] += 1e-3; lm[i] -= 1e-3
        fp = F(w, lp.astype(np.float32))
        fm = F(w, lm.astype(np.float32))
        fd = (fp - fm) / (float(np.float32(lp[i])) - float(np.float32(lm[i])))
        assert abs(fd - dl[i]) <= 1e-4 * max(1.0, abs(dl[i])), (i, fd, dl[i])


@pytest.mark.parametrize("N,T,seed", [(16, 3, 11), (32, 4, 12)])
def test_binary32_adjoint_equals_fp64_when_nothing_rounds(N, T, seed):
    """The binary32 mode of the adjoint applies the same chain rule as the FP64 one: with
    LLRs on a grid of 1/8, weights in {1/2, 3/4, 1} and integer dout, every forward and
    adjoint value has few significant bits, nothing rounds, and the two modes agree exactly
    (a term dropped or reordered in one mode alone would break this)."""
    m = N.bit_length() - 1
    fz = O.bec_frozen(N, N // 2)
    rng = np.random.default_rng(seed)
    llr = (rng.integers(-40, 41, N) / 8.0).astype(np.float32)
    w = rng.choice([0.5, 0.75, 1.0], (T, m, N // 2))
    dout = rng.integers(-3, 4, N).astype(np.float64)
    dout[fz == 1] = 0.0
    dw64, dl64 = O.wms_backward(fz, llr, w, dout)
    dw32, dl32 = O.wms_backward(fz, llr, w, dout, fp32=True)
    assert np.array_equal(dw32, dw64) and np.array_equal(dl32, dl64)
    assert np.count_nonzero(dw64) > 10
    # every value is a binary32 number
    assert np.array_equal(dw32.astype(np.float32).astype(np.float64), dw32)


def test_binary32_adjoint_close_to_fp64():
    """On channel inputs the binary32 adjoint differs from FP64 only by rounding."""
    N, T = 64, 10
    fz, llr, w = setup(N, T, 21)
    dout = np.random.default_rng(22).normal(0, 1, N)
    dout[fz == 1] = 0.0
    dout = dout.astype(np.float32).astype(np.float64)
    w = w.astype(np.float32).astype(np.float64)
    dw64, dl64 = O.wms_backward(fz, llr, w, dout)
    dw32, dl32 = O.wms_backward(fz, llr, w, dout, fp32=True)
    for a, b in ((dw32, dw64), (dl32, dl64)):
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
    assert np.array_equal(dw32.astype(np.float32).astype(np.float64), dw32)
