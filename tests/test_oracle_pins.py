"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test names the passage of arXiv 1505.04979 it pins and what fixes the
expected value: a brute-force enumeration, a library routine standing in for a
textbook definition (np.kron), a hand-derived closed form (tests/golden), an
invariant derived by hand, or maximum-likelihood decoding by exhaustive search.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04979_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
F = np.array([[1, 0], [1, 1]], dtype=np.int64)


def kron_G(N):
    """G = F^{(x)m} built with numpy's Kronecker product (Sec. II)."""
    G = np.ones((1, 1), np.int64)
    while G.shape[0] < N:
        G = np.kron(G, F)
    return G


# --------------------------------------------------------------------------
# Sec. II: frozen set from the BEC recursion, pinned by brute-force erasure
# enumeration of the synthetic channels under successive cancellation.
# --------------------------------------------------------------------------
def _in_span(target, vectors):
    """GF(2) membership of bitmask `target` in the span of bitmask `vectors`."""
    basis = {}
    for v in vectors:
        while v:
            h = v.bit_length() - 1
            if h in basis:
                v ^= basis[h]
            else:
                basis[h] = v
                break
    t = target
    while t:
        h = t.bit_length() - 1
        if h not in basis:
            return False
        t ^= basis[h]
    return True


def brute_force_erasure(N, z0):
    """Erasure probability of u_i given u_0..u_{i-1} when every x_c is erased with prob z0."""
    G = kron_G(N)
    z = np.zeros(N)
    for pattern in range(1 << N):
        erased = [(pattern >> c) & 1 for c in range(N)]
        ne = sum(erased)
        p = (z0 ** ne) * ((1 - z0) ** (N - ne))
        for i in range(N):
            # unknowns u_i..u_{N-1}; bit r-i of a mask stands for u_r
            cols = []
            for c in range(N):
                if not erased[c]:
                    mask = 0
                    for r in range(i, N):
                        if G[r, c]:
                            mask |= 1 << (r - i)
                    cols.append(mask)
            if not _in_span(1, cols):
                z[i] += p
    return z


@pytest.mark.parametrize("N", [2, 4, 8])
@pytest.mark.parametrize("z0", [0.5, 0.3])
def test_bec_z_matches_brute_force_erasure(N, z0):
    a, _ = O.bec_lnz(N, z0)
    np.testing.assert_allclose(np.exp(a), brute_force_erasure(N, z0), rtol=0, atol=1e-12)


def test_bec_8_4_frozen_set():
    """The (8,4) code of Sec. III (Figs. 3-5): frozen set {0,1,2,4}, from the brute-force z."""
    z = brute_force_erasure(8, 0.5)
    expected = set(np.argsort(-z, kind="stable")[:4].tolist())
    assert expected == {0, 1, 2, 4}
    assert set(np.nonzero(O.bec_frozen(8, 4))[0].tolist()) == {0, 1, 2, 4}


CODE_SIZES = [(16, 8), (64, 32), (128, 64), (256, 64), (256, 128), (256, 192), (1024, 256), (1024, 512),
              (1024, 768), (4096, 1024), (4096, 2048), (4096, 3072), (8192, 4096), (16384, 8192),
              (32768, 16384)]


@pytest.mark.parametrize("N,K", CODE_SIZES)
def test_frozen_set_size_and_partial_order(N, K):
    """|A^c| = N-K, and the information set is closed upward in the bitwise partial
    order of polar channels (if i is information and j covers i bitwise, j is information)."""
    fz = O.bec_frozen(N, K)
    assert int(fz.sum()) == N - K
    info = fz == 0
    for b in range(N.bit_length() - 1):
        i = np.arange(N)
        has = (i >> b) & 1
        lo = i[has == 0]
        hi = lo | (1 << b)
        assert not np.any(info[lo] & ~info[hi])


@pytest.mark.parametrize("N", [64, 1024, 32768])
def test_bec_sum_is_conserved(N):
    """A BEC split preserves the sum of erasure probabilities: sum z = N z0."""
    a, _ = O.bec_lnz(N, 0.5)
    assert math.isclose(float(np.exp(a).sum()), N * 0.5, rel_tol=1e-9)


# --------------------------------------------------------------------------
# Sec. II: encoder x = u F^{(x)m}
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [2, 4, 8, 16])
def test_encoder_matches_dense_kronecker(N):
    G = kron_G(N)
    for u in itertools.product([0, 1], repeat=N) if N <= 8 else np.random.default_rng(0).integers(0, 2, (300, N)):
        u = np.array(u, np.uint8)
        assert np.array_equal(O.encode(u), (u.astype(np.int64) @ G % 2).astype(np.uint8))


@pytest.mark.parametrize("N", [2, 64, 1024])
def test_encoder_is_an_involution(N):
    """Eq. (3): (F^{(x)m})^{-1} = F^{(x)m}."""
    u = np.random.default_rng(N).integers(0, 2, (20, N)).astype(np.uint8)
    assert np.array_equal(O.encode(O.encode(u)), u)


# --------------------------------------------------------------------------
# Eq. (2)-(4) and Lemma 1: brute-force maximum likelihood on constituent codes
# --------------------------------------------------------------------------
@pytest.mark.parametrize("S", [2, 4, 8, 16])
def test_lemma1_check_implies_ml(S):
    rng = np.random.default_rng(S)
    G = kron_G(S)
    passes = 0
    for trial in range(300):
        nfz = rng.integers(1 if S > 2 else 0, S)
        fz = np.zeros(S, np.uint8)
        fz[rng.choice(S, nfz, replace=False)] = 1
        if (fz == 0).sum() > 10:
            continue
        # LLRs of a valid codeword plus noise, so the check passes often enough
        u = rng.integers(0, 2, S) * (1 - fz)
        x = u @ G % 2
        R = (1 - 2 * x) * 2.0 + rng.normal(0, 1.0 + trial % 3, S)
        ok, xh, uh = O.csfg_check(R, fz)
        # the check's hard decisions are Eq. (2) and its source word is Eq. (3)
        assert np.array_equal(xh, (R < 0).astype(np.uint8))
        if not ok:
            assert np.any(uh[fz == 1] == 1)
            continue
        passes += 1
        info = np.nonzero(fz == 0)[0]
        U = np.zeros((1 << len(info), S), np.int64)
        U[:, info] = np.array(list(itertools.product([0, 1], repeat=len(info))), np.int64).reshape(-1, len(info))
        best = float(np.max((1 - 2 * (U @ G % 2)) @ R))
        xu = uh.astype(np.int64) @ G % 2
        like = float(np.sum((1 - 2 * xu) * R))
        assert abs(like - best) < 1e-9
        assert abs(like - np.abs(R).sum()) < 1e-9  # the bound used in the proof of Lemma 1
    assert passes > 20


def test_eq2_maps_zero_to_zero():
    """Eq. (2): values >= 0, including -0.0, decide 0."""
    ok, xh, uh = O.csfg_check(np.array([0.0, -0.0, -1.0, 2.0]), np.zeros(4, np.uint8))
    assert xh.tolist() == [0, 0, 1, 0]


# --------------------------------------------------------------------------
# Eq. (1): closed forms worked by hand
# --------------------------------------------------------------------------
def test_n2_is_the_repetition_ml_decoder():
    """(2,1) code, frozen {0}: with alpha = 1 BP decides u_1 = [y_0 + y_1 < 0],
    the maximum-likelihood decision of a length-2 repetition code."""
    rng = np.random.default_rng(2)
    fz = np.array([1, 0], np.uint8)
    for _ in range(500):
        y = rng.normal(0, 3, 2).astype(np.float32)
        if abs(float(y[0]) + float(y[1])) < 1e-6:
            continue
        for it in (1, 4):
            r = O.decode(fz, y, it, alpha=1.0)
            assert r["u_hat"].tolist() == [0, int(float(y[0]) + float(y[1]) < 0)]


def test_n2_first_iteration_messages():
    """(2,1) code, frozen {0}, L[1] = [inf, 0]: after iteration 1, R[1] = [f(y0, y1), y1 + alpha y0]
    and L[0] = [f(inf, y1), 0 + f(inf, y0)] = [alpha y1, alpha y0] (Eq. (1) by hand)."""
    y = np.array([1.5, -0.25], np.float32)
    r = O.decode(np.array([1, 0], np.uint8), y, 1, alpha=0.5, trace=True)
    R1 = r["R"][0][1]
    L0 = r["L"][0][0]
    assert R1.tolist() == [-0.125, -0.25 + 0.75]  # f(y0, y1): alpha*sgn*sgn*min = -0.125
    assert L0.tolist() == [0.5 * -0.25, 0.5 * 1.5]  # f(inf, y1) = alpha y1; 0 + f(inf, y0)


def test_n4_closed_form_two_iterations():
    g = json.load(open(os.path.join(GOLDEN, "n4_closed_form.json")))
    conv = lambda v: [np.inf if e == "inf" else (-np.inf if e == "-inf" else e) for e in v]
    r = O.decode(np.array(g["frozen"], np.uint8), np.array(g["llr"], np.float32), 2, alpha=g["alpha"], trace=True)
    for it, key in ((0, "iter1"), (1, "iter2")):
        e = g[key]
        assert r["R"][it][1].tolist() == conv(e["R1"])
        assert r["R"][it][2].tolist() == conv(e["R2"])
        assert r["L"][it][0].tolist() == conv(e["L0"])
        assert r["L"][it][1].tolist() == conv(e["L1"])
    assert r["u_hat"].tolist() == g["u_hat"]


def test_n4_is_two_repetition_codes():
    """(4,2) code, frozen {0,1}: x = (u2^u3, u3, u2^u3, u3), two repetition codes.
    With alpha = 1, BP (two or more iterations) gives their ML decisions."""
    rng = np.random.default_rng(4)
    fz = np.array([1, 1, 0, 0], np.uint8)
    for _ in range(400):
        y = rng.normal(0, 2, 4).astype(np.float32)
        s02 = float(y[0]) + float(y[2])
        s13 = float(y[1]) + float(y[3])
        if min(abs(s02), abs(s13)) < 1e-6:
            continue
        u3 = int(s13 < 0)
        u2 = int(s02 < 0) ^ u3
        for it in (2, 7):
            assert O.decode(fz, y, it, alpha=1.0)["u_hat"].tolist() == [0, 0, u2, u3]


# --------------------------------------------------------------------------
# Noiseless input: invariants derived by hand (iteration 1 of the sweep yields
# the correct hard decisions at every level, so every check passes)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [8, 64, 1024])
@pytest.mark.parametrize("frac", [0.25, 0.5, 0.75])
def test_noiseless_invariants(N, frac):
    K = int(N * frac)
    m = N.bit_length() - 1
    fz = O.bec_frozen(N, K)
    u = I.info_bits(11, np.arange(4), fz)
    x = O.encode(u)
    llr = I.noiseless_llr(x, 2.5)
    for c in range(4):
        r = O.decode(fz, llr[c], 30, stop=O.STOP_GMATRIX)
        assert (r["iters"], r["pe"]) == (1, m * N // 2) and np.array_equal(r["u_hat"], u[c])
        r = O.decode(fz, llr[c], 30, freeze=O.FREEZE_CSFG)
        assert (r["iters"], r["pe"]) == (2, 3 * N // 2 - 1) and np.array_equal(r["u_hat"], u[c])
        r = O.decode(fz, llr[c], 30, stop=O.STOP_GMATRIX, freeze=O.FREEZE_CSFG)
        assert (r["iters"], r["pe"]) == (1, N - 1) and np.array_equal(r["u_hat"], u[c])
        for it in (1, 5):
            r = O.decode(fz, llr[c], it)
            assert (r["iters"], r["pe"]) == (it, it * m * N // 2) and np.array_equal(r["u_hat"], u[c])


# --------------------------------------------------------------------------
# Invariants on noisy decodes
# --------------------------------------------------------------------------
def _noisy(N, K, B, ebn0, seed):
    fz = O.bec_frozen(N, K)
    idx = np.arange(B)
    u = I.info_bits(seed, idx, fz)
    x = O.encode(u)
    llr = I.channel_llr(x, I.gaussian(seed, idx, N), I.sigma(ebn0, K / N))
    return fz, u, x, llr


@pytest.mark.parametrize("N", [16, 64, 256])
def test_freezing_invariants_on_noisy_input(N):
    """Sec. III: R messages stay finite; the covered set only grows; frozen outputs
    are 0; and every +-inf feedback plane agrees with one PE butterfly of the
    plane to its right (what Eq. (1) yields on +-inf inputs), which is reading R4."""
    m = N.bit_length() - 1
    fz, u, x, llr = _noisy(N, N // 2, 40, 2.0, 5)
    saw_inf_pair = 0
    for c in range(llr.shape[0]):
        for stop in (O.STOP_NONE, O.STOP_GMATRIX):
            r = O.decode(fz, llr[c], 25, stop=stop, freeze=O.FREEZE_CSFG, trace=True)
            assert np.all(np.isfinite(r["R"]))
            assert np.all(np.diff(r["P"]) >= 0)
            assert np.all(r["u_hat"][fz == 1] == 0)
            assert int(r["pe_iter"].sum()) == r["pe"]
            L = r["L"][-1]
            for j in range(1, m):
                S = N >> j
                for k in range(1 << j):
                    blk = slice(k * S, (k + 1) * S)
                    if np.all(np.isinf(L[j, blk])) and np.all(np.isinf(L[j + 1, blk])):
                        h = S // 2
                        xa = L[j + 1, k * S:k * S + h] < 0
                        xb = L[j + 1, k * S + h:(k + 1) * S] < 0
                        got = L[j, blk] < 0
                        assert np.array_equal(got[:h], xa ^ xb) and np.array_equal(got[h:], xb)
                        saw_inf_pair += 1
    assert saw_inf_pair > 0


def test_fp32_mode_rounds_every_message():
    fz, u, x, llr = _noisy(64, 32, 8, 2.5, 9)
    for c in range(8):
        r = O.decode(fz, llr[c], 12, stop=O.STOP_GMATRIX, freeze=O.FREEZE_CSFG, fp32=True, trace=True)
        for planes in (r["L"], r["R"]):
            finite = planes[np.isfinite(planes)]
            assert np.array_equal(finite, finite.astype(np.float32).astype(np.float64))


def test_fp32_and_fp64_agree_away_from_thresholds():
    fz, u, x, llr = _noisy(256, 128, 60, 2.5, 3)
    a = O.decode_batch(fz, llr, 40, stop=O.STOP_GMATRIX, freeze=O.FREEZE_CSFG)
    b = O.decode_batch(fz, llr, 40, stop=O.STOP_GMATRIX, freeze=O.FREEZE_CSFG, fp32=True)
    # a decision taken on a value this far from 0 cannot flip under binary32 rounding here
    safe = a[3] > 1e-4
    assert safe.sum() > 40
    assert np.array_equal(a[0][safe], b[0][safe])
    assert np.array_equal(a[1][safe], b[1][safe])


def test_statistics_at_3db_are_plausible():
    """Sec. IV, (1024,512), alpha = 0.9375, max_iter = 40, 3 dB: the paper reports no FER
    loss from either stop rule and about 26 G-matrix iterations (derived from its -46%/-17%
    figures).  These pin only loosely: 300 codewords."""
    fz, u, x, llr = _noisy(1024, 512, 300, 3.0, 21)
    res = {}
    for mode in ((0, 0), (1, 0), (1, 1), (0, 1)):
        uh, it, pe, _ = O.decode_batch(fz, llr, 40, stop=mode[0], freeze=mode[1])
        res[mode] = ((uh != u).any(1).mean(), it.mean(), pe.mean())
    assert res[(0, 0)][0] < 0.08
    for mode in res:
        assert abs(res[mode][0] - res[(0, 0)][0]) <= 0.02
    assert 18.0 < res[(1, 0)][1] < 32.0
    assert res[(1, 1)][2] <= res[(1, 0)][2]
    assert res[(0, 1)][2] < res[(0, 0)][2]


def test_n8_freeze_hand_trace():
    """Two iterations of the (8,4) code with freezing, worked by hand (Eq. (1), Eqs. (2)-(4),
    Sec. III freezing order, Sec. IV count): a stage-1 CSFG freezes after stage 0 of iteration 1,
    the later stages skip its PEs, every later check fails, and the G test does not stop."""
    g = json.load(open(os.path.join(GOLDEN, "n8_freeze_hand_trace.json")))
    fz = np.array(g["frozen"], np.uint8)
    llr = np.array(g["llr"], np.float32)
    for stop in (0, 1):
        o = O.decode(fz, llr, g["max_iter"], g["alpha"], stop, 1, trace=True)
        assert o["iters"] == g["max_iter"]
        assert o["pe"] == sum(it["pe"] for it in g["iterations"])
        assert np.array_equal(o["u_hat"], np.array(g["u_hat"], np.uint8))
        for t, it in enumerate(g["iterations"]):
            assert o["P"][t] == it["P"]
            assert o["pe_iter"][t] == it["pe"]
            for plane, key in (("R", "R"), ("L", "L")):
                for c, vals in it[key].items():
                    for i, v in vals.items():
                        want = np.inf if v == "inf" else float(v)
                        assert o[plane][t][int(c), int(i)] == want, (stop, t, plane, c, i)


# --------------------------------------------------------------------------
# True flooding schedule (a variant beside the sweep of Eq. (1)): every PE takes
# both its L and its R inputs from the previous iteration
# --------------------------------------------------------------------------
def test_flooding_n4_hand_trace():
    g = json.load(open(os.path.join(GOLDEN, "n4_flooding.json")))
    conv = lambda v: [np.inf if e == "inf" else (-np.inf if e == "-inf" else e) for e in v]
    r = O.decode_flood(np.array(g["frozen"], np.uint8), np.array(g["llr"], np.float32), 2, alpha=g["alpha"],
                       trace=True)
    for it, key in ((0, "iter1"), (1, "iter2")):
        e = g[key]
        assert r["R"][it][1].tolist() == conv(e["R1"])
        assert r["R"][it][2].tolist() == conv(e["R2"])
        assert r["L"][it][0].tolist() == conv(e["L0"])
        assert r["L"][it][1].tolist() == conv(e["L1"])
    assert r["u_hat"].tolist() == g["u_hat"] and r["pe"] == g["pe"]


def test_flooding_n2_equals_sweep():
    """With one stage there is no interior column: both schedules read only the channel
    and the prior, so every message of every iteration is the sweep's (itself pinned by
    the N = 2 closed forms)."""
    rng = np.random.default_rng(9)
    for fz in ([1, 0], [0, 0], [1, 1]):
        fz = np.array(fz, np.uint8)
        for _ in range(50):
            llr = rng.normal(0, 3, 2).astype(np.float32)
            a = O.decode(fz, llr, 4, trace=True)
            b = O.decode_flood(fz, llr, 4, trace=True)
            assert np.array_equal(a["L"], b["L"]) and np.array_equal(a["R"], b["R"])
            assert np.array_equal(a["u_hat"], b["u_hat"]) and a["pe"] == b["pe"]


@pytest.mark.parametrize("N", [8, 64, 256])
def test_flooding_moves_one_column_per_iteration(N):
    """Interior messages start at 0 and a PE whose L (R) inputs are all 0 emits 0 on
    that side, so after t < m iterations R[s] = 0 for s > t and L[s] = 0 for s < m - t;
    the sweep, by contrast, reaches R[m] in its first iteration."""
    m = N.bit_length() - 1
    fz, u, x, llr = _noisy(N, N // 2, 3, 2.0, 21)
    for c in range(llr.shape[0]):
        r = O.decode_flood(fz, llr[c], m, trace=True)
        for t in range(1, m):
            R, L = r["R"][t - 1], r["L"][t - 1]
            assert np.all(R[t + 1:] == 0) and np.any(R[t] != 0)
            assert np.all(L[:m - t] == 0)
        assert np.any(O.decode(fz, llr[c], 1, trace=True)["R"][0][m] != 0)


@pytest.mark.parametrize("N", [8, 64, 1024])
def test_flooding_noiseless_stops_at_iteration_m(N):
    """Noiseless input: every message sign agrees with the codeword, and R[m] stays 0 until
    the channel's wavefront reaches it in iteration m.  So for a nonzero source word the
    G-matrix test fails before iteration m and passes exactly there, with u_hat = u;
    fixed iterations t < m decide 0 on every information position."""
    m = N.bit_length() - 1
    fz = O.bec_frozen(N, N // 2)
    u = I.info_bits(12, np.arange(4), fz)
    x = O.encode(u)
    llr = I.noiseless_llr(x, 2.5)
    for c in range(4):
        assert u[c].any()
        r = O.decode_flood(fz, llr[c], 3 * m, stop=O.STOP_GMATRIX)
        assert (r["iters"], r["pe"]) == (m, m * m * N // 2) and np.array_equal(r["u_hat"], u[c])
        r = O.decode_flood(fz, llr[c], m - 1)
        assert not r["u_hat"].any()
        r = O.decode_flood(fz, llr[c], m)
        assert np.array_equal(r["u_hat"], u[c])


def test_flooding_batch_matches_single_and_fp32():
    fz, u, x, llr = _noisy(64, 32, 30, 2.5, 33)
    uh, it, pe, _ = O.decode_flood_batch(fz, llr, 40, stop=O.STOP_GMATRIX, fp32=True)
    for c in range(llr.shape[0]):
        r = O.decode_flood(fz, llr[c], 40, stop=O.STOP_GMATRIX, fp32=True)
        assert np.array_equal(uh[c], r["u_hat"]) and it[c] == r["iters"] and pe[c] == r["pe"]


# --------------------------------------------------------------------------
# Reading B of the freezing order (a variant): after a CSFG of stage j passes,
# the next CSFG of stage j is checked at once, on the same R[j]
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [8, 64, 1024])
@pytest.mark.parametrize("frac", [0.25, 0.5, 0.75])
def test_reading_b_noiseless_freezes_stage_1(N, frac):
    """Noiseless input, iteration 1: after stage 0, R[1] = (f(y_a, y_b), y_b) with L[1] = 0, whose
    hard decisions are the encodings of the two halves of u.  Both stage-1 CSFGs pass, so reading B
    covers everything after N/2 PE updates, with or without the G-matrix stop (reading A needs
    2 iterations and 3N/2 - 1 PEs there)."""
    K = int(N * frac)
    fz = O.bec_frozen(N, K)
    u = I.info_bits(11, np.arange(4), fz)
    llr = I.noiseless_llr(O.encode(u), 2.5)
    for c in range(4):
        for stop in (O.STOP_NONE, O.STOP_GMATRIX):
            r = O.decode(fz, llr[c], 30, stop=stop, freeze=O.FREEZE_CSFG_MULTI)
            assert (r["iters"], r["pe"]) == (1, N // 2) and np.array_equal(r["u_hat"], u[c])


def test_reading_b_n8_hand_trace_extra_check_fails():
    """The hand-traced (8,4) example: in iteration 1 the stage-1 CSFG [0,4) freezes, and reading B
    then checks [4,8) on the same R1 = (4, 6, -1, 2): x = (0,0,1,0), u = x F = (1,0,1,0), and u(4) = 1
    sits on a frozen position, so it fails; deeper stages and iteration 2 go as under reading A.
    Every value of the fixture must therefore come out unchanged."""
    g = json.load(open(os.path.join(GOLDEN, "n8_freeze_hand_trace.json")))
    conv = lambda v: np.inf if v == "inf" else (-np.inf if v == "-inf" else v)
    r = O.decode(np.array(g["frozen"], np.uint8), np.array(g["llr"], np.float32), g["max_iter"], alpha=g["alpha"],
                 freeze=O.FREEZE_CSFG_MULTI, trace=True)
    for t, e in enumerate(g["iterations"]):
        assert int(r["P"][t]) == e["P"] and int(r["pe_iter"][t]) == e["pe"]
        for col, vals in e["R"].items():
            for i, v in vals.items():
                assert r["R"][t][int(col)][int(i)] == conv(v)
        for col, vals in e["L"].items():
            for i, v in vals.items():
                assert r["L"][t][int(col)][int(i)] == conv(v)
    assert r["u_hat"].tolist() == g["u_hat"]


@pytest.mark.parametrize("N", [16, 64, 256])
def test_reading_b_covers_at_least_reading_a_in_iteration_1(N):
    """In iteration 1 a checked CSFG's R comes from PEs of enclosing CSFGs that are uncovered under
    both readings, all fed by the channel and the zero start, so both readings see the same values
    on it.  Stage by stage, reading B's prefix is then at least reading A's: on the same candidate it
    takes the same decision and may go on along the stage; on a later candidate, A's candidate ends
    before B's prefix."""
    fz, u, x, llr = _noisy(N, N // 2, 40, 3.0, 41)
    for c in range(llr.shape[0]):
        a = O.decode(fz, llr[c], 1, freeze=O.FREEZE_CSFG, trace=True)
        b = O.decode(fz, llr[c], 1, freeze=O.FREEZE_CSFG_MULTI, trace=True)
        assert int(b["P"][0]) >= int(a["P"][0])


# --------------------------------------------------------------------------
# Successive-cancellation decoding (the cross-check of Sec. III's comparison
# between a frozen CSFG's decision and SC decoding of its constituent code)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("N", [8, 64, 1024])
@pytest.mark.parametrize("exact", [True, False])
def test_sc_noiseless(N, exact):
    for frac in (0.25, 0.5, 0.75):
        fz = O.bec_frozen(N, int(N * frac))
        u = I.info_bits(13, np.arange(4), fz)
        llr = I.noiseless_llr(O.encode(u), 2.5)
        assert np.array_equal(O.sc_decode_batch(fz, llr, exact), u)


@pytest.mark.parametrize("exact", [True, False])
def test_sc_n2_closed_forms(exact):
    """N = 2, x = (u0 ^ u1, u1): u0 = HD(f(y0, y1)) (the sign of f is sign(y0) sign(y1) for both f),
    then u1 = HD(y1 + (1 - 2 u0) y0); with u0 frozen, u1 = HD(y0 + y1)."""
    rng = np.random.default_rng(3)
    for _ in range(300):
        y = rng.normal(0, 2, 2).astype(np.float32)
        y0, y1 = float(y[0]), float(y[1])
        if min(abs(y0), abs(y1), abs(y0 + y1), abs(y1 - y0)) < 1e-6:
            continue
        u0 = int((np.sign(y0) * np.sign(y1)) < 0)
        u1 = int(y1 + (1 - 2 * u0) * y0 < 0)
        assert O.sc_decode(np.array([0, 0], np.uint8), y, exact).tolist() == [u0, u1]
        assert O.sc_decode(np.array([1, 0], np.uint8), y, exact).tolist() == [0, int(y0 + y1 < 0)]


@pytest.mark.parametrize("exact", [True, False])
def test_sc_rate_one_is_reencoded_hard_decision(exact):
    """With no frozen position every split keeps the hard decisions of its inputs (the sign of f is
    the xor of the signs, and g keeps the sign of its right input), so u_hat = HD(y) F^{(x)m}."""
    rng = np.random.default_rng(5)
    N = 64
    fz = np.zeros(N, np.uint8)
    y = rng.normal(0, 2, (50, N)).astype(np.float32)
    hd = (y < 0).astype(np.uint8)
    assert np.array_equal(O.sc_decode_batch(fz, y, exact), O.encode(hd))


@pytest.mark.parametrize("exact", [True, False])
def test_sc_repetition_code_is_ml(exact):
    """Only the last position carries information: every earlier bit decides 0, each g then adds
    the two halves, and the last bit decides on the sign of the sum of all LLRs (the ML decision)."""
    rng = np.random.default_rng(6)
    for N in (4, 16, 128):
        fz = np.ones(N, np.uint8)
        fz[-1] = 0
        y = rng.normal(0.3, 2, (40, N)).astype(np.float32)
        s = y.astype(np.float64).sum(axis=1)
        keep = np.abs(s) > 1e-4
        out = O.sc_decode_batch(fz, y[keep], exact)
        assert np.array_equal(out[:, -1], (s[keep] < 0).astype(np.uint8)) and not out[:, :-1].any()


@pytest.mark.parametrize("N", [4, 8])
def test_sc_exact_first_decision_is_bitwise_map(N):
    """With the exact f and no frozen position, the first leaf's LLR is the bitwise MAP LLR of u0 with
    every later bit uniform: log sum_{u: u0=0} P(y|x(u)) / sum_{u: u0=1} P(y|x(u)), x(u) = u F^{(x)m}."""
    rng = np.random.default_rng(7)
    fz = np.zeros(N, np.uint8)
    words = np.array(list(itertools.product([0, 1], repeat=N)), np.uint8)
    xs = O.encode(words).astype(np.float64)
    for _ in range(100):
        y = rng.normal(0, 1.5, N).astype(np.float32)
        # log P(y | x) up to a constant: sum_i (1 - 2 x_i) y_i / 2
        ll = ((1 - 2 * xs) * y.astype(np.float64)).sum(axis=1) / 2
        l0 = np.logaddexp.reduce(ll[words[:, 0] == 0])
        l1 = np.logaddexp.reduce(ll[words[:, 0] == 1])
        if abs(l0 - l1) < 1e-6:
            continue
        assert O.sc_decode(fz, y, True)[0] == int(l0 < l1)


# --------------------------------------------------------------------------
# Quantised messages (16-bit saturating integers; a variant for fixed-point hardware)
# --------------------------------------------------------------------------
def test_quantised_n2_hand_trace():
    """(2,1) code, frozen {0}, llr = (1.3, -0.7), F = 2: q = (rint(5.2), rint(-2.8)) = (5, -3),
    L[1] = (32767, 0).  The one PE (A = 15, f = sign sign ((15 min + 8) >> 4)): t = 0 + (-3) = -3,
    g = f(32767, 5) = (75 + 8) >> 4 = 5, L[0] = (f(32767, -3), 0 + 5) = (-(53 >> 4), 5) = (-3, 5),
    R[1] = (f(5, -3), -3 + 5) = (-3, 2); u_1 = HD(2 + 0) = 0.  Both iterations are the same."""
    r = O.decode_q(np.array([1, 0], np.uint8), np.array([1.3, -0.7], np.float32), 2, A=15, F=2, trace=True)
    for t in range(2):
        assert r["R"][t].tolist() == [[5, -3], [-3, 2]]
        assert r["L"][t].tolist() == [[-3, 5], [32767, 0]]
    assert r["u_hat"].tolist() == [0, 0] and r["pe"] == 2 and r["iters"] == 2


@pytest.mark.parametrize("N", [4, 8, 16])
def test_quantised_matches_float_decoder_without_rounding(N):
    """alpha = 1 (A = 16: (16 min + 8) >> 4 = min) on integer channel values with F = 0 and no
    saturation: every message is the float decoder's (the oracle's FP64 sweep), reading the
    saturated side (|q| > 16384, built from the +32767 prior) as the float decoder's +-inf."""
    rng = np.random.default_rng(8)
    fz = O.bec_frozen(N, N // 2)
    for _ in range(40):
        y = rng.integers(-20, 21, N).astype(np.float32)
        q = O.decode_q(fz, y, 6, A=16, F=0, trace=True)
        f = O.decode(fz, y, 6, alpha=1.0, trace=True)
        for key in ("L", "R"):
            qv = q[key].astype(np.float64)
            qv[qv > 16384] = np.inf
            qv[qv < -16384] = -np.inf
            assert np.array_equal(qv, f[key])
        assert np.array_equal(q["u_hat"], f["u_hat"])


@pytest.mark.parametrize("N", [8, 64, 1024])
def test_quantised_noiseless_stops_in_iteration_1(N):
    m = N.bit_length() - 1
    fz = O.bec_frozen(N, N // 2)
    u = I.info_bits(14, np.arange(4), fz)
    llr = I.noiseless_llr(O.encode(u), 2.5)
    uh, it, pe = O.decode_q_batch(fz, llr, 20, 15, 3, O.STOP_GMATRIX)
    assert np.array_equal(uh, u) and np.all(it == 1) and np.all(pe == m * N // 2)


def test_quantised_channel_values():
    """R[0] is clamp(rint(llr 2^F), -32767, 32767), with rint rounding half to even."""
    llr = np.array([0.3125, -0.3125, 1.0625, 2.9, -5000.0, 5000.0, 0.0, -0.0], np.float32)
    r = O.decode_q(np.zeros(8, np.uint8), llr, 1, A=15, F=3, trace=True)
    want = np.clip(np.rint(llr.astype(np.float64) * 8), -32767, 32767).astype(np.int64)
    assert r["R"][0][0].tolist() == want.tolist() == [2, -2, 8, 23, -32767, 32767, 0, 0]


# ---------------------------------------------------------------------------
# Freeze-rule variants of the CSFG check (Sec. III leaves the decided message
# and any reliability condition open); used only for the comparison study.
# ---------------------------------------------------------------------------
def _rule_inputs(N, K, batch, ebn0, seed):
    fz = O.bec_frozen(N, K)
    idx = np.arange(batch)
    u = I.info_bits(seed, idx, fz)
    llr = I.channel_llr(O.encode(u), I.gaussian(seed, idx, N), I.sigma(ebn0, K / N))
    return fz, u, llr


@pytest.mark.parametrize("stop", [0, 1])
def test_rule_r_is_reading_a(stop):
    fz, u, llr = _rule_inputs(256, 128, 60, 2.5, 71)
    a = O.decode_batch(fz, llr, 40, 0.9375, stop, O.FREEZE_CSFG)
    b = O.decode_rule_batch(fz, llr, 40, 0.9375, stop, O.RULE_R)
    for x, y in zip(a[:3], b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("stop", [0, 1])
def test_threshold_rule_limits(stop):
    """|R| >= 0 always holds (the rule is reading A); no |R| reaches +inf (nothing freezes: the
    decode is that without freezing, every PE of every iteration counted)."""
    N, M = 256, 8
    fz, u, llr = _rule_inputs(N, 128, 40, 2.5, 72)
    a = O.decode_rule_batch(fz, llr, 30, 0.9375, stop, O.RULE_R)
    b = O.decode_rule_batch(fz, llr, 30, 0.9375, stop, O.RULE_THRESHOLD, theta=0.0)
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    c = O.decode_rule_batch(fz, llr, 30, 0.9375, stop, O.RULE_THRESHOLD, theta=float("inf"))
    d = O.decode_batch(fz, llr, 30, 0.9375, stop, O.FREEZE_OFF)
    assert np.array_equal(c[0], d[0]) and np.array_equal(c[1], d[1])
    assert np.array_equal(c[2], c[1].astype(np.int64) * M * N // 2)


def test_r_plus_l_rule_first_iteration():
    """In iteration 1 every interior L is 0, so the checks of stages 1..m-1 see R + L = R: the
    first iteration's PE count (which depends only on them) equals rule R's."""
    fz, u, llr = _rule_inputs(512, 256, 50, 2.0, 73)
    a = O.decode_rule_batch(fz, llr, 1, 0.9375, 0, O.RULE_R)
    b = O.decode_rule_batch(fz, llr, 1, 0.9375, 0, O.RULE_R_PLUS_L)
    assert np.array_equal(a[2], b[2])


@pytest.mark.parametrize("N", [16, 64, 1024])
def test_r_plus_l_rule_noiseless(N):
    """Noiseless inputs: R and L agree with the transmitted codeword, every check passes in order,
    and the decode returns the source word."""
    fz = O.bec_frozen(N, N // 2)
    u = I.info_bits(5, np.arange(6), fz)
    llr = I.noiseless_llr(O.encode(u), 3.0)
    uh, it, pe = O.decode_rule_batch(fz, llr, 30, 0.9375, 0, O.RULE_R_PLUS_L)
    assert np.array_equal(uh, u)
    assert np.all(it <= 2)


# ---------------------------------------------------------------------------
# Bit-reversed codeword order (Arikan's G = B_N F^{(x)m}, Sec. II)
# ---------------------------------------------------------------------------
def _bit_reversal_matrix(N):
    m = N.bit_length() - 1
    B = np.zeros((N, N), np.int64)
    for i in range(N):
        B[i, int(format(i, f"0{m}b")[::-1], 2) if m else 0] = 1
    return B


def _F_kron(N):
    F = np.array([[1, 0], [1, 1]], np.int64)
    G = np.array([[1]], np.int64)
    while G.shape[0] < N:
        G = np.kron(G, F)
    return G


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32])
def test_bit_reversal_commutes_with_the_kernel(N):
    """B_N F^{(x)m} = F^{(x)m} B_N over the integers (hence GF(2)), from the matrices' definitions."""
    B, G = _bit_reversal_matrix(N), _F_kron(N)
    assert np.array_equal(B @ G, G @ B)
    assert np.array_equal(B @ B, np.eye(N, dtype=np.int64))


@pytest.mark.parametrize("N", [2, 8, 16, 32])
def test_bit_reversed_encoder_is_arikans_generator(N):
    rng = np.random.default_rng(N)
    u = rng.integers(0, 2, (20, N)).astype(np.uint8)
    want = (u.astype(np.int64) @ (_bit_reversal_matrix(N) @ _F_kron(N))) % 2
    assert np.array_equal(O.encode_bit_reversed(u), want.astype(np.uint8))
    rev = O.bit_reverse_permutation(N)
    assert np.array_equal(rev[rev], np.arange(N))


@pytest.mark.parametrize("N", [8, 64, 1024])
def test_bit_reversed_noiseless_round_trip(N):
    """Noiseless BPSK of the bit-reversed codeword, put back in code order, decodes to u with the
    noiseless invariants of the natural order (G-stop at iteration 1, freeze-only at 2)."""
    fz = O.bec_frozen(N, N // 2)
    u = I.info_bits(9, np.arange(4), fz)
    llr = O.natural_order_llr(I.noiseless_llr(O.encode_bit_reversed(u), 3.0))
    for stop, freeze, iters in ((1, 0, 1), (0, 1, 2), (1, 1, 1)):
        uh, it, pe, _ = O.decode_batch(fz, llr, 30, 0.9375, stop, freeze)
        assert np.array_equal(uh, u) and np.all(it == iters)
