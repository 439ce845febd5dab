"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Decisions (hard decisions, freeze events, iteration counts, PE-update counts)
are compared bit-exactly with the oracle run in binary32 arithmetic, the
kernel's precision; message planes are compared bit-exactly with the same
oracle on every entry outside covered CSFGs.  Against the FP64 oracle the
decisions must agree on every codeword that the oracle decides alike in FP64
and in binary32 (the others are flagged and counted), and messages must meet
1e-4 relative or 1e-5 absolute (every entry of the first ten iterations, 99.9%
of all entries).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04979_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MODES = [(0, 0), (1, 0), (0, 1), (1, 1)]  # (stop_mode, freeze_mode)
MODES_B = [(0, 2), (1, 2)]  # freezing under reading B (checks continue along a stage while they pass)
ALPHA = 0.9375


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_04979_gb300 import build
    build.build()
    from paper_1505_04979_gb300 import binding
    torch.cuda.set_device(0)
    return binding


def host_inputs(N, K, batch, ebn0, seed, first=0):
    fz = O.bec_frozen(N, K)
    idx = np.arange(first, first + batch)
    u = I.info_bits(seed, idx, fz)
    x = O.encode(u)
    llr = I.channel_llr(x, I.gaussian(seed, idx, N), I.sigma(ebn0, K / N))
    return fz, u, x, llr


def gpu_decode(B, code, llr, max_iter, stop, freeze, scale=ALPHA):
    d = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    uh, it, pe = B.polarbp_decode(code, d, max_iter, scale, stop, freeze)
    torch.cuda.synchronize()
    return uh.cpu().numpy(), it.cpu().numpy(), pe.cpu().numpy()


def thr(P, M, c):
    return 0 if c <= 0 else (P >> (M - c)) << (M - c)


def live_masks(P, M, N):
    """Entries outside covered CSFGs at the end of an iteration with covered prefix P."""
    i = np.arange(N)
    Rm = np.stack([i >= thr(P, M, c) for c in range(M + 1)])
    Rm[0] = True
    Lm = np.stack([i >= thr(P, M, c - 1) for c in range(M + 1)])
    Lm[0] = True
    return Lm, Rm


# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [2, 8, 64, 1024, 4096, 32768])
def test_encode_matches_oracle(B, N):
    code = B.polarbp_construct(N, N // 2)
    rng = np.random.default_rng(N)
    u = rng.integers(0, 2, (7, N)).astype(np.uint8)
    x = B.polarbp_encode(code, torch.from_numpy(u).cuda())
    assert np.array_equal(x.cpu().numpy(), O.encode(u))


@pytest.mark.parametrize("N,K", [(64, 32), (1024, 512), (4096, 1024)])
def test_device_generator_matches_host_generator(B, N, K):
    code = B.polarbp_construct(N, K)
    u, llr = B.polarbp_awgn(code, 77, 1000, 16, 2.0)
    fz, hu, hx, hllr = host_inputs(N, K, 16, 2.0, 77, first=1000)
    assert np.array_equal(u.cpu().numpy(), hu)
    g = llr.cpu().numpy()
    assert np.all(np.abs(g - hllr) <= 1e-4 * np.maximum(1.0, np.abs(hllr)))


@pytest.mark.parametrize("N", [2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("mode", MODES + MODES_B)
def test_decode_matches_binary32_oracle(B, N, mode):
    K = N // 2
    batch = 96 if N <= 1024 else 24
    max_iter = 40
    code = B.polarbp_construct(N, K)
    for ebn0 in (1.5, 3.0):
        fz, u, x, llr = host_inputs(N, K, batch, ebn0, 1000 + N)
        uh, it, pe = gpu_decode(B, code, llr, max_iter, *mode)
        ouh, oit, ope, _ = O.decode_batch(fz, llr, max_iter, ALPHA, mode[0], mode[1], fp32=True)
        assert np.array_equal(it, oit)
        assert np.array_equal(pe, ope)
        assert np.array_equal(uh, ouh)


@pytest.mark.parametrize("N", [256, 512, 1024, 2048, 4096])
@pytest.mark.parametrize("mode", [(1, 1), (0, 1)])
@pytest.mark.parametrize("mapping", [0, 1])
def test_both_thread_mappings_match_binary32_oracle(B, N, mode, mapping):
    """Freezing at N = 256 .. 4096 under each thread mapping (pipelined: a checker warp beside
    the sweep; block: the sweep warps take turns with the checks), whatever the length's
    default: the same bits and counts."""
    K = N // 2
    code = B.polarbp_construct(N, K)
    B.polarbp_set_thread_mapping(code, mapping)
    fz, u, x, llr = host_inputs(N, K, 64 if N < 4096 else 16, 2.5, 3000 + N)
    uh, it, pe = gpu_decode(B, code, llr, 40, *mode)
    ouh, oit, ope, _ = O.decode_batch(fz, llr, 40, ALPHA, mode[0], mode[1], fp32=True)
    assert np.array_equal(it, oit) and np.array_equal(pe, ope) and np.array_equal(uh, ouh)


@pytest.mark.parametrize("N", [8, 16, 64, 128, 512, 1024, 4096])
@pytest.mark.parametrize("mode", MODES + MODES_B)
def test_message_planes_match_binary32_oracle(B, N, mode):
    K = N // 2
    M = N.bit_length() - 1
    batch = 6 if N >= 1024 else 12
    max_iter = 25
    code = B.polarbp_construct(N, K)
    fz, u, x, llr = host_inputs(N, K, batch, 2.0, 500 + N)
    d = torch.from_numpy(llr).cuda()
    uh, it, pe, tL, tR, tP = B.polarbp_decode_trace(code, d, max_iter, ALPHA, *mode)
    torch.cuda.synchronize()
    tL, tR, tP, it = tL.cpu().numpy(), tR.cpu().numpy(), tP.cpu().numpy(), it.cpu().numpy()
    for c in range(batch):
        o = O.decode(fz, llr[c], max_iter, ALPHA, mode[0], mode[1], fp32=True, trace=True)
        assert it[c] == o["iters"]
        assert np.array_equal(tP[c, :o["iters"]], o["P"])
        for t in range(o["iters"]):
            Lm, Rm = live_masks(int(o["P"][t]), M, N)
            gL = tL[c, t].astype(np.float64)
            gR = tR[c, t].astype(np.float64)
            assert np.array_equal(gL[Lm], o["L"][t][Lm]), (c, t)
            assert np.array_equal(gR[Rm], o["R"][t][Rm]), (c, t)


def test_config_small_code_full_message_parity(B):
    """(64,32), Eb/N0 2.5 dB, 1000 codewords, alpha 0.9375, 40 fixed iterations: every
    message of every iteration, bit for bit against the binary32 oracle."""
    N, K, batch, max_iter = 64, 32, 1000, 40
    code = B.polarbp_construct(N, K)
    fz, u, x, llr = host_inputs(N, K, batch, 2.5, I.DEFAULT_SEED)
    d = torch.from_numpy(llr).cuda()
    uh, it, pe, tL, tR, tP = B.polarbp_decode_trace(code, d, max_iter, ALPHA, 0, 0)
    torch.cuda.synchronize()
    tL, tR = tL.cpu().numpy(), tR.cpu().numpy()
    uh = uh.cpu().numpy()
    for c in range(batch):
        o = O.decode(fz, llr[c], max_iter, ALPHA, 0, 0, fp32=True, trace=True)
        assert np.array_equal(tL[c].astype(np.float64), o["L"])
        assert np.array_equal(tR[c].astype(np.float64), o["R"])
        assert np.array_equal(uh[c], o["u_hat"])


def _oracle_precisions_agree(a, b):
    return a["iters"] == b["iters"] and np.array_equal(a["u_hat"], b["u_hat"]) and a["pe"] == b["pe"]


@pytest.mark.parametrize("mode", MODES)
def test_fp64_decisions_agree_where_precision_does_not_decide(B, mode):
    """Against the FP64 oracle, the GPU must take every decision the FP64 oracle takes on
    each codeword whose FP64 and binary32 oracle runs decide alike; the other codewords
    (precision decides them) are counted and reported as flagged."""
    N, K, batch = 1024, 512, 256
    code = B.polarbp_construct(N, K)
    fz, u, x, llr = host_inputs(N, K, batch, 3.0, 4242)
    uh, it, pe = gpu_decode(B, code, llr, 60, *mode)
    d64 = O.decode_batch(fz, llr, 60, ALPHA, mode[0], mode[1])
    d32 = O.decode_batch(fz, llr, 60, ALPHA, mode[0], mode[1], fp32=True)
    same = (d64[1] == d32[1]) & (d64[2] == d32[2]) & np.all(d64[0] == d32[0], axis=1)
    flagged = int((~same).sum())
    print(f"mode {mode}: {flagged} of {batch} codewords flagged (binary32 and FP64 decide differently)")
    assert flagged <= batch // 10
    assert np.array_equal(uh[same], d64[0][same])
    assert np.array_equal(it[same], d64[1][same])
    assert np.array_equal(pe[same], d64[2][same])


@pytest.mark.parametrize("N,ebn0,mode,max_iter", [(64, 2.5, (0, 0), 40), (1024, 3.0, (1, 1), 60),
                                                  (1024, 3.0, (0, 0), 40), (256, 3.0, (0, 1), 40)])
def test_fp64_messages_within_tolerance(B, N, ebn0, mode, max_iter):
    """Messages against the FP64 oracle: |gpu - fp64| <= 1e-5 or <= 1e-4 |fp64| on live entries.
    Binary32 rounding accumulates over iterations, so the bound is required on every entry of
    the first ten iterations and on 99.9% of the entries over the whole run (codewords the two
    precisions decide differently are left out)."""
    K = N // 2
    M = N.bit_length() - 1
    batch = 8 if N >= 1024 else 24
    code = B.polarbp_construct(N, K)
    fz, u, x, llr = host_inputs(N, K, batch, ebn0, 77 + N)
    d = torch.from_numpy(llr).cuda()
    _, it, _, tL, tR, tP = B.polarbp_decode_trace(code, d, max_iter, ALPHA, *mode)
    torch.cuda.synchronize()
    tL, tR = tL.cpu().numpy(), tR.cpu().numpy()
    hit = tot = hit10 = tot10 = 0
    for c in range(batch):
        o = O.decode(fz, llr[c], max_iter, ALPHA, mode[0], mode[1], trace=True)
        o32 = O.decode(fz, llr[c], max_iter, ALPHA, mode[0], mode[1], fp32=True)
        if not _oracle_precisions_agree(o, o32):
            continue
        for t in range(o["iters"]):
            Lm, Rm = live_masks(int(o["P"][t]), M, N)
            for g, ref, mask in ((tL[c, t], o["L"][t], Lm), (tR[c, t], o["R"][t], Rm)):
                gv = g.astype(np.float64)[mask]
                rv = ref[mask]
                inf = ~np.isfinite(rv)
                assert np.array_equal(gv[inf], rv[inf])
                dd = np.abs(gv[~inf] - rv[~inf])
                ok = (dd <= 1e-5) | (dd <= 1e-4 * np.abs(rv[~inf]))
                hit += int(ok.sum())
                tot += ok.size
                if t < 10:
                    hit10 += int(ok.sum())
                    tot10 += ok.size
    print(f"N={N} {ebn0} dB mode {mode}: tolerance met on {hit}/{tot} entries ({hit / tot:.6f})")
    assert tot > 0 and hit10 == tot10
    assert hit >= 0.999 * tot


@pytest.mark.parametrize("N", [8, 64, 1024, 4096])
def test_noiseless_invariants(B, N):
    K = N // 2
    M = N.bit_length() - 1
    code = B.polarbp_construct(N, K)
    fz = O.bec_frozen(N, K)
    u = I.info_bits(3, np.arange(5), fz)
    llr = I.noiseless_llr(O.encode(u), 3.0)
    for mode, iters, pe in (((1, 0), 1, M * N // 2), ((0, 1), 2, 3 * N // 2 - 1), ((1, 1), 1, N - 1),
                            ((0, 0), 7, 7 * M * N // 2)):
        uh, it, p = gpu_decode(B, code, llr, 7 if mode == (0, 0) else 30, *mode)
        assert np.all(it == iters) and np.all(p == pe)
        assert np.array_equal(uh, u)


@pytest.mark.parametrize("N,K", [(16, 0), (16, 16), (64, 1), (1024, 1023)])
@pytest.mark.parametrize("mode", MODES)
def test_degenerate_rates(B, N, K, mode):
    code = B.polarbp_construct(N, K)
    fz = O.bec_frozen(N, K)
    rng = np.random.default_rng(K)
    llr = rng.normal(1.0, 2.0, (20, N)).astype(np.float32)
    uh, it, pe = gpu_decode(B, code, llr, 20, *mode)
    ouh, oit, ope, _ = O.decode_batch(fz, llr, 20, ALPHA, mode[0], mode[1], fp32=True)
    assert np.array_equal(uh, ouh) and np.array_equal(it, oit) and np.array_equal(pe, ope)


@pytest.mark.parametrize("max_iter,scale", [(1, ALPHA), (3, 1.0), (100, 0.75)])
def test_iteration_cap_and_scale(B, max_iter, scale):
    N, K = 256, 128
    code = B.polarbp_construct(N, K)
    fz, u, x, llr = host_inputs(N, K, 50, 2.0, 9)
    for mode in MODES:
        uh, it, pe = gpu_decode(B, code, llr, max_iter, *mode, scale=scale)
        ouh, oit, ope, _ = O.decode_batch(fz, llr, max_iter, scale, mode[0], mode[1], fp32=True)
        assert np.array_equal(uh, ouh) and np.array_equal(it, oit) and np.array_equal(pe, ope)


def test_empty_batch_and_errors(B):
    code = B.polarbp_construct(64, 32)
    empty = torch.empty((0, 64), dtype=torch.float32, device="cuda")
    uh, it, pe = B.polarbp_decode(code, empty, 10)
    assert uh.shape == (0, 64)
    llr = torch.zeros((2, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(B.PolarBPError):
        B.polarbp_decode(code, llr, 0)
    with pytest.raises(B.PolarBPError):
        B.polarbp_decode(code, llr, 5, scale=float("nan"))
    with pytest.raises(B.PolarBPError):
        B.polarbp_decode(code, llr, 5, stop_mode=7)
    # long codes run on thread-block clusters, but not in the persistent mixed-length launch
    big = B.polarbp_construct(8192, 4096)
    z = torch.zeros((1, 8192), dtype=torch.float32, device="cuda")
    seg = (big, z, torch.empty((1, 8192), dtype=torch.uint8, device="cuda"),
           torch.empty(1, dtype=torch.int32, device="cuda"), torch.empty(1, dtype=torch.int64, device="cuda"))
    with pytest.raises(B.PolarBPError) as e:
        B.polarbp_decode_segments([seg], 5)
    assert e.value.code == B.POLARBP_ERR_UNSUPPORTED


def test_nonfinite_llr_sets_status(B):
    code = B.polarbp_construct(64, 32)
    llr = torch.ones((3, 64), dtype=torch.float32, device="cuda")
    assert B.polarbp_get_status(code) == B.POLARBP_OK
    B.polarbp_decode(code, llr, 5)
    assert B.polarbp_get_status(code) == B.POLARBP_OK
    llr[1, 7] = float("nan")
    B.polarbp_decode(code, llr, 5)
    assert B.polarbp_get_status(code) == B.POLARBP_ERR_NONFINITE
    assert B.polarbp_get_status(code) == B.POLARBP_OK


def test_host_entry_point_matches_device_entry_point(B):
    N, K, batch = 1024, 512, 300
    code = B.polarbp_construct(N, K)
    fz, u, x, llr = host_inputs(N, K, batch, 2.5, 31)
    ws = torch.empty(B.polarbp_decode_host_workspace(code, batch), dtype=torch.uint8, device="cuda")
    h_llr = torch.from_numpy(llr).pin_memory()
    h_u = torch.empty((batch, N), dtype=torch.uint8).pin_memory()
    h_it = torch.empty(batch, dtype=torch.int32).pin_memory()
    h_pe = torch.empty(batch, dtype=torch.int64).pin_memory()
    B.polarbp_decode_host(code, h_llr, 60, ALPHA, 1, 1, h_u, h_it, h_pe, ws)
    uh, it, pe = gpu_decode(B, code, llr, 60, 1, 1)
    assert np.array_equal(h_u.numpy(), uh) and np.array_equal(h_it.numpy(), it) and np.array_equal(h_pe.numpy(), pe)


def test_host_entry_point_pipelined(B):
    """A batch of more than two chunks of 64 MiB of LLRs runs as the copy/decode pipeline on the
    handle's streams, with a ragged last chunk; the results equal the device entry point's on the
    same LLRs, with and without the iteration and PE-count outputs, and repeat on a second call."""
    N, K = 1024, 512
    cb = (64 << 20) // (4 * N)
    batch = 2 * cb + 1234
    code = B.polarbp_construct(N, K)
    _, llr = B.polarbp_awgn(code, 17, 0, batch, 2.5, with_u=False)
    uh, it, pe = B.polarbp_decode(code, llr, 60, ALPHA, 1, 1)
    torch.cuda.synchronize()
    ws = torch.empty(B.polarbp_decode_host_workspace(code, batch), dtype=torch.uint8, device="cuda")
    h_llr = llr.cpu().pin_memory()
    h_u = torch.empty((batch, N), dtype=torch.uint8).pin_memory()
    h_it = torch.empty(batch, dtype=torch.int32).pin_memory()
    h_pe = torch.empty(batch, dtype=torch.int64).pin_memory()
    for _ in range(2):
        h_u.fill_(7)
        h_it.fill_(-1)
        h_pe.fill_(-1)
        B.polarbp_decode_host(code, h_llr, 60, ALPHA, 1, 1, h_u, h_it, h_pe, ws)
        assert torch.equal(h_u, uh.cpu()) and torch.equal(h_it, it.cpu()) and torch.equal(h_pe, pe.cpu())
    h_u.fill_(7)
    B.polarbp_decode_host(code, h_llr, 60, ALPHA, 1, 1, h_u, None, None, ws)
    assert torch.equal(h_u, uh.cpu())


def test_full_size_launch_sampled(B):
    """The benchmark's launch: (1024,512), 2^20 codewords in one launch, G-matrix stop and
    freezing, 60 iterations.  Bulk inputs come from the device generator; 64 rows at
    scattered positions are overwritten with host-generated inputs, and those rows are
    checked against the binary32 oracle."""
    N, K, batch = 1024, 512, 1 << 20
    code = B.polarbp_construct(N, K)
    _, llr = B.polarbp_awgn(code, 5, 0, batch, 3.0, with_u=False)
    rows = np.unique(np.random.default_rng(0).integers(0, batch, 64))
    rows[0], rows[-1] = 0, batch - 1
    fz, u, x, hllr = host_inputs(N, K, len(rows), 3.0, 6)
    llr[torch.from_numpy(rows).cuda()] = torch.from_numpy(hllr).cuda()
    for mode in ((1, 1), (0, 0)):
        uh, it, pe = B.polarbp_decode(code, llr, 60, ALPHA, *mode)
        torch.cuda.synchronize()
        sel = torch.from_numpy(rows).cuda()
        ouh, oit, ope, _ = O.decode_batch(fz, hllr, 60, ALPHA, mode[0], mode[1], fp32=True)
        assert np.array_equal(uh[sel].cpu().numpy(), ouh)
        assert np.array_equal(it[sel].cpu().numpy(), oit)
        assert np.array_equal(pe[sel].cpu().numpy(), ope)
        if mode == (0, 0):
            assert int(it.min()) == 60 and int(it.max()) == 60


def test_n8_freeze_hand_trace(B):
    """The (8,4) freezing example worked by hand (tests/golden/n8_freeze_hand_trace.json): every
    value is a small integer, exact in binary32, so the kernel must reproduce it exactly."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "n8_freeze_hand_trace.json")))
    code = B.polarbp_construct(8, 4)
    assert np.array_equal(code.frozen_mask(), np.array(g["frozen"], np.uint8))
    d = torch.tensor([g["llr"]], dtype=torch.float32, device="cuda")
    for stop in (0, 1):
        uh, it, pe, tL, tR, tP = B.polarbp_decode_trace(code, d, g["max_iter"], g["alpha"], stop, 1)
        torch.cuda.synchronize()
        assert int(it[0]) == g["max_iter"]
        assert int(pe[0]) == sum(x["pe"] for x in g["iterations"])
        assert np.array_equal(uh.cpu().numpy()[0], np.array(g["u_hat"], np.uint8))
        tL, tR, tP = tL.cpu().numpy(), tR.cpu().numpy(), tP.cpu().numpy()
        for t, x in enumerate(g["iterations"]):
            assert tP[0, t] == x["P"]
            for plane, arr in (("R", tR), ("L", tL)):
                for c, vals in x[plane].items():
                    for i, v in vals.items():
                        want = np.inf if v == "inf" else float(v)
                        assert arr[0, t, int(c), int(i)] == want, (stop, t, plane, c, i)


def test_reading_b_limits(B):
    """Reading B runs on the one-block kernels only (N <= 4096)."""
    code = B.polarbp_construct(8192, 4096)
    llr = torch.zeros((1, 8192), dtype=torch.float32, device="cuda")
    with pytest.raises(B.PolarBPError) as e:
        B.polarbp_decode(code, llr, 5, ALPHA, 1, B.POLARBP_FREEZE_CSFG_MULTI)
    assert e.value.code == B.POLARBP_ERR_UNSUPPORTED
    with pytest.raises(B.PolarBPError) as e:
        B.polarbp_decode(B.polarbp_construct(64, 32), torch.zeros((1, 64), dtype=torch.float32, device="cuda"),
                         5, ALPHA, 1, 3)
    assert e.value.code == B.POLARBP_ERR_ARG
