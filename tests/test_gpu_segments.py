"""Persistent decoding of a mixed stream (polarbp_decode_segments, one launch per
length, and polarbp_decode_mixed, one launch for the whole stream): codewords of
lengths 256 .. 4096 and rates 1/4, 1/2, 3/4 at per-codeword Eb/N0 in [1.5, 3.5]
dB, in one call, against the binary32 oracle codeword by codeword."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04979_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

CLASSES = [(256, 64), (256, 128), (256, 192), (1024, 256), (1024, 512), (1024, 768), (4096, 1024), (4096, 2048),
           (4096, 3072)]
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


def class_inputs(N, K, idx, seed):
    fz = O.bec_frozen(N, K)
    u = I.info_bits(seed, idx, fz)
    x = O.encode(u)
    ebn0 = I.uniform(seed, idx, 1.5, 3.5)
    llr = I.channel_llr(x, I.gaussian(seed, idx, N), I.sigma(ebn0, K / N))
    return fz, llr


def run_segments(B, codes, llrs, max_iter, mode, entry="polarbp_decode_segments", **kw):
    segs, outs = [], []
    for code, llr in zip(codes, llrs):
        n = llr.shape[0]
        d = torch.from_numpy(llr).cuda()
        uh = torch.empty((n, code.N), dtype=torch.uint8, device="cuda")
        it = torch.empty(n, dtype=torch.int32, device="cuda")
        pe = torch.empty(n, dtype=torch.int64, device="cuda")
        segs.append((code, d, uh, it, pe))
        outs.append((uh, it, pe))
    getattr(B, entry)(segs, max_iter, ALPHA, *mode, **kw)
    torch.cuda.synchronize()
    return segs, [tuple(t.cpu().numpy() for t in o) for o in outs]


@pytest.mark.parametrize("mode", [(1, 1), (1, 0), (0, 1), (0, 0)])
@pytest.mark.parametrize("mapping,cpc", [(0, 1), (1, 1), (1, 2), (1, 4)])
def test_mixed_segments_match_binary32_oracle(B, mode, mapping, cpc):
    """Per-length persistent launches under every (thread mapping, codewords per block) pair:
    the pipelined mapping (checker warp beside the sweep) with one codeword per block, the
    block mapping with 1, 2 or 4."""
    counts = [40, 40, 40, 24, 24, 24, 6, 6, 6]
    codes, llrs, fzs = [], [], []
    first = 0
    for (N, K), n in zip(CLASSES, counts):
        code = B.polarbp_construct(N, K)
        B.polarbp_set_thread_mapping(code, mapping)
        assert B.polarbp_get_thread_mapping(code) == mapping
        try:
            B.polarbp_set_codewords_per_block(code, cpc)
        except B.PolarBPError:
            pass  # not admissible at this length: keep the default
        fz, llr = class_inputs(N, K, np.arange(first, first + n), 77)
        first += n
        codes.append(code)
        llrs.append(llr)
        fzs.append(fz)
    _, outs = run_segments(B, codes, llrs, 30, mode)
    for fz, llr, (uh, it, pe) in zip(fzs, llrs, outs):
        ouh, oit, ope, _ = O.decode_batch(fz, llr, 30, ALPHA, mode[0], mode[1], fp32=True)
        assert np.array_equal(it, oit) and np.array_equal(pe, ope) and np.array_equal(uh, ouh)


def test_segments_graph_capture_and_replay(B):
    codes, llrs = [], []
    for (N, K), n in zip(CLASSES[::2], [64, 32, 16, 8, 4]):
        codes.append(B.polarbp_construct(N, K))
        llrs.append(class_inputs(N, K, np.arange(n), 5)[1])
    segs, ref = run_segments(B, codes, llrs, 40, (1, 1))
    for _, _, uh, it, pe in segs:
        uh.zero_(), it.zero_(), pe.zero_()
    ws = torch.empty(B.polarbp_decode_segments_workspace(), dtype=torch.uint8, device="cuda")
    B.polarbp_decode_segments(segs, 40, ALPHA, 1, 1, workspace=ws)  # first call outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        B.polarbp_decode_segments(segs, 40, ALPHA, 1, 1, workspace=ws, stream=torch.cuda.current_stream())
    for _ in range(2):
        for _, _, uh, it, pe in segs:
            uh.zero_(), it.zero_(), pe.zero_()
        g.replay()
        torch.cuda.synchronize()
        for (_, _, uh, it, pe), r in zip(segs, ref):
            assert np.array_equal(uh.cpu().numpy(), r[0]) and np.array_equal(it.cpu().numpy(), r[1])
            assert np.array_equal(pe.cpu().numpy(), r[2])


@pytest.mark.parametrize("N", [256, 1024, 4096])
@pytest.mark.parametrize("freeze", [0, 1])
def test_autotune_picks_an_admissible_pair(B, N, freeze):
    code = B.polarbp_construct(N, N // 2)
    cpc = B.polarbp_autotune(code, 40, freeze_mode=freeze)
    mapping = B.polarbp_get_thread_mapping(code)
    assert cpc in (1, 2, 4) and mapping in (B.POLARBP_MAP_PIPELINED, B.POLARBP_MAP_BLOCK)
    if mapping == B.POLARBP_MAP_PIPELINED and freeze == 1:
        assert cpc == 1  # the pipelined mapping holds one codeword per block
    B.polarbp_set_codewords_per_block(code, cpc)


def test_thread_mapping_rejects_unknown_values(B):
    # the defaults: the block mapping below N = 1024, pipelined from there
    assert B.polarbp_get_thread_mapping(B.polarbp_construct(256, 128)) == B.POLARBP_MAP_BLOCK
    assert B.polarbp_get_thread_mapping(B.polarbp_construct(512, 256)) == B.POLARBP_MAP_BLOCK
    assert B.polarbp_get_thread_mapping(B.polarbp_construct(2048, 1024)) == B.POLARBP_MAP_PIPELINED
    code = B.polarbp_construct(1024, 512)
    assert B.polarbp_get_thread_mapping(code) == B.POLARBP_MAP_PIPELINED
    with pytest.raises(B.PolarBPError) as e:
        B.polarbp_set_thread_mapping(code, 2)
    assert e.value.code == B.POLARBP_ERR_ARG
    assert B.polarbp_get_thread_mapping(code) == B.POLARBP_MAP_PIPELINED


@pytest.mark.parametrize("entry", ["polarbp_decode_segments", "polarbp_decode_mixed"])
def test_mixed_full_size_sampled(B, entry):
    """The mixed-stream configuration at full size: 2^20 codewords, each drawing its length
    from {256, 1024, 4096}, its rate from {1/4, 1/2, 3/4} and its Eb/N0 from U[1.5, 3.5] dB,
    decoded with G-matrix stop and freezing (max 60 iterations) in one call with autotuned
    codewords per block.  Bulk inputs come from the device generator; 6 rows of every class
    are overwritten with host-generated inputs and checked against the binary32 oracle."""
    total = 1 << 20
    seed = 1505049792
    idx = np.arange(total)
    cls = I.choice(seed, idx, 9, which=1)
    segs, host_rows, checks = [], [], []
    for k, (N, K) in enumerate(CLASSES):
        members = idx[cls == k]
        code = B.polarbp_construct(N, K)
        B.polarbp_autotune(code, 60)
        ebn0 = torch.from_numpy(I.uniform(seed, members, 1.5, 3.5).astype(np.float32)).cuda()
        _, llr = B.polarbp_awgn_ebn0(code, seed, 0, ebn0, with_u=False)
        rows = np.unique(np.random.default_rng(k).integers(0, len(members), 6))
        fz, hllr = class_inputs(N, K, members[rows], seed + 1)
        llr[torch.from_numpy(rows).cuda()] = torch.from_numpy(hllr).cuda()
        n = len(members)
        uh = torch.empty((n, N), dtype=torch.uint8, device="cuda")
        it = torch.empty(n, dtype=torch.int32, device="cuda")
        pe = torch.empty(n, dtype=torch.int64, device="cuda")
        segs.append((code, llr, uh, it, pe))
        checks.append((fz, hllr, rows))
    getattr(B, entry)(segs, 60, ALPHA, 1, 1)
    torch.cuda.synchronize()
    for (code, llr, uh, it, pe), (fz, hllr, rows) in zip(segs, checks):
        sel = torch.from_numpy(rows).cuda()
        ouh, oit, ope, _ = O.decode_batch(fz, hllr, 60, ALPHA, 1, 1, fp32=True)
        assert np.array_equal(uh[sel].cpu().numpy(), ouh)
        assert np.array_equal(it[sel].cpu().numpy(), oit)
        assert np.array_equal(pe[sel].cpu().numpy(), ope)


@pytest.mark.parametrize("entry", ["polarbp_decode_segments", "polarbp_decode_mixed"])
def test_nonfinite_input_reported_on_its_own_code(B, entry):
    """Two runs of the same length with different codes: a NaN in the second run's LLRs sets
    the status word of the second code only."""
    c1, c2 = B.polarbp_construct(1024, 512), B.polarbp_construct(1024, 256)
    l1 = class_inputs(1024, 512, np.arange(8), 9)[1]
    l2 = class_inputs(1024, 256, np.arange(8, 16), 9)[1]
    l2[3, 17] = np.nan
    assert B.polarbp_get_status(c1) == B.POLARBP_OK and B.polarbp_get_status(c2) == B.POLARBP_OK
    run_segments(B, [c1, c2], [l1, l2], 20, (1, 1), entry)
    assert B.polarbp_get_status(c1) == B.POLARBP_OK
    assert B.polarbp_get_status(c2) == B.POLARBP_ERR_NONFINITE


# --- one launch for the whole stream (polarbp_decode_mixed) -----------------------------------

ALL_LENGTHS = [(256, 64), (256, 192), (512, 128), (512, 384), (1024, 512), (1024, 768), (2048, 1024),
               (2048, 512), (4096, 2048), (4096, 3072)]


def mixed_case(B, classes, counts, seed, bitrev=()):
    codes, llrs, fzs = [], [], []
    first = 0
    for k, ((N, K), n) in enumerate(zip(classes, counts)):
        code = B.polarbp_construct(N, K)
        fz = O.bec_frozen(N, K)
        idx = np.arange(first, first + n)
        first += n
        if k in bitrev:
            code.set_bit_reversed(True)
            u = I.info_bits(seed, idx, fz)
            ebn0 = I.uniform(seed, idx, 1.5, 3.5)
            llr = I.channel_llr(O.encode_bit_reversed(u), I.gaussian(seed, idx, N), I.sigma(ebn0, K / N))
            llr = np.ascontiguousarray(llr, dtype=np.float32)
        else:
            llr = class_inputs(N, K, idx, seed)[1]
        codes.append(code)
        llrs.append(llr)
        fzs.append((fz, k in bitrev))
    return codes, llrs, fzs


def check_against_oracle(fzs, llrs, outs, max_iter, mode):
    for (fz, rev), llr, (uh, it, pe) in zip(fzs, llrs, outs):
        ollr = O.natural_order_llr(llr) if rev else llr
        ouh, oit, ope, _ = O.decode_batch(fz, ollr, max_iter, ALPHA, mode[0], mode[1], fp32=True)
        assert np.array_equal(it, oit) and np.array_equal(pe, ope) and np.array_equal(uh, ouh)


@pytest.mark.parametrize("mode", [(1, 1), (1, 0), (0, 1), (0, 0)])
def test_one_launch_all_lengths_match_binary32_oracle(B, mode):
    """Every length 256 .. 4096 in one launch (blocks of 512 threads splitting down to warps),
    two rates per length, one run in bit-reversed order."""
    counts = [70, 50, 40, 30, 24, 20, 10, 9, 5, 4]
    codes, llrs, fzs = mixed_case(B, ALL_LENGTHS, counts, 31, bitrev=(3,))
    _, outs = run_segments(B, codes, llrs, 30, mode, "polarbp_decode_mixed")
    check_against_oracle(fzs, llrs, outs, 30, mode)


@pytest.mark.parametrize("classes,counts", [
    ([(256, 128)], [300]),                                   # a single length: blocks of one warp
    ([(512, 256), (256, 128)], [90, 200]),                   # longest 512
    ([(1024, 512), (256, 64), (256, 192)], [60, 0, 150]),    # a run with no codewords; skipped lengths
    ([(2048, 1024), (512, 256)], [20, 64]),                  # longest 2048, no 1024 or 256
    ([(4096, 2048), (256, 128)], [3, 500]),                  # 512-thread blocks down to warps
])
def test_one_launch_stream_shapes(B, classes, counts):
    codes, llrs, fzs = mixed_case(B, classes, counts, 47)
    _, outs = run_segments(B, codes, llrs, 40, (1, 1), "polarbp_decode_mixed")
    check_against_oracle(fzs, llrs, outs, 40, (1, 1))


def test_one_launch_equals_per_length_launches(B):
    """The two mixed-stream entry points give the same bits, iteration and PE counts on a
    stream larger than one wave of blocks."""
    counts = [3000, 2000, 1500, 1200, 900, 700, 400, 300, 150, 120]
    codes, llrs, _ = mixed_case(B, ALL_LENGTHS, counts, 53)
    _, a = run_segments(B, codes, llrs, 60, (1, 1), "polarbp_decode_segments")
    _, b = run_segments(B, codes, llrs, 60, (1, 1), "polarbp_decode_mixed")
    for x, y in zip(a, b):
        for u, v in zip(x, y):
            assert np.array_equal(u, v)


def test_one_launch_graph_capture_and_replay(B):
    codes, llrs, _ = mixed_case(B, ALL_LENGTHS[::2], [64, 40, 32, 16, 8], 59)
    segs, ref = run_segments(B, codes, llrs, 40, (1, 1), "polarbp_decode_mixed")
    ws = torch.empty(B.polarbp_decode_segments_workspace(), dtype=torch.uint8, device="cuda")
    B.polarbp_decode_mixed(segs, 40, ALPHA, 1, 1, workspace=ws)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        B.polarbp_decode_mixed(segs, 40, ALPHA, 1, 1, workspace=ws, stream=torch.cuda.current_stream())
    for _ in range(2):
        for _, _, uh, it, pe in segs:
            uh.zero_(), it.zero_(), pe.zero_()
        g.replay()
        torch.cuda.synchronize()
        for (_, _, uh, it, pe), r in zip(segs, ref):
            assert np.array_equal(uh.cpu().numpy(), r[0]) and np.array_equal(it.cpu().numpy(), r[1])
            assert np.array_equal(pe.cpu().numpy(), r[2])


def test_one_launch_rejects_unsupported_lengths(B):
    code = B.polarbp_construct(128, 64)
    d = torch.zeros((4, 128), dtype=torch.float32, device="cuda")
    uh = torch.empty((4, 128), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.PolarBPError) as e:
        B.polarbp_decode_mixed([(code, d, uh, None, None)], 10)
    assert e.value.code == B.POLARBP_ERR_UNSUPPORTED
