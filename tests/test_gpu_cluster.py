"""GPU parity of the long-code decoder (N = 8192, 16384, 32768: one codeword per
thread-block cluster of 2, 4 or 8 blocks) against the CPU oracle.

Decisions, iteration counts and PE-update counts are compared bit-exactly with
the oracle run in binary32 arithmetic, at the sizes and signal-to-noise ratios
of the long-code workload (K = N/2, Eb/N0 2.0 / 2.5 / 3.0 dB, at most 100
iterations), plus 4 dB where freezing covers the whole code, which exercises
freezes of CSFGs that span blocks and the completion of enclosing CSFGs across
block boundaries.  Message planes are compared bit-exactly on every entry
outside covered CSFGs.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04979_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

MODES = [(0, 0), (1, 0), (0, 1), (1, 1)]  # (stop_mode, freeze_mode)
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


def live_masks(P, M, N):
    """Entries outside covered CSFGs at the end of an iteration with covered prefix P."""
    def thr(c):
        return 0 if c <= 0 else (P >> (M - c)) << (M - c)
    i = np.arange(N)
    Rm = np.stack([i >= thr(c) for c in range(M + 1)])
    Rm[0] = True
    Lm = np.stack([i >= thr(c - 1) for c in range(M + 1)])
    Lm[0] = True
    return Lm, Rm


@pytest.mark.parametrize("N", [8192, 16384, 32768])
@pytest.mark.parametrize("mode", MODES)
def test_cluster_decode_matches_binary32_oracle(B, N, mode):
    K = N // 2
    batch = 8
    code = B.polarbp_construct(N, K)
    points = (2.0, 2.5, 3.0) + ((4.0,) if mode[1] else ())
    for ebn0 in points:
        fz, u, x, llr = host_inputs(N, K, batch, ebn0, 2000 + N + int(10 * ebn0))
        uh, it, pe = gpu_decode(B, code, llr, 100, *mode)
        ouh, oit, ope, _ = O.decode_batch(fz, llr, 100, ALPHA, mode[0], mode[1], fp32=True)
        assert np.array_equal(it, oit), (ebn0, it, oit)
        assert np.array_equal(pe, ope), (ebn0, pe, ope)
        assert np.array_equal(uh, ouh), ebn0


def test_cluster_freezing_reaches_full_coverage(B):
    """Freeze-only decoding at 4 dB ends with every position covered, so the last CSFGs
    frozen span blocks: the iteration counts and PE counts pin those events."""
    N, K = 16384, 8192
    code = B.polarbp_construct(N, K)
    fz, u, x, llr = host_inputs(N, K, 8, 4.0, 31)
    uh, it, pe = gpu_decode(B, code, llr, 200, 0, 1)
    ouh, oit, ope, _ = O.decode_batch(fz, llr, 200, ALPHA, 0, 1, fp32=True)
    assert np.all(oit < 200)  # the oracle covered everything before the cap
    assert np.array_equal(it, oit) and np.array_equal(pe, ope) and np.array_equal(uh, ouh)


@pytest.mark.parametrize("N,mode,ebn0,max_iter", [(8192, (0, 1), 4.0, 100), (8192, (1, 1), 3.0, 60),
                                                  (16384, (0, 1), 3.5, 40), (32768, (1, 1), 2.5, 20),
                                                  (32768, (0, 0), 2.0, 6)])
def test_cluster_message_planes_match_binary32_oracle(B, N, mode, ebn0, max_iter):
    K = N // 2
    M = N.bit_length() - 1
    code = B.polarbp_construct(N, K)
    fz, u, x, llr = host_inputs(N, K, 1, ebn0, 700 + N)
    d = torch.from_numpy(llr).cuda()
    uh, it, pe, tL, tR, tP = B.polarbp_decode_trace(code, d, max_iter, ALPHA, *mode)
    torch.cuda.synchronize()
    it, tP = it.cpu().numpy(), tP.cpu().numpy()
    o = O.decode(fz, llr[0], max_iter, ALPHA, mode[0], mode[1], fp32=True, trace=True)
    assert it[0] == o["iters"]
    assert np.array_equal(tP[0, :o["iters"]], o["P"])
    assert np.array_equal(uh.cpu().numpy()[0], o["u_hat"])
    for t in range(o["iters"]):
        Lm, Rm = live_masks(int(o["P"][t]), M, N)
        gL = tL[0, t].cpu().numpy().astype(np.float64)
        gR = tR[0, t].cpu().numpy().astype(np.float64)
        assert np.array_equal(gL[Lm], o["L"][t][Lm]), t
        assert np.array_equal(gR[Rm], o["R"][t][Rm]), t


@pytest.mark.parametrize("N", [8192, 16384, 32768])
def test_cluster_noiseless_invariants(B, N):
    K = N // 2
    M = N.bit_length() - 1
    code = B.polarbp_construct(N, K)
    fz = O.bec_frozen(N, K)
    u = I.info_bits(3, np.arange(3), fz)
    llr = I.noiseless_llr(O.encode(u), 3.0)
    for mode, iters, pe in (((1, 0), 1, M * N // 2), ((0, 1), 2, 3 * N // 2 - 1), ((1, 1), 1, N - 1),
                            ((0, 0), 3, 3 * M * N // 2)):
        uh, it, p = gpu_decode(B, code, llr, 3 if mode == (0, 0) else 30, *mode)
        assert np.all(it == iters) and np.all(p == pe), (mode, it, p)
        assert np.array_equal(uh, u)


@pytest.mark.parametrize("K", [0, 1, 8191, 8192])
@pytest.mark.parametrize("mode", MODES)
def test_cluster_degenerate_rates(B, K, mode):
    N = 8192
    code = B.polarbp_construct(N, K)
    fz = O.bec_frozen(N, K)
    rng = np.random.default_rng(K)
    llr = rng.normal(1.0, 2.0, (4, N)).astype(np.float32)
    uh, it, pe = gpu_decode(B, code, llr, 20, *mode)
    ouh, oit, ope, _ = O.decode_batch(fz, llr, 20, ALPHA, mode[0], mode[1], fp32=True)
    assert np.array_equal(uh, ouh) and np.array_equal(it, oit) and np.array_equal(pe, ope)


def test_cluster_device_generator_and_full_batch_sampled(B):
    """The long-code workload's launch: a 2048-codeword batch of N = 32768 at 2.5 dB from the
    device generator, G-matrix stop and freezing, 100 iterations; sampled codewords against
    the binary32 oracle, recomputed on the host from the same seeds."""
    N, K, batch = 32768, 16384, 2048
    code = B.polarbp_construct(N, K)
    u, llr = B.polarbp_awgn(code, I.DEFAULT_SEED, 0, batch, 2.5)
    uh, it, pe = B.polarbp_decode(code, llr, 100, ALPHA, 1, 1)
    torch.cuda.synchronize()
    uh, it, pe = uh.cpu().numpy(), it.cpu().numpy(), pe.cpu().numpy()
    sample = np.array([0, 1, 777, 1024, 2047])
    hllr = llr.cpu().numpy()[sample]
    fz = O.bec_frozen(N, K)
    ouh, oit, ope, _ = O.decode_batch(fz, hllr, 100, ALPHA, 1, 1, fp32=True)
    assert np.array_equal(uh[sample], ouh) and np.array_equal(it[sample], oit) and np.array_equal(pe[sample], ope)
    assert np.all((it >= 1) & (it <= 100))
    assert np.all(uh[:, fz.astype(bool)] == 0)
    fer = float(np.mean(np.any(uh != u.cpu().numpy(), axis=1)))
    assert fer < 0.5
