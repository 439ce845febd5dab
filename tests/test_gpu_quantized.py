"""GPU parity of the quantised-message decoder (polarbp_decode_quantized, through the C ABI)
against the CPU oracle's integer decoder: decisions, iteration counts, PE counts and every
integer message plane compared exactly."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04979_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_04979_gb300 import build
    build.build()
    from paper_1505_04979_gb300 import binding
    torch.cuda.set_device(0)
    return binding


def host_inputs(N, K, batch, ebn0, seed):
    fz = O.bec_frozen(N, K)
    idx = np.arange(batch)
    u = I.info_bits(seed, idx, fz)
    llr = I.channel_llr(O.encode(u), I.gaussian(seed, idx, N), I.sigma(ebn0, K / N))
    return fz, u, llr


def gpu_q(B, code, llr, max_iter, A, F, stop, trace=False):
    d = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    out = B.polarbp_decode_quantized(code, d, max_iter, A, F, stop, trace=trace)
    torch.cuda.synchronize()
    return tuple(t.cpu().numpy() for t in out)


def test_hand_traced_n2(B):
    code = B.polarbp_construct(2, 1, frozen_mask=np.array([1, 0], np.uint8))
    uh, it, pe, tl, tr = gpu_q(B, code, np.array([[1.3, -0.7]], np.float32), 2, 15, 2, 0, trace=True)
    for t in range(2):
        assert tr[0, t].tolist() == [[5, -3], [-3, 2]]
        assert tl[0, t].tolist() == [[-3, 5], [32767, 0]]
    assert uh[0].tolist() == [0, 0] and int(pe[0]) == 2 and int(it[0]) == 2


@pytest.mark.parametrize("N", [2, 8, 64, 256, 1024])
@pytest.mark.parametrize("stop", [0, 1])
def test_decisions_match_oracle(B, N, stop):
    K = N // 2
    batch = 200 if N <= 256 else 80
    code = B.polarbp_construct(N, K)
    for ebn0, seed, (A, F) in ((1.5, 2, (15, 3)), (3.0, 3, (15, 2)), (2.5, 4, (12, 5))):
        fz, u, llr = host_inputs(N, K, batch, ebn0, seed)
        uh, it, pe = gpu_q(B, code, llr, 40, A, F, stop)
        ouh, oit, ope = O.decode_q_batch(fz, llr, 40, A, F, stop)
        assert np.array_equal(uh, ouh) and np.array_equal(it, oit) and np.array_equal(pe, ope)


@pytest.mark.parametrize("N", [16, 64, 1024])
def test_message_planes_match_oracle(B, N):
    fz, u, llr = host_inputs(N, N // 2, 8, 2.0, 9)
    code = B.polarbp_construct(N, N // 2)
    uh, it, pe, tl, tr = gpu_q(B, code, llr, 25, 15, 3, 1, trace=True)
    for c in range(llr.shape[0]):
        o = O.decode_q(fz, llr[c], 25, 15, 3, O.STOP_GMATRIX, trace=True)
        n = o["iters"]
        assert it[c] == n
        assert np.array_equal(tl[c, :n].astype(np.int32), o["L"])
        assert np.array_equal(tr[c, :n].astype(np.int32), o["R"])


def test_arguments_and_status(B):
    code = B.polarbp_construct(64, 32)
    llr = torch.zeros((2, 64), dtype=torch.float32, device="cuda")
    for args in ((0, 15, 3, 0), (5, 0, 3, 0), (5, 17, 3, 0), (5, 15, 9, 0), (5, 15, 3, 2)):
        with pytest.raises(B.PolarBPError) as e:
            B.polarbp_decode_quantized(code, llr, *args)
        assert e.value.code == B.POLARBP_ERR_ARG
    big = B.polarbp_construct(2048, 1024)
    with pytest.raises(B.PolarBPError) as e:
        B.polarbp_decode_quantized(big, torch.zeros((1, 2048), dtype=torch.float32, device="cuda"), 5)
    assert e.value.code == B.POLARBP_ERR_UNSUPPORTED
    B.polarbp_decode_quantized(code, torch.empty((0, 64), dtype=torch.float32, device="cuda"), 5)
    assert B.polarbp_get_status(code) == B.POLARBP_OK
    llr[0, 3] = float("inf")
    B.polarbp_decode_quantized(code, llr, 3)
    assert B.polarbp_get_status(code) == B.POLARBP_ERR_NONFINITE
