"""Bit-reversed codeword order (x = u B_N F^{(x)m}, Sec. II with Arikan's B_N) on the GPU,
through the C ABI, against the oracle: the encoder bit for bit, the device channel against the
shared host generator, and the decoders (one block per codeword, pipelined, cluster, host entry
point, mixed stream) on LLRs received in channel order against the oracle's natural decode of
the same LLRs put back in code order."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04979_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

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


def bitrev_code(B, N, K):
    code = B.polarbp_construct(N, K)
    code.set_bit_reversed(True)
    assert code.bit_reversed()
    return code


def channel_inputs(N, K, batch, ebn0, seed):
    """Source bits and the LLRs of their bit-reversed codewords in channel order."""
    fz = O.bec_frozen(N, K)
    idx = np.arange(batch)
    u = I.info_bits(seed, idx, fz)
    llr = I.channel_llr(O.encode_bit_reversed(u), I.gaussian(seed, idx, N), I.sigma(ebn0, K / N))
    return fz, u, np.ascontiguousarray(llr, dtype=np.float32)


@pytest.mark.parametrize("N", [2, 16, 256, 4096])
def test_encoder(B, N):
    code = bitrev_code(B, N, N // 2)
    u = np.random.default_rng(N).integers(0, 2, (33, N)).astype(np.uint8)
    x = B.polarbp_encode(code, torch.from_numpy(u).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), O.encode_bit_reversed(u))


@pytest.mark.parametrize("N", [8, 64, 256, 1024, 2048, 4096, 8192])
@pytest.mark.parametrize("mode", [(1, 1), (0, 1), (1, 0)])
def test_decode_matches_oracle(B, N, mode):
    K = N // 2
    batch = 48 if N <= 1024 else 8
    code = bitrev_code(B, N, K)
    fz, u, llr = channel_inputs(N, K, batch, 2.5, 600 + N)
    d = torch.from_numpy(llr).cuda()
    uh, it, pe = B.polarbp_decode(code, d, 40, ALPHA, *mode)
    torch.cuda.synchronize()
    ouh, oit, ope, _ = O.decode_batch(fz, O.natural_order_llr(llr), 40, ALPHA, mode[0], mode[1], fp32=True)
    assert np.array_equal(it.cpu().numpy(), oit)
    assert np.array_equal(pe.cpu().numpy(), ope)
    assert np.array_equal(uh.cpu().numpy(), ouh)


def test_device_channel_and_host_entry_point(B):
    N, K, batch = 1024, 512, 64
    code = bitrev_code(B, N, K)
    fz = O.bec_frozen(N, K)
    u, llr = B.polarbp_awgn(code, 17, 0, batch, 3.0)
    torch.cuda.synchronize()
    idx = np.arange(batch)
    hu = I.info_bits(17, idx, fz)
    hllr = I.channel_llr(O.encode_bit_reversed(hu), I.gaussian(17, idx, N), I.sigma(3.0, K / N))
    assert np.array_equal(u.cpu().numpy(), hu)
    g = llr.cpu().numpy()
    assert np.all(np.abs(g - hllr) <= 1e-4 * np.maximum(1.0, np.abs(hllr)))
    # the host entry point on the device generator's LLRs, against the oracle on the same values
    h = torch.empty((batch, N), dtype=torch.float32).pin_memory()
    h.copy_(llr)
    hu_out = torch.empty((batch, N), dtype=torch.uint8).pin_memory()
    hit = torch.empty(batch, dtype=torch.int32).pin_memory()
    hpe = torch.empty(batch, dtype=torch.int64).pin_memory()
    ws = torch.empty(B.polarbp_decode_host_workspace(code, batch), dtype=torch.uint8, device="cuda")
    B.polarbp_decode_host(code, h, 60, ALPHA, 1, 1, hu_out, hit, hpe, ws)
    ouh, oit, ope, _ = O.decode_batch(fz, O.natural_order_llr(h.numpy()), 60, ALPHA, 1, 1, fp32=True)
    assert np.array_equal(hu_out.numpy(), ouh) and np.array_equal(hit.numpy(), oit)
    assert np.array_equal(hpe.numpy(), ope)


def test_variant_decoders_reject_bit_reversed_codes(B):
    code = bitrev_code(B, 64, 32)
    d = torch.zeros((4, 64), dtype=torch.float32, device="cuda")
    with pytest.raises(B.PolarBPError) as e:
        B.polarbp_decode_flooding(code, d, 10, ALPHA, 1)
    assert e.value.code == B.POLARBP_ERR_UNSUPPORTED
