"""GPU parity of the true flooding schedule (polarbp_decode_flooding, through the C ABI)
against the CPU oracle's flooding decoder run in binary32 arithmetic.

Decisions, iteration counts and PE counts are compared bit-exactly; message planes are
compared bit-exactly on every entry of every iteration (flooding has no covered CSFGs).
The hand-traced (4,2) example pins both sides to the same values.
"""
import json
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1505_04979_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ALPHA = 0.9375
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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
    x = O.encode(u)
    llr = I.channel_llr(x, I.gaussian(seed, idx, N), I.sigma(ebn0, K / N))
    return fz, u, x, llr


def gpu_flood(B, code, llr, max_iter, stop, scale=ALPHA, trace=False):
    d = torch.from_numpy(np.ascontiguousarray(llr)).cuda()
    out = B.polarbp_decode_flooding(code, d, max_iter, scale, stop, trace=trace)
    torch.cuda.synchronize()
    return tuple(t.cpu().numpy() for t in out)


def test_hand_traced_n4(B):
    g = json.load(open(os.path.join(GOLDEN, "n4_flooding.json")))
    conv = lambda v: [np.inf if e == "inf" else (-np.inf if e == "-inf" else e) for e in v]
    code = B.polarbp_construct(4, 2, frozen_mask=np.array(g["frozen"], np.uint8))
    uh, it, pe, tl, tr = gpu_flood(B, code, np.array([g["llr"]], np.float32), 2, 0, scale=g["alpha"], trace=True)
    for t, key in ((0, "iter1"), (1, "iter2")):
        e = g[key]
        assert tr[0, t, 1].tolist() == conv(e["R1"])
        assert tr[0, t, 2].tolist() == conv(e["R2"])
        assert tl[0, t, 0].tolist() == conv(e["L0"])
        assert tl[0, t, 1].tolist() == conv(e["L1"])
    assert uh[0].tolist() == g["u_hat"] and int(pe[0]) == g["pe"] and int(it[0]) == 2


def test_flooding_configuration_every_message(B):
    """The tiny-code configuration: (64,32), Eb/N0 2.5 dB, 1000 codewords, 40 fixed iterations,
    alpha 0.9375: every message of every iteration equals the binary32 oracle's."""
    N, K, batch, iters = 64, 32, 1000, 40
    code = B.polarbp_construct(N, K)
    fz, u, x, llr = host_inputs(N, K, batch, 2.5, 1)
    uh, it, pe, tl, tr = gpu_flood(B, code, llr, iters, 0, trace=True)
    ouh, oit, ope, _ = O.decode_flood_batch(fz, llr, iters, ALPHA, O.STOP_NONE, fp32=True)
    assert np.array_equal(uh, ouh) and np.array_equal(it, oit) and np.array_equal(pe, ope)
    for c in range(0, batch, 37):
        o = O.decode_flood(fz, llr[c], iters, ALPHA, fp32=True, trace=True)
        assert np.array_equal(tl[c].astype(np.float64), o["L"])
        assert np.array_equal(tr[c].astype(np.float64), o["R"])


@pytest.mark.parametrize("N", [2, 8, 32, 256, 1024])
@pytest.mark.parametrize("stop", [0, 1])
def test_decisions_match_oracle(B, N, stop):
    K = N // 2
    batch = 300 if N <= 256 else 120
    code = B.polarbp_construct(N, K)
    for ebn0, seed in ((1.5, 2), (3.0, 3)):
        fz, u, x, llr = host_inputs(N, K, batch, ebn0, seed)
        uh, it, pe = gpu_flood(B, code, llr, 60, stop)
        ouh, oit, ope, _ = O.decode_flood_batch(fz, llr, 60, ALPHA, stop, fp32=True)
        assert np.array_equal(uh, ouh) and np.array_equal(it, oit) and np.array_equal(pe, ope)


@pytest.mark.parametrize("N", [8, 64, 1024])
def test_noiseless_stops_at_iteration_m(B, N):
    m = N.bit_length() - 1
    code = B.polarbp_construct(N, N // 2)
    fz = O.bec_frozen(N, N // 2)
    u = I.info_bits(12, np.arange(16), fz)
    llr = I.noiseless_llr(O.encode(u), 2.5)
    uh, it, pe = gpu_flood(B, code, llr, 3 * m, 1)
    nz = u.any(axis=1)
    assert np.array_equal(uh, u)
    assert np.all(it[nz] == m) and np.all(pe[nz] == m * m * N // 2)


def test_empty_batch_bad_arguments_and_status(B):
    code = B.polarbp_construct(64, 32)
    empty = torch.empty((0, 64), dtype=torch.float32, device="cuda")
    B.polarbp_decode_flooding(code, empty, 10)
    llr = torch.zeros((2, 64), dtype=torch.float32, device="cuda")
    for kw in ({"max_iter": 0}, {"scale": 0.0}, {"stop_mode": 3}):
        args = dict(max_iter=10, scale=ALPHA, stop_mode=0)
        args.update(kw)
        with pytest.raises(B.PolarBPError) as e:
            B.polarbp_decode_flooding(code, llr, args["max_iter"], args["scale"], args["stop_mode"])
        assert e.value.code == B.POLARBP_ERR_ARG
    big = B.polarbp_construct(2048, 1024)
    with pytest.raises(B.PolarBPError) as e:
        B.polarbp_decode_flooding(big, torch.zeros((1, 2048), dtype=torch.float32, device="cuda"), 5)
    assert e.value.code == B.POLARBP_ERR_UNSUPPORTED
    assert B.polarbp_get_status(code) == B.POLARBP_OK
    llr[1, 5] = float("nan")
    B.polarbp_decode_flooding(code, llr, 3)
    assert B.polarbp_get_status(code) == B.POLARBP_ERR_NONFINITE
