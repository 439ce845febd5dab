"""The allocation-free host entry point, for callers that may not call cudaMalloc
(real-time receive chains that forbid device allocation once running, plug-ins
whose host application owns all device memory).

polarbp_decode_host_noalloc stages through the library's built-in device array
instead of a caller workspace.  Two calls in a row, on different inputs, must
give exactly what polarbp_decode_host gives with a caller workspace, and a
batch whose staging does not fit the array must be rejected.  The file is named
to run last, so a stop at the first failure has run every other test first.
"""
import numpy as np
import pytest

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


def _pinned(shape, dtype):
    return torch.empty(shape, dtype=dtype).pin_memory()


def _with_workspace(B, code, h_llr, max_iter, mode):
    batch, N = h_llr.shape
    ws = torch.empty(B.polarbp_decode_host_workspace(code, batch), dtype=torch.uint8, device="cuda")
    u, it, pe = _pinned((batch, N), torch.uint8), _pinned(batch, torch.int32), _pinned(batch, torch.int64)
    B.polarbp_decode_host(code, h_llr, max_iter, 0.9375, *mode, u, it, pe, ws)
    return u.numpy().copy(), it.numpy().copy(), pe.numpy().copy()


def _no_alloc(B, code, h_llr, max_iter, mode):
    batch, N = h_llr.shape
    u, it, pe = _pinned((batch, N), torch.uint8), _pinned(batch, torch.int32), _pinned(batch, torch.int64)
    B.polarbp_decode_host_noalloc(code, h_llr, max_iter, 0.9375, *mode, u, it, pe)
    return u.numpy().copy(), it.numpy().copy(), pe.numpy().copy()


@pytest.mark.parametrize("N,K,batch", [(1024, 512, 1500), (64, 32, 700)])
def test_two_calls_match_the_workspace_entry_point(B, N, K, batch):
    code = B.polarbp_construct(N, K)
    inputs = []
    for seed in (11, 12):
        _, llr = B.polarbp_awgn(code, seed, 0, batch, 2.5, with_u=False)
        h = _pinned((batch, N), torch.float32)
        h.copy_(llr)
        inputs.append(h)
    torch.cuda.synchronize()
    for mode in ((1, 1), (0, 0)):
        want = [_with_workspace(B, code, h, 40, mode) for h in inputs]
        got = [_no_alloc(B, code, h, 40, mode) for h in inputs]  # two calls in a row
        for w, g in zip(want, got):
            for a, b in zip(w, g):
                assert np.array_equal(a, b)
        assert not np.array_equal(got[0][0], got[1][0])


@pytest.mark.parametrize("N,K", [(1024, 512), (32768, 16384)])
def test_limit_is_exact(B, N, K):
    """A batch one codeword over the limit is rejected with the limit in the message; a batch
    of exactly the limit fits and decodes as polarbp_decode_host does with a workspace."""
    import re
    code = B.polarbp_construct(N, K)
    over = (16 << 20) // (N * 5) + 8  # 4 B of LLR + 1 B of u_hat per position: surely too many
    h = _pinned((over, N), torch.float32)
    h.zero_()
    u, it, pe = _pinned((over, N), torch.uint8), _pinned(over, torch.int32), _pinned(over, torch.int64)
    with pytest.raises(B.PolarBPError) as e:
        B.polarbp_decode_host_noalloc(code, h, 10, 0.9375, 1, 1, u, it, pe)
    assert e.value.code == B.POLARBP_ERR_ARG
    assert "16 MiB" in str(e.value)
    limit = int(re.search(r"at most (\d+) codewords", str(e.value)).group(1))
    assert 0 < limit < over
    assert B.polarbp_decode_host_workspace(code, limit) <= 16 << 20 < B.polarbp_decode_host_workspace(code, limit + 1)
    with pytest.raises(B.PolarBPError) as e:
        B.polarbp_decode_host_noalloc(code, h[: limit + 1], 10, 0.9375, 1, 1, u[: limit + 1], it[: limit + 1],
                                      pe[: limit + 1])
    assert e.value.code == B.POLARBP_ERR_ARG
    _, llr = B.polarbp_awgn(code, 21, 0, limit, 3.0, with_u=False)
    hl = _pinned((limit, N), torch.float32)
    hl.copy_(llr)
    torch.cuda.synchronize()
    want = _with_workspace(B, code, hl, 20, (1, 1))
    got = _no_alloc(B, code, hl, 20, (1, 1))
    for a, b in zip(want, got):
        assert np.array_equal(a, b)
