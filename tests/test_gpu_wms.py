"""Weighted min-sum forward / adjoint on the GPU (through the C ABI and the
torch.autograd.Function) against the oracle."""
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


def inputs(N, T, batch, seed, lo=1.0, hi=4.0):
    K = N // 2
    m = N.bit_length() - 1
    fz = O.bec_frozen(N, K)
    idx = np.arange(batch)
    u = I.info_bits(seed, idx, fz)
    ebn0 = I.uniform(seed, idx, lo, hi)
    llr = I.channel_llr(O.encode(u), I.gaussian(seed, idx, N), I.sigma(ebn0, K / N))
    w = np.random.default_rng(seed).uniform(0.6, 1.3, (T, m, N // 2)).astype(np.float32)
    return fz, u, llr, w


@pytest.mark.parametrize("N", [2, 8, 16, 128, 256, 1024])
def test_forward_planes_match_binary32_oracle(B, N):
    T = 10
    m = N.bit_length() - 1
    batch = 6
    fz, u, llr, w = inputs(N, T, batch, N)
    code = B.polarbp_construct(N, N // 2)
    ws = torch.empty(B.polarbp_wms_workspace(code, batch, T), dtype=torch.uint8, device="cuda")
    out = B.polarbp_wms_forward(code, torch.from_numpy(llr).cuda(), torch.from_numpy(w).cuda(), ws)
    torch.cuda.synchronize()
    ck = ws[: batch * T * 2 * (m + 1) * N * 4].view(torch.float32).view(batch, T, 2, m + 1, N).cpu().numpy()
    out = out.cpu().numpy()
    for c in range(batch):
        o, tl, tr = O.wms_forward(fz, llr[c], w.astype(np.float64), fp32=True, trace=True)
        assert np.array_equal(ck[c, :, 0].astype(np.float64), tl)
        assert np.array_equal(ck[c, :, 1].astype(np.float64), tr)
        assert np.array_equal(out[c].astype(np.float64), o)


def test_constant_weights_match_the_decoder(B):
    N, T, batch = 256, 10, 8
    m = 8
    fz, u, llr, _ = inputs(N, T, batch, 3)
    code = B.polarbp_construct(N, N // 2)
    w = torch.full((T, m, N // 2), 0.9375, dtype=torch.float32, device="cuda")
    d = torch.from_numpy(llr).cuda()
    ws = torch.empty(B.polarbp_wms_workspace(code, batch, T), dtype=torch.uint8, device="cuda")
    B.polarbp_wms_forward(code, d, w, ws)
    _, _, _, tL, tR, _ = B.polarbp_decode_trace(code, d, T, 0.9375, 0, 0)
    torch.cuda.synchronize()
    ck = ws[: batch * T * 2 * (m + 1) * N * 4].view(torch.float32).view(batch, T, 2, m + 1, N)
    assert torch.equal(ck[:, :, 0], tL) and torch.equal(ck[:, :, 1], tR)


@pytest.mark.parametrize("N,T", [(16, 10), (128, 10), (256, 10)])
def test_gradient_matches_fp64_oracle(B, N, T):
    batch = 12
    fz, u, llr, w = inputs(N, T, batch, 40 + N)
    code = B.polarbp_construct(N, N // 2)
    rng = np.random.default_rng(N)
    dout = rng.normal(0, 1, (batch, N)).astype(np.float32)
    dout[:, fz == 1] = 0.0
    d_llr = torch.from_numpy(llr).cuda()
    d_w = torch.from_numpy(w).cuda()
    ws = torch.empty(B.polarbp_wms_workspace(code, batch, T), dtype=torch.uint8, device="cuda")
    B.polarbp_wms_forward(code, d_llr, d_w, ws)
    gw, gl = B.polarbp_wms_backward(code, d_llr, d_w, torch.from_numpy(dout).cuda(), ws)
    torch.cuda.synchronize()
    gw, gl = gw.cpu().numpy().astype(np.float64), gl.cpu().numpy().astype(np.float64)
    ow = np.zeros_like(w, dtype=np.float64)
    ol = np.zeros((batch, N))
    for c in range(batch):
        dw_c, dl_c = O.wms_backward(fz, llr[c], w.astype(np.float64), dout[c].astype(np.float64))
        ow += dw_c
        ol[c] = dl_c
    for g, o in ((gw, ow), (gl, ol)):
        assert np.linalg.norm(g - o) <= 1e-4 * np.linalg.norm(o) + 1e-6
        assert np.mean(np.abs(g - o) <= 1e-4 * np.abs(o).max() + 1e-6) >= 0.999


def test_autograd_function_and_training_step(B):
    N, T, batch = 128, 10, 512
    m = 7
    fz, u, llr, _ = inputs(N, T, batch, 9)
    code = B.polarbp_construct(N, N // 2)
    info = torch.from_numpy(np.nonzero(fz == 0)[0]).cuda()
    d_llr = torch.from_numpy(llr).cuda()
    target = torch.from_numpy(u).cuda()[:, info].float()
    w = torch.full((T, m, N // 2), 0.9375, dtype=torch.float32, device="cuda", requires_grad=True)

    def loss_fn():
        out = B.weighted_min_sum(code, d_llr, w)
        return torch.nn.functional.binary_cross_entropy_with_logits(-out[:, info], target)

    loss = loss_fn()
    loss.backward()
    g_auto = w.grad.detach().clone()
    # the same gradient through the C ABI directly
    out = B.polarbp_wms_forward(code, d_llr, w.detach(),
                                ws := torch.empty(B.polarbp_wms_workspace(code, batch, T), dtype=torch.uint8,
                                                  device="cuda"))
    x = (-out[:, info]).detach().requires_grad_(True)
    torch.nn.functional.binary_cross_entropy_with_logits(x, target).backward()
    dout = torch.zeros((batch, N), dtype=torch.float32, device="cuda")
    dout[:, info] = -x.grad
    g_direct, _ = B.polarbp_wms_backward(code, d_llr, w.detach(), dout, ws)
    assert torch.allclose(g_auto, g_direct)
    opt = torch.optim.Adam([w], lr=0.01)
    first = float(loss.detach())
    for _ in range(30):
        opt.zero_grad()
        l = loss_fn()
        l.backward()
        opt.step()
    assert float(loss_fn().detach()) < first
