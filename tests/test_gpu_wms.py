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


def checkpoints(ws, batch, T, k, m, N):
    """The forward's checkpoints in the workspace.  k = 1: [batch][T][2][m+1][N], the L and R
    planes after every iteration.  k > 1: [batch][(T-1)//k][m-1][N], checkpoint j = L columns
    1..m-1 after iteration (j+1) k - 1."""
    if k == 1:
        return ws[: batch * T * 2 * (m + 1) * N * 4].view(torch.float32).view(batch, T, 2, m + 1, N)
    nc = (T - 1) // k
    return ws[: batch * nc * (m - 1) * N * 4].view(torch.float32).view(batch, nc, m - 1, N)


@pytest.mark.parametrize("N", [2, 8, 16, 128, 256, 1024])
@pytest.mark.parametrize("k", [1, 3])
def test_forward_state_matches_binary32_oracle(B, N, k):
    """The soft outputs and the checkpoints (both planes after every iteration for k = 1, L
    columns 1..m-1 after every k-th iteration otherwise) are bit-exact against the oracle's
    binary32 forward."""
    T = 10
    m = N.bit_length() - 1
    batch = 6
    fz, u, llr, w = inputs(N, T, batch, N)
    code = B.polarbp_construct(N, N // 2)
    if N == 1024 and k > 1:  # 3 + 2k planes of 45 KB
        with pytest.raises(B.PolarBPError) as e:
            B.polarbp_wms_forward(code, torch.from_numpy(llr).cuda(), torch.from_numpy(w).cuda(),
                                  torch.empty(B.polarbp_wms_workspace(code, batch, T, k), dtype=torch.uint8,
                                              device="cuda"), checkpoint_every=k)
        assert e.value.code == B.POLARBP_ERR_UNSUPPORTED  # the adjoint's planes exceed shared memory
        return
    ws = torch.empty(B.polarbp_wms_workspace(code, batch, T, k), dtype=torch.uint8, device="cuda")
    out = B.polarbp_wms_forward(code, torch.from_numpy(llr).cuda(), torch.from_numpy(w).cuda(), ws,
                                checkpoint_every=k)
    torch.cuda.synchronize()
    ck = checkpoints(ws, batch, T, k, m, N).cpu().numpy()
    out = out.cpu().numpy()
    for c in range(batch):
        o, tl, tr = O.wms_forward(fz, llr[c], w.astype(np.float64), fp32=True, trace=True)
        if k == 1:
            assert np.array_equal(ck[c, :, 0].astype(np.float64), tl)
            assert np.array_equal(ck[c, :, 1].astype(np.float64), tr)
        for j in range((T - 1) // k if k > 1 else 0):
            assert np.array_equal(ck[c, j].astype(np.float64), tl[(j + 1) * k - 1][1:m])
        assert np.array_equal(out[c].astype(np.float64), o)


def test_constant_weights_match_the_decoder(B):
    N, T, batch = 256, 10, 8
    m = 8
    fz, u, llr, _ = inputs(N, T, batch, 3)
    code = B.polarbp_construct(N, N // 2)
    w = torch.full((T, m, N // 2), 0.9375, dtype=torch.float32, device="cuda")
    d = torch.from_numpy(llr).cuda()
    ws = torch.empty(B.polarbp_wms_workspace(code, batch, T), dtype=torch.uint8, device="cuda")
    out = B.polarbp_wms_forward(code, d, w, ws)
    _, _, _, tL, tR, _ = B.polarbp_decode_trace(code, d, T, 0.9375, 0, 0)
    torch.cuda.synchronize()
    ck = checkpoints(ws, batch, T, 1, m, N)
    assert torch.equal(ck[:, :, 0], tL) and torch.equal(ck[:, :, 1], tR)
    assert torch.equal(out, tR[:, T - 1, m] + tL[:, T - 1, m])


def branch_signature(fz, llr, w, fp32):
    """Every comparison and sign the adjoint of Eq. (1) branches on, for all PEs of all
    iterations of one codeword: |Ra| <= |t|, |La| <= |t|, |La| <= |Ra| and the signs of
    La, Ra and t = Lb + Rb, from the oracle's forward planes."""
    N = fz.shape[0]
    m = N.bit_length() - 1
    _, tl, tr = O.wms_forward(fz, llr, w.astype(np.float64), fp32=fp32, trace=True)
    prior = np.zeros((m + 1, N))
    prior[m] = np.where(fz == 1, np.inf, 0.0)
    sig = []
    for t in range(tl.shape[0]):
        Lp = prior if t == 0 else tl[t - 1]
        for s in range(m):
            h = 1 << (m - 1 - s)
            a = np.array([i for i in range(N) if not i & h])
            La, Lb, Ra, Rb = Lp[s + 1][a], Lp[s + 1][a + h], tr[t][s][a], tr[t][s][a + h]
            with np.errstate(invalid="ignore"):
                tt = Lb + Rb
            sig += [np.abs(Ra) <= np.abs(tt), np.abs(La) <= np.abs(tt), np.abs(La) <= np.abs(Ra),
                    np.sign(La), np.sign(Ra), np.sign(tt)]
    return np.concatenate([np.asarray(x, np.float64).ravel() for x in sig])


@pytest.mark.parametrize("N,T", [(16, 10), (128, 10), (256, 10)])
@pytest.mark.parametrize("k", [1, 4, 10])
def test_gradient_matches_oracle_element_by_element(B, N, T, k):
    """The adjoint of Eq. (1) with per-PE weights, entry by entry.
    * Against the oracle's binary32 adjoint (every operation rounded to binary32, the same
      chain-rule order): the LLR gradient of every codeword and the weight gradient, summed
      over the batch in codeword order, are bit-exact.
    * Against the FP64 adjoint: on codewords whose binary32 forward takes every min and sign
      branch the FP64 forward takes, every entry is within 1e-4 relative or 1e-5 absolute.
      The others are flagged and counted; their dout is zeroed in a second backward pass so
      that the batch-summed weight gradient is compared over the unflagged codewords alone.
    With a checkpoint every k iterations the adjoint recomputes the iterations in between; the
    results are the same bit for bit for every k."""
    batch = 12
    fz, u, llr, w = inputs(N, T, batch, 40 + N)
    code = B.polarbp_construct(N, N // 2)
    rng = np.random.default_rng(N)
    dout = rng.normal(0, 1, (batch, N)).astype(np.float32)
    dout[:, fz == 1] = 0.0
    d_llr = torch.from_numpy(llr).cuda()
    d_w = torch.from_numpy(w).cuda()
    ws = torch.empty(B.polarbp_wms_workspace(code, batch, T, k), dtype=torch.uint8, device="cuda")
    B.polarbp_wms_forward(code, d_llr, d_w, ws, checkpoint_every=k)

    def gpu_backward(d):
        gw, gl = B.polarbp_wms_backward(code, d_llr, d_w, torch.from_numpy(d).cuda(), ws, checkpoint_every=k)
        torch.cuda.synchronize()
        return gw.cpu().numpy().astype(np.float64), gl.cpu().numpy().astype(np.float64)

    gw, gl = gpu_backward(dout)
    w64 = w.astype(np.float64)
    ow32 = np.zeros(w.shape, np.float32)
    for c in range(batch):
        dw_c, dl_c = O.wms_backward(fz, llr[c], w64, dout[c].astype(np.float64), fp32=True)
        assert np.array_equal(gl[c], dl_c), c
        ow32 = (ow32 + dw_c.astype(np.float32)).astype(np.float32)
    assert np.array_equal(gw, ow32.astype(np.float64))

    flagged = [c for c in range(batch)
               if not np.array_equal(branch_signature(fz, llr[c], w, True), branch_signature(fz, llr[c], w, False))]
    print(f"N={N}: {len(flagged)} of {batch} codewords take a different branch in binary32")
    assert len(flagged) <= batch // 2
    d2 = dout.copy()
    d2[flagged] = 0.0
    gw2, gl2 = gpu_backward(d2)
    ow = np.zeros_like(w64)
    for c in range(batch):
        if c in flagged:
            continue
        dw_c, dl_c = O.wms_backward(fz, llr[c], w64, d2[c].astype(np.float64))
        ow += dw_c
        err = np.abs(gl2[c] - dl_c)
        assert np.all((err <= 1e-4 * np.abs(dl_c)) | (err <= 1e-5)), (c, err.max())
    err = np.abs(gw2 - ow)
    bad = ~((err <= 1e-4 * np.abs(ow)) | (err <= 1e-5))
    assert not bad.any(), (int(bad.sum()), float(err[bad].max()))


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
        out = B.weighted_min_sum(code, d_llr, w, checkpoint_every=3)
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


def test_checkpoint_interval_arguments(B):
    code = B.polarbp_construct(128, 64)
    d = torch.zeros((4, 128), dtype=torch.float32, device="cuda")
    w = torch.ones((10, 7, 64), dtype=torch.float32, device="cuda")
    ws = torch.empty(B.polarbp_wms_workspace(code, 4, 10, 1), dtype=torch.uint8, device="cuda")
    with pytest.raises(B.PolarBPError) as e:
        B.polarbp_wms_forward(code, d, w, ws, checkpoint_every=0)
    assert e.value.code == B.POLARBP_ERR_ARG
    # an interval above the iteration count acts as the iteration count: no checkpoint at all
    assert B.polarbp_wms_workspace(code, 4, 10, 50) == B.polarbp_wms_workspace(code, 4, 10, 10)
    assert B.polarbp_wms_workspace(code, 4, 10, 10) < B.polarbp_wms_workspace(code, 4, 10, 1)
