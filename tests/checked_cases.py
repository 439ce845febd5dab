"""Decode cases for the memory checks, run on whichever build of the library the
binding loads (POLARBP_LIBRARY selects the checked build).

Every decoder kernel runs at small sizes with ragged batches: the one-block and
pipelined decoders for N = 2 .. 4096 in every stop and freeze mode, message
planes, the cluster decoder for N = 8192 .. 32768, the persistent mixed stream
(one launch per length and one launch for all), the host entry points, the
flooding, quantised and weighted min-sum kernels.  Every output is written
into the middle of a buffer whose GUARD bytes on either side hold a sentinel,
so a store past either end of an output shows as a changed sentinel.  After
each case the code handles' status is read; on the checked build a store into
a shared-memory redzone makes it POLARBP_ERR_CHECK.

``python tests/checked_cases.py OUT.npz`` runs every case and saves the
outputs, the sentinel checks and the status of each case.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

from paper_1505_04979_gb300 import binding as B  # noqa: E402

SEED = 0x5EED
GUARD = 4096  # sentinel bytes on each side of an output
SCALE = 0.9375


class Guarded:
    """A tensor of `shape` in the middle of a sentinel-filled buffer."""

    def __init__(self, shape, dtype, fill, device="cuda", pin=False):
        import torch
        n = int(np.prod(shape))
        self.g = GUARD // torch.empty((), dtype=dtype).element_size()
        self.n = n
        self.fill = fill
        self.buf = torch.full((n + 2 * self.g,), fill, dtype=dtype, device=device)
        if pin:
            self.buf = self.buf.pin_memory()
        self.t = self.buf[self.g:self.g + n].view(shape)

    def intact(self) -> bool:
        b = self.buf
        return bool((b[:self.g] == self.fill).all()) and bool((b[self.g + self.n:] == self.fill).all())


def _outs(batch, N, device="cuda", pin=False):
    import torch
    return (Guarded((batch, N), torch.uint8, 0xA5, device, pin), Guarded((batch,), torch.int32, -7, device, pin),
            Guarded((batch,), torch.int64, -7, device, pin))


def _status(codes) -> tuple[int, str]:
    """Worst status of the handles (read and cleared), with the library's message."""
    import torch
    torch.cuda.synchronize()
    for c in codes:
        rc = B.lib().polarbp_get_status(c.handle, None)
        if rc != B.POLARBP_OK:
            return rc, B.lib().polarbp_last_error().decode()
    return B.POLARBP_OK, ""


def _llr(code, batch, ebn0, first=0):
    _, llr = B.polarbp_awgn(code, SEED, first, batch, ebn0, with_u=False)
    return llr


def case_decode(N, K, batch, ebn0, max_iter, stop, freeze, mapping=None):
    code = B.polarbp_construct(N, K)
    if mapping is not None:
        B.polarbp_set_thread_mapping(code, mapping)
    llr = _llr(code, batch, ebn0)
    u, it, pe = _outs(batch, N)
    B.polarbp_decode(code, llr, max_iter, SCALE, stop, freeze, u.t, it.t, pe.t)
    rc, msg = _status([code])
    out = {"u_hat": u.t.cpu().numpy(), "iterations": it.t.cpu().numpy(), "pe": pe.t.cpu().numpy()}
    return out, [u, it, pe], rc, msg


def case_trace(N, K, batch, ebn0, max_iter, stop, freeze):
    code = B.polarbp_construct(N, K)
    llr = _llr(code, batch, ebn0)
    u, it, pe, tL, tR, tP = B.polarbp_decode_trace(code, llr, max_iter, SCALE, stop, freeze)
    rc, msg = _status([code])
    out = {"u_hat": u.cpu().numpy(), "iterations": it.cpu().numpy(), "pe": pe.cpu().numpy(),
           "trace_P": tP.cpu().numpy()}
    return out, [], rc, msg


def _stream_codes(lengths):
    return [B.polarbp_construct(N, N // 2) for N in lengths]


def case_segments(lengths, counts, ebn0, max_iter, stop, freeze, entry, cpc=None, mapping=None):
    codes = _stream_codes(lengths)
    segs, guards, outs = [], [], []
    for k, (code, n) in enumerate(zip(codes, counts)):
        if cpc is not None:
            try:
                B.polarbp_set_codewords_per_block(code, cpc)
            except B.PolarBPError as e:  # more codewords per block than the length admits
                assert e.code == B.POLARBP_ERR_UNSUPPORTED, e
        if mapping is not None:
            B.polarbp_set_thread_mapping(code, mapping)
        llr = _llr(code, n, ebn0 + 0.25 * k, first=1000 * k)
        u, it, pe = _outs(n, code.N)
        segs.append((code, llr, u.t, it.t, pe.t))
        guards += [u, it, pe]
        outs.append((u, it, pe))
    (B.polarbp_decode_segments if entry == "segments" else B.polarbp_decode_mixed)(
        segs, max_iter, SCALE, stop, freeze)
    rc, msg = _status(codes)
    out = {}
    for k, (u, it, pe) in enumerate(outs):
        out[f"u_hat{k}"] = u.t.cpu().numpy()
        out[f"iterations{k}"] = it.t.cpu().numpy()
        out[f"pe{k}"] = pe.t.cpu().numpy()
    return out, guards, rc, msg


def case_host(N, batch, ebn0, max_iter, stop, freeze, noalloc):
    import torch
    code = B.polarbp_construct(N, N // 2)
    llr = _llr(code, batch, ebn0).cpu().pin_memory()
    u, it, pe = _outs(batch, N, device="cpu", pin=True)
    if noalloc:
        B.polarbp_decode_host_noalloc(code, llr, max_iter, SCALE, stop, freeze, u.t, it.t, pe.t)
    else:
        ws = torch.empty(B.polarbp_decode_host_workspace(code, batch), dtype=torch.uint8, device="cuda")
        B.polarbp_decode_host(code, llr, max_iter, SCALE, stop, freeze, u.t, it.t, pe.t, ws)
    rc, msg = _status([code])
    out = {"u_hat": u.t.numpy().copy(), "iterations": it.t.numpy().copy(), "pe": pe.t.numpy().copy()}
    return out, [u, it, pe], rc, msg


def case_autotune(N, max_iter):
    code = B.polarbp_construct(N, N // 2)
    B.polarbp_autotune(code, max_iter, SCALE, 1, 1)
    rc, msg = _status([code])
    return {}, [], rc, msg


def case_flooding(N, batch, ebn0, max_iter, stop):
    code = B.polarbp_construct(N, N // 2)
    llr = _llr(code, batch, ebn0)
    u, it, pe = _outs(batch, N)
    B.polarbp_decode_flooding(code, llr, max_iter, SCALE, stop, u.t, it.t, pe.t)
    rc, msg = _status([code])
    out = {"u_hat": u.t.cpu().numpy(), "iterations": it.t.cpu().numpy(), "pe": pe.t.cpu().numpy()}
    return out, [u, it, pe], rc, msg


def case_quantized(N, batch, ebn0, max_iter):
    code = B.polarbp_construct(N, N // 2)
    llr = _llr(code, batch, ebn0)
    u, it, pe = _outs(batch, N)
    B.polarbp_decode_quantized(code, llr, max_iter, 15, 3, 1, u.t, it.t, pe.t)
    rc, msg = _status([code])
    out = {"u_hat": u.t.cpu().numpy(), "iterations": it.t.cpu().numpy(), "pe": pe.t.cpu().numpy()}
    return out, [u, it, pe], rc, msg


def case_wms(N, batch, T, k):
    import torch
    code = B.polarbp_construct(N, N // 2)
    llr = _llr(code, batch, 3.0)
    m = code.m
    g = torch.Generator().manual_seed(7)
    w = (0.75 + 0.5 * torch.rand((T, m, N // 2), generator=g)).cuda()
    ws = torch.empty(B.polarbp_wms_workspace(code, batch, T, k), dtype=torch.uint8, device="cuda")
    out_f = Guarded((batch, N), torch.float32, -123.0)
    B.polarbp_wms_forward(code, llr, w, ws, out=out_f.t, checkpoint_every=k)
    dout = torch.randn((batch, N), generator=g).cuda()
    dw, dllr = B.polarbp_wms_backward(code, llr, w, dout, ws, checkpoint_every=k)
    rc, msg = _status([code])
    out = {"out": out_f.t.cpu().numpy(), "dw": dw.cpu().numpy(), "dllr": dllr.cpu().numpy()}
    return out, [out_f], rc, msg


def cases():
    """(name, function, kwargs) of every case, in a fixed order."""
    cs = []
    codes = [(2, 1), (8, 4), (16, 8), (64, 32), (128, 64), (256, 128), (512, 256), (1024, 512), (2048, 1024),
             (4096, 2048)]
    modes = [(0, 0), (1, 0), (0, 1), (1, 1), (1, 2)]
    for N, K in codes:
        batch = 19 if N <= 1024 else 7
        for stop, freeze in modes:
            cs.append((f"decode_N{N}_s{stop}f{freeze}", case_decode,
                       dict(N=N, K=K, batch=batch, ebn0=2.5, max_iter=25, stop=stop, freeze=freeze)))
        if N >= 256:
            for stop in (0, 1):
                cs.append((f"decode_N{N}_s{stop}f1_block", case_decode,
                           dict(N=N, K=K, batch=batch, ebn0=2.5, max_iter=25, stop=stop, freeze=1,
                                mapping=B.POLARBP_MAP_BLOCK)))
    for N in (64, 1024):
        for stop, freeze in ((0, 0), (1, 1)):
            cs.append((f"trace_N{N}_s{stop}f{freeze}", case_trace,
                       dict(N=N, K=N // 2, batch=3, ebn0=2.5, max_iter=8, stop=stop, freeze=freeze)))
    for N in (8192, 16384, 32768):
        for stop, freeze in modes[:4]:
            cs.append((f"cluster_N{N}_s{stop}f{freeze}", case_decode,
                       dict(N=N, K=N // 2, batch=3, ebn0=2.5, max_iter=20, stop=stop, freeze=freeze)))
    cs.append(("trace_N8192_s1f1", case_trace, dict(N=8192, K=4096, batch=1, ebn0=2.5, max_iter=4, stop=1, freeze=1)))
    mix = dict(lengths=(256, 1024, 4096), counts=(50, 30, 9), ebn0=2.5, max_iter=30)
    for cpc in (1, 2, 4):
        for mapping in (B.POLARBP_MAP_PIPELINED, B.POLARBP_MAP_BLOCK):
            for stop, freeze in ((1, 1), (1, 0)):
                cs.append((f"segments_cpc{cpc}_map{mapping}_s{stop}f{freeze}", case_segments,
                           dict(mix, stop=stop, freeze=freeze, entry="segments", cpc=cpc, mapping=mapping)))
    for stop, freeze in modes[:4]:
        cs.append((f"mixed_top4096_s{stop}f{freeze}", case_segments,
                   dict(mix, stop=stop, freeze=freeze, entry="mixed")))
    for lengths, counts in (((256, 512, 1024), (40, 21, 13)), ((256, 2048), (33, 5)), ((256,), (45,))):
        cs.append((f"mixed_top{lengths[-1]}_s1f1", case_segments,
                   dict(lengths=lengths, counts=counts, ebn0=2.5, max_iter=30, stop=1, freeze=1, entry="mixed")))
    cs.append(("host_piped_N1024", case_host, dict(N=1024, batch=33000, ebn0=3.0, max_iter=30, stop=1, freeze=1,
                                                    noalloc=False)))
    cs.append(("host_N256", case_host, dict(N=256, batch=77, ebn0=3.0, max_iter=30, stop=1, freeze=1,
                                             noalloc=False)))
    cs.append(("host_noalloc_N4096", case_host, dict(N=4096, batch=13, ebn0=3.0, max_iter=30, stop=1, freeze=1,
                                                      noalloc=True)))
    cs.append(("autotune_N1024", case_autotune, dict(N=1024, max_iter=20)))
    for N in (64, 1024):
        cs.append((f"flooding_N{N}", case_flooding, dict(N=N, batch=9, ebn0=2.5, max_iter=20, stop=1)))
    cs.append(("quantized_N1024", case_quantized, dict(N=1024, batch=9, ebn0=2.5, max_iter=20)))
    for k in (1, 2):
        cs.append((f"wms_N128_k{k}", case_wms, dict(N=128, batch=16, T=5, k=k)))
    return cs


def run(only=None):
    """Run the cases; returns {name: (outputs, sentinels intact, status, message)}."""
    import torch
    torch.cuda.set_device(0)
    res = {}
    for name, fn, kw in cases():
        if only is not None and name not in only:
            continue
        out, guards, rc, msg = fn(**kw)
        res[name] = (out, all(g.intact() for g in guards), rc, msg)
    return res


def save(res, path):
    arrays, meta = {}, {}
    for name, (out, ok, rc, msg) in res.items():
        for k, v in out.items():
            arrays[f"{name}/{k}"] = v
        meta[name] = {"guards_intact": ok, "status": rc, "message": msg}
    meta["_version"] = B.polarbp_version()
    arrays["_meta"] = np.frombuffer(json.dumps(meta).encode(), dtype=np.uint8)
    np.savez(path, **arrays)


def load(path):
    z = np.load(path)
    meta = json.loads(bytes(z["_meta"]).decode())
    arrays = {k: z[k] for k in z.files if k != "_meta"}
    return arrays, meta


if __name__ == "__main__":
    save(run(), sys.argv[1])
