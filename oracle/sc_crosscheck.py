"""Cross-check of Sec. III's comparison with successive-cancellation decoding, on the CPU oracle.

TEST INFRASTRUCTURE ONLY: it runs the oracle (FP64) on seeded synthetic inputs.

Sec. III argues that a CSFG frozen by the proposed scheme decides its constituent code at least
as well as SC decoding would: its inputs are at least as reliable as the SC sub-tree's, and the
check of Eqs. (2)-(4) yields the ML decision (Lemma 1).  Frozen CSFGs cover a prefix [0, P) of the
source positions, so on the same codewords the script compares
  * the rate of codewords whose stored decisions on [0, P) hold an error (BP with G-matrix stop and
    CSFG freezing, max 60 iterations, alpha 0.9375), with
  * the rate of codewords whose SC decisions on the same [0, P) hold an error (exact box-plus and
    min-sum SC),
and reports the overall frame error rates of the three decoders beside them.

python -m oracle.sc_crosscheck [--codewords 50000] [--ebn0 1.5 2.0 2.5 3.0 3.5]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1505_04979_gb300 import inputs as I  # noqa: E402

SEED = 1505049790 + 31


def wilson(k: int, n: int, z: float = 1.96):
    p = k / n
    d = 1 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return max(0.0, c - h), min(1.0, c + h)


def point(N: int, K: int, ebn0: float, n: int):
    fz = O.bec_frozen(N, K)
    idx = np.arange(n)
    u = I.info_bits(SEED, idx, fz)
    llr = I.channel_llr(O.encode(u), I.gaussian(SEED, idx, N), I.sigma(ebn0, K / N))
    uh, it, pe, _, cover = O.decode_batch(fz, llr, 60, 0.9375, O.STOP_GMATRIX, O.FREEZE_CSFG, cover=True)
    pos = np.arange(N)[None, :]
    prefix = pos < cover[:, None]
    out = {"ebn0_db": ebn0, "codewords": n, "avg_cover": float(cover.mean()), "avg_iters": float(it.mean())}
    err = (uh != u)
    k_bp, k_bp_prefix = int(err.any(1).sum()), int((err & prefix).any(1).sum())
    out["bp_freeze"] = {"fer": k_bp / n, "fer_ci95": wilson(k_bp, n),
                        "prefix_error_rate": k_bp_prefix / n, "prefix_ci95": wilson(k_bp_prefix, n)}
    for name, exact in (("sc_exact", True), ("sc_minsum", False)):
        us = O.sc_decode_batch(fz, llr, exact)
        e = (us != u)
        k, kp = int(e.any(1).sum()), int((e & prefix).any(1).sum())
        out[name] = {"fer": k / n, "fer_ci95": wilson(k, n), "prefix_error_rate": kp / n,
                     "prefix_ci95": wilson(kp, n)}
    return out


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--codewords", type=int, default=50000)
    ap.add_argument("--ebn0", type=float, nargs="+", default=[1.5, 2.0, 2.5, 3.0, 3.5])
    ap.add_argument("--N", type=int, default=1024)
    ap.add_argument("--K", type=int, default=512)
    args = ap.parse_args(argv)
    O.build()
    rows = [point(args.N, args.K, eb, args.codewords) for eb in args.ebn0]
    for r in rows:
        b, se, sm = r["bp_freeze"], r["sc_exact"], r["sc_minsum"]
        print(f"{r['ebn0_db']:4.1f} dB  cover {r['avg_cover']:6.1f}  FER bp+freeze {b['fer']:.5f}  "
              f"SC exact {se['fer']:.5f}  SC min-sum {sm['fer']:.5f}  |  errors on [0,P): bp+freeze "
              f"{b['prefix_error_rate']:.5f}  SC exact {se['prefix_error_rate']:.5f}  "
              f"SC min-sum {sm['prefix_error_rate']:.5f}", flush=True)
    print(json.dumps({"N": args.N, "K": args.K, "seed": SEED, "points": rows}))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
