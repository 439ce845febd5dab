"""Comparison of the freezing rules Sec. III leaves open, on the CPU oracle.

TEST INFRASTRUCTURE ONLY: it runs the oracle (FP64) on seeded synthetic inputs.

Sec. III freezes a CSFG when the hard decisions of its inputs (Eq. (2)), inverted through
F^{(x)(m-j)} (Eq. (3)), meet the frozen-bit constraints (Eq. (4)).  The text does not settle
which message Eq. (2) decides on, and says nothing of how reliable the inputs must be.  On the
same (1024,512) codewords the script runs reading A (one check per stage per iteration) with
  * rule R:        Eq. (2) on R, as printed (every other part of the library);
  * rule R+L:      Eq. (2) on the a-posteriori message R + L of the CSFG's input node;
  * rule |R|>=t:   rule R, and a CSFG freezes only when every input has |R| >= t;
beside the G-matrix stop alone and plain BP with fixed iterations, and reports FER with Wilson
95 % intervals, BER, average iterations and PE updates per codeword (Sec. IV count).

python -m oracle.freeze_rules [--codewords 10000] [--ebn0 2.5 3.0] [--max-iter 60]
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

SEED = 1505049790 + 41
N, K, ALPHA = 1024, 512, 0.9375


def wilson(k: int, n: int, z: float = 1.96):
    p = k / n
    d = 1 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return max(0.0, c - h), min(1.0, c + h)


def stats(u, uh, it, pe):
    n = u.shape[0]
    errs = int(np.any(uh != u, axis=1).sum())
    lo, hi = wilson(errs, n)
    return {"fer": errs / n, "fer_ci95": [lo, hi], "ber": float((uh != u).sum()) / (n * K),
            "avg_iters": float(it.mean()), "pe_per_codeword": float(pe.mean())}


def main() -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--codewords", type=int, default=10000)
    ap.add_argument("--ebn0", type=float, nargs="+", default=[2.5, 3.0])
    ap.add_argument("--max-iter", type=int, default=60)
    ap.add_argument("--thresholds", type=float, nargs="+", default=[1.0, 2.0, 4.0])
    args = ap.parse_args()
    fz = O.bec_frozen(N, K)
    idx = np.arange(args.codewords)
    out = []
    for eb in args.ebn0:
        u = I.info_bits(SEED, idx, fz)
        llr = I.channel_llr(O.encode(u), I.gaussian(SEED, idx, N), I.sigma(eb, K / N))
        row = {"ebn0_db": eb, "max_iter": args.max_iter, "codewords": args.codewords}
        uh, it, pe, _ = O.decode_batch(fz, llr, args.max_iter, ALPHA, O.STOP_NONE, O.FREEZE_OFF)
        row["fixed"] = stats(u, uh, it, pe)
        uh, it, pe, _ = O.decode_batch(fz, llr, args.max_iter, ALPHA, O.STOP_GMATRIX, O.FREEZE_OFF)
        row["gstop"] = stats(u, uh, it, pe)
        for stop, sname in ((O.STOP_NONE, "freeze"), (O.STOP_GMATRIX, "gstop_freeze")):
            rules = [("R", O.RULE_R, 0.0), ("R+L", O.RULE_R_PLUS_L, 0.0)]
            rules += [(f"|R|>={t:g}", O.RULE_THRESHOLD, t) for t in args.thresholds]
            for rname, rule, theta in rules:
                uh, it, pe = O.decode_rule_batch(fz, llr, args.max_iter, ALPHA, stop, rule, theta)
                row[f"{sname} {rname}"] = stats(u, uh, it, pe)
        out.append(row)
        print(f"Eb/N0 {eb} dB, max {args.max_iter} iterations, {args.codewords} codewords", flush=True)
        for name, s in row.items():
            if isinstance(s, dict):
                print(f"  {name:22s} FER {s['fer']:.5f} [{s['fer_ci95'][0]:.5f}, {s['fer_ci95'][1]:.5f}]  "
                      f"iterations {s['avg_iters']:6.2f}  PE/codeword {s['pe_per_codeword']:9.0f}", flush=True)
    print(json.dumps({"freeze_rules": out}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
