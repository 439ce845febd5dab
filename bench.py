"""Benchmark: decoded information Gbit/s of BP polar decoding on GB300.

Workload (one step = one pass of the whole decode path over one batch):
  (1024, 512) polar code, frozen set from the BEC(0.5) recursion, BPSK over AWGN
  at Eb/N0 = 3.0 dB (the operating point of the paper's Sec. IV comparison),
  2^20 codewords per step per GPU, scaled min-sum alpha = 0.9375, at most 60
  iterations, G-matrix early stop + CSFG freezing, binary32 messages.
The same batch is also decoded with fixed iterations and with the G-matrix stop
alone; FER (95% Wilson interval), average iterations and PE updates per
codeword are reported for all three.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun every rank decodes its own codewords (weak scaling); rank 0
prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "info Gbit/s/GB300 at N=1024,R=1/2 vs plain BP at equal FER; PE updates/codeword"
N, K = 1024, 512
ALPHA = 0.9375
EBN0 = 3.0
MAX_ITER = 60
SEED = 1505049790
# Issue-slot ceiling of the PE update: SMs x 128 lanes (4 schedulers x 32) x the
# maximum SM clock, over 15 lane instructions per PE update -- Eq. (1) with the
# min-sum f is 3 adds, 3 min-magnitude selections, 3 scalings by alpha and 3 sign
# products each merged into the magnitude by one logic operation.  The SM count
# is read from the device and the clock from MEASURED_PEAKS.json when they are
# available (GB300: 152 SMs, 2070 MHz).
LANES, OPS_PER_PE = 128, 15
SMS, SM_MAX_HZ = 152, 2.07e9


def _device_constants():
    """SM count of cuda:0 and the measured maximum SM clock, when available."""
    global SMS, SM_MAX_HZ, PEAK_PE_PER_S
    try:
        import torch
        if torch.cuda.is_available():
            SMS = torch.cuda.get_device_properties(0).multi_processor_count
    except Exception:
        pass
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            mhz = json.load(fh).get("sm_max_mhz")
        if mhz:
            SM_MAX_HZ = float(mhz) * 1e6
    except (OSError, ValueError):
        pass
    PEAK_PE_PER_S = SMS * LANES * SM_MAX_HZ / OPS_PER_PE


PEAK_PE_PER_S = SMS * LANES * SM_MAX_HZ / OPS_PER_PE
# (stop_mode, freeze_mode): plain BP with fixed iterations (the paper's baseline [14]), the
# G-matrix stop ([18]), freezing alone (the paper's proposed method: decoding ends when every
# CSFG is frozen or at max_iter), and both
MODES = {"fixed": (0, 0), "gstop": (1, 0), "freeze": (0, 1), "gstop_freeze": (1, 1)}
PROFILE = os.path.join(ROOT, "profiles", "bp_decode_pipe_n1024_ebn0_3db.md")
# the headline kernel's sources: the pipelined decoder and the sweep it shares
KERNEL_SRCS = [os.path.join(ROOT, "paper_1505_04979_gb300", "csrc", f)
               for f in ("bp_pipe.cuh", "bp_decode.cuh", "checked.cuh")]


def kernel_source_sha256() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SRCS:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def wilson(k: int, n: int, z: float = 1.96):
    if n == 0:
        return (0.0, 1.0)
    p = k / n
    d = 1 + z * z / n
    c = (p + z * z / (2 * n)) / d
    h = z * math.sqrt(p * (1 - p) / n + z * z / (4 * n * n)) / d
    return (max(0.0, c - h), min(1.0, c + h))


def kernel_traffic():
    """DRAM bytes per full launch from the committed ncu summary, or None when the
    kernel source changed since that capture."""
    if not os.path.exists(PROFILE):
        return None
    text = open(PROFILE).read()
    m_sha = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    m_tr = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    if not m_sha or not m_tr:
        return None
    return float(m_tr.group(1)) if kernel_source_sha256() == m_sha.group(1) else None


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(gpus: int):
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, local, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _reduce_device():
    import torch.distributed as dist
    return "cuda" if dist.get_backend() == "nccl" else "cpu"


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, world):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor(v, dtype=torch.float64, device=_reduce_device())
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.tolist()


def shard_first(rank: int, batch: int) -> int:
    """First codeword index of a rank: codewords are independent and the keyed generator
    regenerates any of them, so rank r decodes [r * batch, (r + 1) * batch) (weak scaling)."""
    return rank * batch


# ---------------------------------------------------------------------------
# CPU oracle leg (baseline / reference arm)
# ---------------------------------------------------------------------------
def oracle_inputs(count: int, first: int):
    from oracle import oracle as O
    from paper_1505_04979_gb300 import inputs as I
    fz = O.bec_frozen(N, K)
    idx = np.arange(first, first + count)
    u = I.info_bits(SEED, idx, fz)
    x = O.encode(u)
    llr = I.channel_llr(x, I.gaussian(SEED, idx, N), I.sigma(EBN0, K / N))
    return fz, u, llr


def oracle_time(count: int, first: int = 0):
    from oracle import oracle as O
    fz, u, llr = oracle_inputs(count, first)
    t0 = time.perf_counter()
    uh, it, pe, _ = O.decode_batch(fz, llr, MAX_ITER, ALPHA, 1, 1)
    dt = time.perf_counter() - t0
    return dt, uh, u, it, pe


def cpu_baseline(target_s: float = 12.0):
    from oracle import oracle as O
    O.build()
    dt, *_ = oracle_time(256, first=1 << 40)
    rate = 256 / max(dt, 1e-6)
    count = int(min(60000, max(512, rate * target_s)))
    dt, uh, u, it, pe = oracle_time(count, first=1 << 40)
    value = count * K / dt / 1e9
    # the single-core figure on a tenth of the sample
    fz, _, llr1 = oracle_inputs(max(64, count // 10), 1 << 40)
    t0 = time.perf_counter()
    O.decode_batch(fz, llr1, MAX_ITER, ALPHA, 1, 1, nthreads=1)
    dt1 = time.perf_counter() - t0
    return {"value": value, "unit": "Gbit/s", "cores": O.max_threads(), "kind": "oracle",
            "sample": (f"{count} codewords of the same workload ((1024,512), 3.0 dB, G-matrix stop + CSFG "
                       f"freezing, max 60 iterations), FP64 oracle threaded over codewords, {dt:.1f} s"),
            "avg_iters": float(it.mean()),
            "single_core": {"value": llr1.shape[0] * K / dt1 / 1e9, "unit": "Gbit/s",
                            "codewords_per_s": llr1.shape[0] / dt1, "sample": f"{llr1.shape[0]} codewords, 1 thread"}}


def oracle_code_sample(N: int, K: int, idx, ebn0, max_iter: int, seed: int):
    """Time the FP64 oracle (threaded over codewords) on the host-generated codewords `idx` of an
    (N, K) code, G-matrix stop + CSFG freezing; ebn0 is a scalar or one value per codeword."""
    from oracle import oracle as O
    from paper_1505_04979_gb300 import inputs as I
    fz = O.bec_frozen(N, K)
    idx = np.asarray(idx)
    u = I.info_bits(seed, idx, fz)
    x = O.encode(u)
    llr = I.channel_llr(x, I.gaussian(seed, idx, N), I.sigma(ebn0, K / N))
    t0 = time.perf_counter()
    O.decode_batch(fz, llr, max_iter, ALPHA, 1, 1)
    return time.perf_counter() - t0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import oracle as O
    O.build()
    dt, *_ = oracle_time(128, first=1 << 41)
    rate = 128 / max(dt, 1e-6)
    per_step = int(min(4096, max(64, rate * 4.0)))
    total_t, total_cw = 0.0, 0
    for s in range(args.warmup + args.steps):
        dt, *_ = oracle_time(per_step, first=(1 << 41) + s * per_step)
        if s >= args.warmup:
            total_t += dt
            total_cw += per_step
    value = total_cw * K / total_t / 1e9
    cores = O.max_threads()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Gbit/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_t / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(per_step),
            "cpu_baseline": {"value": value, "unit": "Gbit/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} codewords per step of the same workload on {cores} host threads"},
            "e2e": {"value": value, "unit": "Gbit/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(batch: int):
    return {"workload": (f"polar ({N},{K}) BP decoding, BPSK/AWGN Eb/N0 {EBN0} dB, {batch} codewords per step "
                         f"per GPU, scaled min-sum alpha {ALPHA}, max {MAX_ITER} iterations, G-matrix stop + CSFG "
                         "freezing"),
            "N": N, "K": K, "ebn0_db": EBN0, "codewords_per_step": batch, "max_iter": MAX_ITER, "alpha": ALPHA,
            "frozen_set": "BEC(0.5) Bhattacharyya", "l2": "inputs larger than L2 (4 B x N per codeword), no flush"}


# ---------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------
def time_mode(B, code, llr, outs, mode, steps, warmup, stream):
    import torch
    uh, it, pe = outs
    for _ in range(warmup):
        B.polarbp_decode(code, llr, MAX_ITER, ALPHA, *mode, uh, it, pe, stream=stream)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(steps):
        B.polarbp_decode(code, llr, MAX_ITER, ALPHA, *mode, uh, it, pe, stream=stream)
    e.record(stream)
    torch.cuda.synchronize()
    return s.elapsed_time(e)


def run_ours(args):
    import torch
    from paper_1505_04979_gb300 import binding as B
    from paper_1505_04979_gb300 import build
    rank, local, world = dist_setup(args.gpus)
    if world == 1:
        build.build()
    else:
        if rank == 0:
            build.build()
        barrier(world)
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    batch = args.batch
    code = B.polarbp_construct(N, K)
    first = shard_first(rank, batch)
    u, llr = B.polarbp_awgn(code, SEED, first, batch, EBN0)
    uh = torch.empty((batch, N), dtype=torch.uint8, device="cuda")
    it = torch.empty(batch, dtype=torch.int32, device="cuda")
    pe = torch.empty(batch, dtype=torch.int64, device="cuda")
    outs = (uh, it, pe)
    main = MODES["gstop_freeze"]

    # warm-up, then the timed steps of the headline mode
    for _ in range(args.warmup):
        B.polarbp_decode(code, llr, MAX_ITER, ALPHA, *main, uh, it, pe, stream=stream)
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            B.polarbp_decode(code, llr, MAX_ITER, ALPHA, *main, uh, it, pe, stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms_total = max_over_ranks(ev0.elapsed_time(ev1), world)
    ms_step = ms_total / args.steps
    gpu_launches = args.steps

    per_mode = {}
    stats_local = {}
    for name, mode in MODES.items():
        if name == "gstop_freeze":
            ms = ms_step
        elif args.only_main:
            continue
        else:
            ms = time_mode(B, code, llr, outs, mode, args.mode_steps, 1, stream) / args.mode_steps
            ms = max_over_ranks(ms, world)
        B.polarbp_decode(code, llr, MAX_ITER, ALPHA, *mode, uh, it, pe, stream=stream)
        torch.cuda.synchronize()
        errs = int((uh != u).any(dim=1).sum().item())
        bit_errs = int((uh != u).sum().item())
        sums = sum_over_ranks([errs, bit_errs, float(it.double().sum().item()), float(pe.double().sum().item())],
                              world)
        n_cw = batch * world
        fer = sums[0] / n_cw
        lo, hi = wilson(int(sums[0]), n_cw)
        pe_cw = sums[3] / n_cw
        gbit = n_cw * K / (ms * 1e-3) / 1e9
        pe_rate = n_cw * pe_cw / (ms * 1e-3)
        per_mode[name] = {"info_gbit_s": gbit, "ms_per_step": ms, "fer": fer, "fer_ci95": [lo, hi],
                          "ber": sums[1] / (n_cw * K), "avg_iters": sums[2] / n_cw, "pe_per_codeword": pe_cw,
                          "pe_per_s": pe_rate, "alu_frac": pe_rate / world / PEAK_PE_PER_S}
        stats_local[name] = pe_cw

    # end-to-end through the host entry point: H2D of the LLRs and D2H of the results every step
    e2e = None
    if not args.skip_e2e:
        h_llr = torch.empty((batch, N), dtype=torch.float32, pin_memory=True)
        h_llr.copy_(llr)
        h_u = torch.empty((batch, N), dtype=torch.uint8).pin_memory()
        h_it = torch.empty(batch, dtype=torch.int32).pin_memory()
        h_pe = torch.empty(batch, dtype=torch.int64).pin_memory()
        ws = torch.empty(B.polarbp_decode_host_workspace(code, batch), dtype=torch.uint8, device="cuda")
        e2e_steps = max(1, min(args.steps, 5))
        B.polarbp_decode_host(code, h_llr, MAX_ITER, ALPHA, *main, h_u, h_it, h_pe, ws, stream=stream)
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            B.polarbp_decode_host(code, h_llr, MAX_ITER, ALPHA, *main, h_u, h_it, h_pe, ws, stream=stream)
        dt = max_over_ranks(time.perf_counter() - t0, world)
        # the host entry point decodes a large batch as a pipeline of chunks of 64 MiB of
        # LLRs, one kernel launch each (a smaller batch is one launch)
        cb = max(1, (64 << 20) // (N * 4))
        launches_per_call = -(-batch // cb) if batch >= 2 * cb else 1
        e2e = {"value": batch * world * K * e2e_steps / dt / 1e9, "unit": "Gbit/s",
               "h2d_bytes_per_step": batch * N * 4, "d2h_bytes_per_step": batch * (N + 4 + 8),
               "steps": e2e_steps, "entry_point": "polarbp_decode_host",
               "gpu_launches": launches_per_call * e2e_steps}
        del h_llr, h_u, h_it, h_pe, ws

    if rank != 0:
        return 0
    head = per_mode["gstop_freeze"]
    achieved = head["pe_per_s"] / world
    traffic = kernel_traffic()
    line = {
        "metric": METRIC, "value": head["info_gbit_s"], "unit": "Gbit/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": workload_config(batch),
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": PEAK_PE_PER_S / 1e9, "unit": "GPE/s",
                     "frac": achieved / PEAK_PE_PER_S,
                     "traffic": None if traffic is None else traffic,
                     "kernel": "bp_decode_pipe_kernel<10, GSTOP>",
                     "peak_basis": (f"{SMS} SMs x {LANES} lanes x {SM_MAX_HZ / 1e6:.0f} MHz / {OPS_PER_PE} "
                                    "lane instructions per PE update"),
                     "algorithmic_bytes_per_launch": batch * (4 * N + N + 12)},
        "modes": per_mode,
        "equal_fer": equal_fer(per_mode) if all(m in per_mode for m in ("fixed", "gstop", "gstop_freeze")) else None,
        "gpu_launches": gpu_launches,
        "clocks": clk.summary(),
        "e2e": e2e,
    }
    if world == 1 and not args.skip_cpu:
        line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    print(json.dumps(line), flush=True)
    return 0


def equal_fer(per_mode):
    """The metric's comparison made explicit: G-stop + freezing against fixed iterations and
    against G-stop alone on the same codewords, with the Wilson 95 % intervals of their FER
    (disjoint intervals mean the FERs differ) and the throughput ratio."""
    head = per_mode["gstop_freeze"]
    out = {}
    for other in ("fixed", "gstop"):
        o = per_mode[other]
        lo_h, hi_h = head["fer_ci95"]
        lo_o, hi_o = o["fer_ci95"]
        out[f"vs_{other}"] = {
            "fer": head["fer"], "fer_other": o["fer"],
            "ci_overlap": not (hi_h < lo_o or hi_o < lo_h),
            "fer_lower": head["fer"] < o["fer"],
            "throughput_ratio": head["info_gbit_s"] / o["info_gbit_s"],
        }
    return out


MIXED_CLASSES = [(256, 64), (256, 128), (256, 192), (1024, 256), (1024, 512), (1024, 768), (4096, 1024),
                 (4096, 2048), (4096, 3072)]


def run_mixed(args):
    """Mixed stream: 2^20 codewords, each drawing N from {256, 1024, 4096}, rate from
    {1/4, 1/2, 3/4} and Eb/N0 from U[1.5, 3.5] dB; G-matrix stop + CSFG freezing, max 60
    iterations; one persistent launch per code length, captured in a CUDA graph."""
    import torch
    from paper_1505_04979_gb300 import binding as B
    from paper_1505_04979_gb300 import build
    from paper_1505_04979_gb300 import inputs as I
    build.build()
    torch.cuda.set_device(0)
    total = args.batch
    seed = SEED + 2
    idx = np.arange(total)
    cls = I.choice(seed, idx, len(MIXED_CLASSES), which=1)
    segs, us, info_bits, cpcs = [], [], 0, {}
    for k, (n_, k_) in enumerate(MIXED_CLASSES):
        members = idx[cls == k]
        code = B.polarbp_construct(n_, k_)
        cpc = B.polarbp_autotune(code, MAX_ITER)
        mapping = "pipelined" if B.polarbp_get_thread_mapping(code) == B.POLARBP_MAP_PIPELINED else "block"
        cpcs[f"{n_},{k_}"] = {"codewords_per_block": cpc, "thread_mapping": mapping}
        ebn0 = torch.from_numpy(I.uniform(seed, members, 1.5, 3.5).astype(np.float32)).cuda()
        u, llr = B.polarbp_awgn_ebn0(code, seed, int(members[0]) if len(members) else 0, ebn0)
        n = len(members)
        segs.append((code, llr, torch.empty((n, n_), dtype=torch.uint8, device="cuda"),
                     torch.empty(n, dtype=torch.int32, device="cuda"), torch.empty(n, dtype=torch.int64, device="cuda")))
        us.append(u)
        info_bits += k_ * n
    ws = torch.empty(B.polarbp_decode_segments_workspace(), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    B.polarbp_decode_segments(segs, MAX_ITER, ALPHA, 1, 1, workspace=ws, stream=stream)
    torch.cuda.synchronize()

    def timed(fn, steps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / steps

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        B.polarbp_decode_segments(segs, MAX_ITER, ALPHA, 1, 1, workspace=ws, stream=torch.cuda.current_stream())
    with ClockSampler(0) as clk:
        ms_graph = timed(g.replay, args.steps)
    ms_persist = timed(lambda: B.polarbp_decode_segments(segs, MAX_ITER, ALPHA, 1, 1, workspace=ws, stream=stream),
                       max(3, args.steps // 4))

    def per_class():
        for code, llr, uh, it, pe in segs:
            B.polarbp_decode(code, llr, MAX_ITER, ALPHA, 1, 1, uh, it, pe, stream=stream)
    ms_plain = timed(per_class, max(3, args.steps // 4))

    # the whole stream in one persistent launch (blocks split longest length first)
    B.polarbp_decode_mixed(segs, MAX_ITER, ALPHA, 1, 1, workspace=ws, stream=stream)
    torch.cuda.synchronize()
    g1 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g1):
        B.polarbp_decode_mixed(segs, MAX_ITER, ALPHA, 1, 1, workspace=ws, stream=torch.cuda.current_stream())
    with ClockSampler(0) as clk1:
        ms_one = timed(g1.replay, args.steps)
    ms_one_unc = timed(lambda: B.polarbp_decode_mixed(segs, MAX_ITER, ALPHA, 1, 1, workspace=ws, stream=stream),
                       max(3, args.steps // 4))
    ms_per_len = ms_graph
    one_launch = ms_one < ms_graph
    if one_launch:
        ms_graph, clk = ms_one, clk1
        g1.replay()
    else:
        g.replay()
    torch.cuda.synchronize()
    per = {}
    pe_total = 0.0
    for (n_, k_), (code, llr, uh, it, pe), u in zip(MIXED_CLASSES, segs, us):
        n = uh.shape[0]
        errs = int((uh != u).any(dim=1).sum().item())
        pe_total += float(pe.double().sum().item())
        per[f"N={n_},K={k_}"] = {"codewords": n, "fer": errs / max(n, 1), "fer_ci95": list(wilson(errs, n)),
                                 "avg_iters": float(it.double().mean().item()),
                                 "pe_per_codeword": float(pe.double().mean().item())}
    line = {"metric": "info Gbit/s/GB300, mixed stream (N in {256,1024,4096}, R in {1/4,1/2,3/4}, Eb/N0 U[1.5,3.5])",
            "value": info_bits / (ms_graph * 1e-3) / 1e9, "unit": "Gbit/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"mixed stream, {total} codewords per step, G-matrix stop + CSFG freezing, "
                                   f"max {MAX_ITER} iterations, "
                                   + ("one persistent launch for all lengths (polarbp_decode_mixed)" if one_launch
                                      else "one persistent launch per length (polarbp_decode_segments)")
                                   + " in a CUDA graph, the faster of the two",
                       "autotuned": cpcs},
            "variants_ms_per_step": {"one_launch_graph": ms_one, "one_launch_uncaptured": ms_one_unc,
                                     "per_length_graph": ms_per_len,
                                     "per_length_uncaptured": ms_persist,
                                     "one_block_per_codeword": ms_plain},
            "roofline": {"bound": "alu", "achieved": pe_total / (ms_graph * 1e-3) / 1e9,
                         "peak": PEAK_PE_PER_S / 1e9, "unit": "GPE/s",
                         "frac": pe_total / (ms_graph * 1e-3) / PEAK_PE_PER_S},
            "classes": per, "clocks": clk.summary(),
            "gpu_launches": args.steps * (1 if one_launch else len({c[0] for c in MIXED_CLASSES}))}
    if not args.skip_cpu:
        # the oracle on a sample of the same stream: the first codewords of each class
        from oracle import oracle as O
        from paper_1505_04979_gb300 import inputs as I
        O.build()
        bits, secs, ncw = 0.0, 0.0, 0
        for k, (n_, k_) in enumerate(MIXED_CLASSES):
            members = idx[cls == k][: max(8, 16384 // n_)]
            eb = I.uniform(seed, members, 1.5, 3.5)
            dt = oracle_code_sample(n_, k_, members, eb, MAX_ITER, seed)
            bits += k_ * len(members)
            secs += dt
            ncw += len(members)
        line["cpu_baseline"] = {"value": bits / secs / 1e9, "unit": "Gbit/s", "cores": O.max_threads(),
                                "kind": "oracle",
                                "sample": (f"{ncw} codewords of the stream (the first of each class), FP64 oracle "
                                           f"threaded over codewords, {secs:.1f} s")}
    print(json.dumps(line), flush=True)
    return 0


def run_bitrev(args):
    """Natural against bit-reversed codeword order (x = u B_N F^{(x)m}) on the benchmark's code and
    mode ((1024,512), 3.0 dB, G-matrix stop + CSFG freezing, max 60 iterations), --batch
    codewords per order from the device generator (the same source bits and noise, the channel
    positions permuted): FER with Wilson 95 % intervals, average iterations, PE updates per
    codeword and info Gbit/s.  B_N only permutes the channel positions, so the two rows must
    agree within their intervals."""
    import torch
    from paper_1505_04979_gb300 import binding as B
    from paper_1505_04979_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n_cw = args.batch
    rows = {}
    with ClockSampler(0) as clk:
        for order in ("natural", "bit_reversed"):
            code = B.polarbp_construct(N, K)
            code.set_bit_reversed(order == "bit_reversed")
            u, llr = B.polarbp_awgn(code, SEED + 13, 0, n_cw, EBN0)
            uh = torch.empty((n_cw, N), dtype=torch.uint8, device="cuda")
            it = torch.empty(n_cw, dtype=torch.int32, device="cuda")
            pe = torch.empty(n_cw, dtype=torch.int64, device="cuda")
            for _ in range(max(1, args.warmup)):
                B.polarbp_decode(code, llr, MAX_ITER, ALPHA, 1, 1, uh, it, pe, stream=stream)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            steps = max(1, min(args.steps, 5))
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(steps):
                B.polarbp_decode(code, llr, MAX_ITER, ALPHA, 1, 1, uh, it, pe, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / steps
            errs = int((uh != u).any(dim=1).sum().item())
            rows[order] = {"fer": errs / n_cw, "fer_ci95": list(wilson(errs, n_cw)),
                           "avg_iters": float(it.double().mean().item()),
                           "pe_per_codeword": float(pe.double().mean().item()),
                           "info_gbit_s": n_cw * K / (ms * 1e-3) / 1e9, "ms": ms}
            del u, llr, uh, it, pe
            code.close()
    line = {"metric": "natural vs bit-reversed codeword order, (1024,512) 3.0 dB, G-stop + freezing",
            "unit": "Gbit/s", "value": rows["bit_reversed"]["info_gbit_s"], "n_gpus": 1, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"(1024,512) code, {n_cw} codewords per order, max {MAX_ITER} iterations"},
            "orders": rows, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    return 0


def run_sweep(args):
    """FER sweep of the (1024,512) code: Eb/N0 1.0 .. 3.5 dB in 0.5 dB steps, the four modes
    (fixed iterations, G-matrix stop, freezing alone, G-matrix stop + freezing) at max 60
    iterations on the same codewords, 10^6 codewords per point (device generator), and the four
    modes at max 40 iterations at 2.5 / 3.0 / 3.5 dB (the paper's setting is 40 at 3 dB), with
    freezing's iteration and PE-update changes against plain BP and the G-matrix stop."""
    import torch
    from paper_1505_04979_gb300 import binding as B
    from paper_1505_04979_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    n_cw = args.sweep_codewords
    code = B.polarbp_construct(N, K)
    stream = torch.cuda.current_stream()
    uh = torch.empty((n_cw, N), dtype=torch.uint8, device="cuda")
    it = torch.empty(n_cw, dtype=torch.int32, device="cuda")
    pe = torch.empty(n_cw, dtype=torch.int64, device="cuda")
    modes = MODES
    points = []
    with ClockSampler(0) as clk:
        for eb, mi in [(e, MAX_ITER) for e in (1.0, 1.5, 2.0, 2.5, 3.0, 3.5)] + [(e, 40) for e in (2.5, 3.0, 3.5)]:
            u, llr = B.polarbp_awgn(code, SEED + 7, 0, n_cw, eb)
            row = {"ebn0_db": eb, "max_iter": mi, "codewords": n_cw}
            for name, mode in modes.items():
                B.polarbp_decode(code, llr, mi, ALPHA, *mode, uh, it, pe, stream=stream)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                B.polarbp_decode(code, llr, mi, ALPHA, *mode, uh, it, pe, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                errs = int((uh != u).any(dim=1).sum().item())
                bit_errs = int((uh != u).sum().item())
                pe_sum = float(pe.double().sum().item())
                row[name] = {"fer": errs / n_cw, "fer_ci95": list(wilson(errs, n_cw)), "ber": bit_errs / (n_cw * K),
                             "avg_iters": float(it.double().mean().item()), "pe_per_codeword": pe_sum / n_cw,
                             "info_gbit_s": n_cw * K / (ms * 1e-3) / 1e9, "ms": ms,
                             "alu_frac": pe_sum / (ms * 1e-3) / PEAK_PE_PER_S}
            # the paper's comparison (Sec. IV): freezing against plain BP with max_iter fixed
            # iterations and against the G-matrix stop, in average iterations and PE updates
            row["freeze_vs_fixed"] = {"iterations": row["freeze"]["avg_iters"] / row["fixed"]["avg_iters"] - 1.0,
                                      "pe_updates": row["freeze"]["pe_per_codeword"] / row["fixed"]["pe_per_codeword"] - 1.0}
            row["freeze_vs_gstop"] = {"iterations": row["freeze"]["avg_iters"] / row["gstop"]["avg_iters"] - 1.0,
                                      "pe_updates": row["freeze"]["pe_per_codeword"] / row["gstop"]["pe_per_codeword"] - 1.0}
            points.append(row)
            del u, llr
            torch.cuda.empty_cache()
    line = {"metric": "FER / throughput sweep, (1024,512), Eb/N0 1.0-3.5 dB, three modes", "unit": "Gbit/s",
            "value": next(p for p in points if p["ebn0_db"] == 3.0 and p["max_iter"] == MAX_ITER)["gstop_freeze"]["info_gbit_s"],
            "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"(1024,512) code, {n_cw} codewords per point, alpha {ALPHA}, device generator"},
            "points": points, "clocks": clk.summary(), "gpu_launches": 2 * len(modes) * len(points)}
    print(json.dumps(line), flush=True)
    return 0


def run_flooding(args):
    """True flooding schedule (every PE from the previous iteration's messages) against the
    paper's left-to-right sweep, on the same codewords: the tiny-code configuration ((64,32),
    Eb/N0 2.5 dB, 40 fixed iterations, alpha 0.9375; its 1000-codeword case is a parity test,
    here --batch codewords, 2^20 by default, from the device generator) and (1024,512) at
    3.0 dB with the G-matrix stop, max 60 iterations.  FER with Wilson 95 % intervals, average iterations, and info
    Gbit/s timed with CUDA events (K steps after W warm-up steps per line)."""
    import torch
    from oracle import oracle as O
    from paper_1505_04979_gb300 import binding as B
    from paper_1505_04979_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    steps = max(1, min(args.steps, 5))
    cases = [("N=64,K=32,2.5dB,fixed40", 64, 32, 2.5, 40, 0), ("N=1024,K=512,3.0dB,gstop60", 1024, 512, 3.0, 60, 1)]
    out = {}
    with ClockSampler(0) as clk:
        for name, n, k, eb, iters, stop in cases:
            code = B.polarbp_construct(n, k)
            n_cw = args.batch
            u, llr = B.polarbp_awgn(code, SEED + 11, 0, n_cw, eb)
            uh = torch.empty((n_cw, n), dtype=torch.uint8, device="cuda")
            it = torch.empty(n_cw, dtype=torch.int32, device="cuda")
            pe = torch.empty(n_cw, dtype=torch.int64, device="cuda")
            row = {}
            for sched in ("sweep", "flooding"):
                def call():
                    if sched == "sweep":
                        B.polarbp_decode(code, llr, iters, ALPHA, stop, 0, uh, it, pe, stream=stream)
                    else:
                        B.polarbp_decode_flooding(code, llr, iters, ALPHA, stop, uh, it, pe, stream=stream)
                for _ in range(max(1, args.warmup)):
                    call()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(steps):
                    call()
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / steps
                errs = int((uh != u).any(dim=1).sum().item())
                pe_sum = float(pe.double().sum().item())
                row[sched] = {"fer": errs / n_cw, "fer_ci95": list(wilson(errs, n_cw)),
                              "avg_iters": float(it.double().mean().item()), "pe_per_codeword": pe_sum / n_cw,
                              "ms_per_step": ms, "info_gbit_s": n_cw * k / (ms * 1e-3) / 1e9,
                              "pe_per_s": pe_sum / (ms * 1e-3), "alu_frac": pe_sum / (ms * 1e-3) / PEAK_PE_PER_S}
            row["codewords"] = n_cw
            out[name] = row
            del u, llr, uh, it, pe
            torch.cuda.empty_cache()
            code.close()
    # oracle (flooding) on a bounded sample of the tiny-code configuration, sized to about 10 s
    O.build()
    from paper_1505_04979_gb300 import inputs as I
    fz = O.bec_frozen(64, 32)

    def oracle_sample(count):
        idx = np.arange(1 << 40, (1 << 40) + count)
        uu = I.info_bits(SEED, idx, fz)
        ll = I.channel_llr(O.encode(uu), I.gaussian(SEED, idx, 64), I.sigma(2.5, 0.5))
        t0 = time.perf_counter()
        O.decode_flood_batch(fz, ll, 40, ALPHA, 0)
        return time.perf_counter() - t0

    probe = 20000
    rate = probe / max(oracle_sample(probe), 1e-6)
    n_cpu = int(min(1 << 20, max(probe, rate * 10.0)))
    dt = oracle_sample(n_cpu)
    head = out["N=64,K=32,2.5dB,fixed40"]["flooding"]
    line = {"metric": "info Gbit/s/GB300, true flooding schedule vs the paper's sweep", "unit": "Gbit/s",
            "value": head["info_gbit_s"], "n_gpus": 1, "steps": steps, "warmup": max(1, args.warmup),
            "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "flooding schedule: (64,32) 2.5 dB 40 fixed iterations and (1024,512) 3.0 dB "
                                   f"G-matrix stop max 60, {args.batch} codewords each, alpha 0.9375, device generator",
                       "l2": f"LLR inputs of {args.batch * 1024 * 4 >> 20} MiB at N=1024 and "
                             f"{args.batch * 64 * 4 >> 20} MiB at N=64 (L2 is 129 MB), no flush"},
            "cases": out, "clocks": clk.summary(), "gpu_launches": 2 * len(cases) * (steps + max(1, args.warmup)),
            "cpu_baseline": {"value": n_cpu * 32 / dt / 1e9, "unit": "Gbit/s", "cores": O.max_threads(),
                             "kind": "oracle", "sample": f"{n_cpu} codewords of (64,32) at 2.5 dB, 40 flooding "
                                                         f"iterations, FP64 oracle threaded over codewords, {dt:.1f} s"}}
    print(json.dumps(line), flush=True)
    return 0


def run_readings(args):
    """The freezing order of Sec. III under reading A (one check per stage per iteration, the
    decoder's default) and reading B (checks continue along a stage while they pass), with the
    G-matrix stop, on the same (1024,512) codewords at 2.5, 3.0 and 3.5 dB, max 60 iterations:
    FER with Wilson 95 % intervals, iterations, PE updates per codeword and info Gbit/s."""
    import torch
    from paper_1505_04979_gb300 import binding as B
    from paper_1505_04979_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n_cw = args.batch
    code = B.polarbp_construct(N, K)
    uh = torch.empty((n_cw, N), dtype=torch.uint8, device="cuda")
    it = torch.empty(n_cw, dtype=torch.int32, device="cuda")
    pe = torch.empty(n_cw, dtype=torch.int64, device="cuda")
    points = []
    with ClockSampler(0) as clk:
        for eb in (2.5, 3.0, 3.5):
            u, llr = B.polarbp_awgn(code, SEED + 13, 0, n_cw, eb)
            row = {"ebn0_db": eb, "codewords": n_cw}
            for name, fm in (("reading_A", 1), ("reading_B", 2)):
                B.polarbp_decode(code, llr, MAX_ITER, ALPHA, 1, fm, uh, it, pe, stream=stream)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                B.polarbp_decode(code, llr, MAX_ITER, ALPHA, 1, fm, uh, it, pe, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                errs = int((uh != u).any(dim=1).sum().item())
                pe_sum = float(pe.double().sum().item())
                row[name] = {"fer": errs / n_cw, "fer_ci95": list(wilson(errs, n_cw)),
                             "avg_iters": float(it.double().mean().item()), "pe_per_codeword": pe_sum / n_cw,
                             "info_gbit_s": n_cw * K / (ms * 1e-3) / 1e9, "ms": ms,
                             "alu_frac": pe_sum / (ms * 1e-3) / PEAK_PE_PER_S}
            # the paper's comparison (Sec. IV): freezing against plain BP with max_iter fixed
            # iterations and against the G-matrix stop, in average iterations and PE updates
            row["freeze_vs_fixed"] = {"iterations": row["freeze"]["avg_iters"] / row["fixed"]["avg_iters"] - 1.0,
                                      "pe_updates": row["freeze"]["pe_per_codeword"] / row["fixed"]["pe_per_codeword"] - 1.0}
            row["freeze_vs_gstop"] = {"iterations": row["freeze"]["avg_iters"] / row["gstop"]["avg_iters"] - 1.0,
                                      "pe_updates": row["freeze"]["pe_per_codeword"] / row["gstop"]["pe_per_codeword"] - 1.0}
            points.append(row)
            del u, llr
            torch.cuda.empty_cache()
    head = next(p for p in points if p["ebn0_db"] == 3.0)["reading_B"]
    line = {"metric": "freezing order readings A and B, (1024,512), G-matrix stop, FER / PE updates / Gbit/s",
            "unit": "Gbit/s", "value": head["info_gbit_s"], "n_gpus": 1, "steps": 1, "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"(1024,512) code, {n_cw} codewords per point, alpha {ALPHA}, max 60 "
                                   "iterations, device generator"},
            "points": points, "clocks": clk.summary(), "gpu_launches": 2 * 2 * len(points)}
    print(json.dumps(line), flush=True)
    return 0


def run_quantized(args):
    """Quantised 16-bit messages (fixed-point variant) against binary32 messages on the same
    (1024,512) codewords at 2.5 and 3.0 dB, G-matrix stop, max 60 iterations, alpha 0.9375 (A = 15),
    2, 3 and 5 fractional bits: FER with Wilson 95 % intervals, iterations and info Gbit/s."""
    import torch
    from paper_1505_04979_gb300 import binding as B
    from paper_1505_04979_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    n_cw = args.batch
    code = B.polarbp_construct(N, K)
    uh = torch.empty((n_cw, N), dtype=torch.uint8, device="cuda")
    it = torch.empty(n_cw, dtype=torch.int32, device="cuda")
    pe = torch.empty(n_cw, dtype=torch.int64, device="cuda")
    points = []
    with ClockSampler(0) as clk:
        for eb in (2.5, 3.0):
            u, llr = B.polarbp_awgn(code, SEED + 17, 0, n_cw, eb)
            row = {"ebn0_db": eb, "codewords": n_cw}
            variants = [("binary32", None)] + [(f"int16_F{f}", f) for f in (2, 3, 5)]
            for name, F in variants:
                def call():
                    if F is None:
                        B.polarbp_decode(code, llr, MAX_ITER, ALPHA, 1, 0, uh, it, pe, stream=stream)
                    else:
                        B.polarbp_decode_quantized(code, llr, MAX_ITER, 15, F, 1, uh, it, pe, stream=stream)
                call()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                call()
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1)
                errs = int((uh != u).any(dim=1).sum().item())
                pe_sum = float(pe.double().sum().item())
                row[name] = {"fer": errs / n_cw, "fer_ci95": list(wilson(errs, n_cw)),
                             "avg_iters": float(it.double().mean().item()), "ms": ms,
                             "info_gbit_s": n_cw * K / (ms * 1e-3) / 1e9,
                             "pe_per_s": pe_sum / (ms * 1e-3), "alu_frac": pe_sum / (ms * 1e-3) / PEAK_PE_PER_S}
            # the paper's comparison (Sec. IV): freezing against plain BP with max_iter fixed
            # iterations and against the G-matrix stop, in average iterations and PE updates
            row["freeze_vs_fixed"] = {"iterations": row["freeze"]["avg_iters"] / row["fixed"]["avg_iters"] - 1.0,
                                      "pe_updates": row["freeze"]["pe_per_codeword"] / row["fixed"]["pe_per_codeword"] - 1.0}
            row["freeze_vs_gstop"] = {"iterations": row["freeze"]["avg_iters"] / row["gstop"]["avg_iters"] - 1.0,
                                      "pe_updates": row["freeze"]["pe_per_codeword"] / row["gstop"]["pe_per_codeword"] - 1.0}
            points.append(row)
            del u, llr
            torch.cuda.empty_cache()
    head = next(p for p in points if p["ebn0_db"] == 3.0)["int16_F3"]
    line = {"metric": "info Gbit/s/GB300, 16-bit quantised messages vs binary32, (1024,512), G-matrix stop",
            "unit": "Gbit/s", "value": head["info_gbit_s"], "n_gpus": 1, "steps": 1, "warmup": 1,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int16", "data": "synthetic",
            "config": {"workload": f"(1024,512) code, {n_cw} codewords per point, alpha 15/16, max 60 iterations, "
                                   "G-matrix stop, device generator"},
            "points": points, "clocks": clk.summary(), "gpu_launches": 2 * 4 * len(points)}
    print(json.dumps(line), flush=True)
    return 0


def run_long(args):
    """Long codes: N in {8192, 16384, 32768}, K = N/2, Eb/N0 in {2.0, 2.5, 3.0} dB, 10^5
    codewords per point (device generator), G-matrix stop + CSFG freezing, at most 100
    iterations; one codeword per thread-block cluster of N/4096 blocks."""
    import torch
    from paper_1505_04979_gb300 import binding as B
    from paper_1505_04979_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    n_cw = args.long_codewords
    stream = torch.cuda.current_stream()
    points, tot_bits, tot_ms, tot_pe = {}, 0.0, 0.0, 0.0
    with ClockSampler(0) as clk:
        for N in ((args.long_n,) if args.long_n else (8192, 16384, 32768)):
            K = N // 2
            code = B.polarbp_construct(N, K)
            for eb in ((args.long_ebn0,) if args.long_ebn0 is not None else (2.0, 2.5, 3.0)):
                u, llr = B.polarbp_awgn(code, SEED + 3, 0, n_cw, eb)
                uh = torch.empty((n_cw, N), dtype=torch.uint8, device="cuda")
                it = torch.empty(n_cw, dtype=torch.int32, device="cuda")
                pe = torch.empty(n_cw, dtype=torch.int64, device="cuda")
                for _ in range(args.warmup):
                    B.polarbp_decode(code, llr, 100, ALPHA, 1, 1, uh, it, pe, stream=stream)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(args.steps):
                    B.polarbp_decode(code, llr, 100, ALPHA, 1, 1, uh, it, pe, stream=stream)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / args.steps
                errs = int((uh != u).any(dim=1).sum().item())
                pe_sum = float(pe.double().sum().item())
                points[f"N={N},{eb}dB"] = {
                    "codewords": n_cw, "ms": ms, "info_gbps": K * n_cw / (ms * 1e-3) / 1e9,
                    "codewords_per_s": n_cw / (ms * 1e-3), "fer": errs / n_cw, "fer_ci95": list(wilson(errs, n_cw)),
                    "avg_iters": float(it.double().mean().item()), "pe_per_codeword": pe_sum / n_cw,
                    "gpe_per_s": pe_sum / (ms * 1e-3) / 1e9}
                tot_bits += K * n_cw
                tot_ms += ms
                tot_pe += pe_sum
                del u, llr, uh, it, pe
                torch.cuda.empty_cache()
    cpu = None
    if not args.skip_cpu:
        from oracle import oracle as O
        O.build()
        bits, secs, parts = 0.0, 0.0, []
        for N, cnt in ((8192, 64), (16384, 32), (32768, 16)):
            dt = oracle_code_sample(N, N // 2, np.arange(cnt), 2.5, 100, SEED + 3)
            bits += cnt * (N // 2)
            secs += dt
            parts.append(f"{cnt} x N={N}")
        cpu = {"value": bits / secs / 1e9, "unit": "Gbit/s", "cores": O.max_threads(), "kind": "oracle",
               "sample": (", ".join(parts) + " codewords at 2.5 dB, G-matrix stop + CSFG freezing, max 100 "
                          f"iterations, FP64 oracle threaded over codewords, {secs:.1f} s")}
    line = {"metric": "info Gbit/s/GB300, long codes N in {8192,16384,32768}, Eb/N0 {2.0,2.5,3.0} dB",
            "value": tot_bits / (tot_ms * 1e-3) / 1e9, "unit": "Gbit/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tot_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"long codes, K=N/2, {n_cw} codewords per point, {len(points)} points per step, "
                                   "G-matrix stop + CSFG freezing, max 100 iterations, thread-block clusters",
                       "l2": "inputs larger than L2 (13 GB of LLRs at N=32768)"},
            "roofline": {"bound": "alu", "achieved": tot_pe / (tot_ms * 1e-3) / 1e9, "peak": PEAK_PE_PER_S / 1e9,
                         "unit": "GPE/s", "frac": tot_pe / (tot_ms * 1e-3) / PEAK_PE_PER_S},
            "points": points, "clocks": clk.summary(), "gpu_launches": len(points) * args.steps, "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)
    return 0


def run_wms(args):
    """Learned weighted min-sum: per-(iteration, stage, PE) weights, 10 unrolled iterations,
    N in {128, 256}, K = N/2, training batches of 4096 codewords at Eb/N0 ~ U[1, 4] dB, BCE on
    the information positions, Adam; then FER of the learned weights against constant 0.9375."""
    import torch
    from paper_1505_04979_gb300 import binding as B
    from paper_1505_04979_gb300 import build
    from paper_1505_04979_gb300 import inputs as I
    build.build()
    torch.cuda.set_device(0)
    T, batch = 10, 4096
    hbm = 6794.8e9
    try:
        hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"] * 1e9
    except (OSError, KeyError, ValueError):
        pass
    results = {}
    stream = torch.cuda.current_stream()
    for N in (128, 256):
        K = N // 2
        m = N.bit_length() - 1
        code = B.polarbp_construct(N, K)
        info = torch.from_numpy(np.nonzero(code.frozen_mask() == 0)[0]).cuda()
        w = torch.full((T, m, N // 2), ALPHA, dtype=torch.float32, device="cuda", requires_grad=True)
        opt = torch.optim.Adam([w], lr=args.wms_lr)
        kk = args.wms_k
        ws = torch.empty(B.polarbp_wms_workspace(code, batch, T, kk), dtype=torch.uint8, device="cuda")
        losses, fwd_ms, bwd_ms = [], 0.0, 0.0
        e0, e1, e1b, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        for step in range(args.wms_steps):
            ebn0 = torch.from_numpy(I.uniform(SEED + 5, np.arange(step * batch, (step + 1) * batch), 1.0, 4.0)
                                    .astype(np.float32)).cuda()
            u, llr = B.polarbp_awgn_ebn0(code, SEED + 5, step * batch, ebn0)
            target = u[:, info].float()
            opt.zero_grad()
            e0.record(stream)
            out = B.polarbp_wms_forward(code, llr, w.detach(), ws, checkpoint_every=kk)
            e1.record(stream)
            x = (-out[:, info]).detach().requires_grad_(True)
            loss = torch.nn.functional.binary_cross_entropy_with_logits(x, target)
            loss.backward()
            dout = torch.zeros((batch, N), dtype=torch.float32, device="cuda")
            dout[:, info] = -x.grad
            e1b.record(stream)
            dw, _ = B.polarbp_wms_backward(code, llr, w.detach(), dout, ws, checkpoint_every=kk)
            e2.record(stream)
            w.grad = dw
            opt.step()
            torch.cuda.synchronize()
            if step >= 3:
                fwd_ms += e0.elapsed_time(e1)
                bwd_ms += e1b.elapsed_time(e2)
            losses.append(float(loss.detach()))
        timed = max(1, args.wms_steps - 3)
        fwd_ms /= timed
        bwd_ms /= timed
        def wms_bytes(k):
            """Algorithmic bytes per batch: LLRs in and soft outputs out, the checkpoints (both
            planes of every iteration for k = 1, L columns 1..m-1 after every k-th iteration
            otherwise) written by the forward and read by the adjoint, dout in, dllr out and the
            per-codeword weight-gradient partials out."""
            ck = T * 2 * (m + 1) * N * 4 if k == 1 else ((T - 1) // min(k, T)) * (m - 1) * N * 4
            return batch * (4 * N + 4 * N + ck), batch * (ck + 4 * N * 3 + T * m * (N // 2) * 4)

        fwd_bytes, bwd_bytes = wms_bytes(kk)
        # forward and adjoint times against the checkpoint interval, on the last training batch
        ksweep = {}
        for k in (1, 2, 5, 10):
            wsk = torch.empty(B.polarbp_wms_workspace(code, batch, T, k), dtype=torch.uint8, device="cuda")
            fb, bb = wms_bytes(k)
            tf = tb = 0.0
            for rep in range(5):
                e0.record(stream)
                B.polarbp_wms_forward(code, llr, w.detach(), wsk, checkpoint_every=k)
                e1.record(stream)
                B.polarbp_wms_backward(code, llr, w.detach(), dout, wsk, checkpoint_every=k)
                e2.record(stream)
                torch.cuda.synchronize()
                if rep >= 2:
                    tf += e0.elapsed_time(e1) / 3
                    tb += e1.elapsed_time(e2) / 3
            ksweep[f"k={k}"] = {"forward_ms": tf, "backward_ms": tb, "workspace_bytes": wsk.numel(),
                                "forward_hbm_frac": fb / (tf * 1e-3) / hbm, "backward_hbm_frac": bb / (tb * 1e-3) / hbm}
            del wsk
        fer = {}
        with torch.no_grad():
            for eb in (2.0, 3.0, 4.0):
                n_eval, errs_l, errs_c = 0, 0, 0
                wc = torch.full_like(w, ALPHA)
                for chunk in range(args.wms_eval // batch):
                    first = (1 << 30) + chunk * batch
                    u, llr = B.polarbp_awgn(code, SEED + 6, first, batch, eb)
                    for weights, key in ((w.detach(), "learned"), (wc, "constant")):
                        out = B.polarbp_wms_forward(code, llr, weights, ws, checkpoint_every=kk)
                        uh = (out[:, info] < 0).to(torch.uint8)
                        e = int((uh != u[:, info]).any(dim=1).sum().item())
                        if key == "learned":
                            errs_l += e
                        else:
                            errs_c += e
                    n_eval += batch
                fer[f"{eb} dB"] = {"codewords": n_eval, "learned": errs_l / n_eval,
                                   "learned_ci95": list(wilson(errs_l, n_eval)),
                                   "constant_0.9375": errs_c / n_eval,
                                   "constant_ci95": list(wilson(errs_c, n_eval))}
        results[f"N={N}"] = {
            "train_steps": args.wms_steps, "loss_first": losses[0], "loss_last": float(np.mean(losses[-10:])),
            "forward_ms": fwd_ms, "backward_ms": bwd_ms,
            "train_codewords_per_s": batch / ((fwd_ms + bwd_ms) * 1e-3),
            "forward_GBps": fwd_bytes / (fwd_ms * 1e-3) / 1e9, "backward_GBps": bwd_bytes / (bwd_ms * 1e-3) / 1e9,
            "forward_hbm_frac": fwd_bytes / (fwd_ms * 1e-3) / hbm, "backward_hbm_frac": bwd_bytes / (bwd_ms * 1e-3) / hbm,
            "checkpoint_every": kk, "checkpoint_sweep": ksweep, "fer": fer}
    line = {"metric": "weighted min-sum training: codewords/s (forward + adjoint), FER learned vs constant",
            "value": results["N=256"]["train_codewords_per_s"], "unit": "codewords/s", "n_gpus": 1,
            "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"weighted min-sum, T={T}, batch {batch}, Eb/N0 U[1,4] dB, Adam lr {args.wms_lr}"},
            "roofline": {"bound": "hbm", "unit": "GB/s", "peak": hbm / 1e9,
                         "achieved": results["N=256"]["backward_GBps"],
                         "frac": results["N=256"]["backward_hbm_frac"], "kernel": "wms_backward_kernel"},
            "results": results}
    if not args.skip_cpu:
        # the oracle's forward and adjoint (FP64, one thread) on a sample of N = 256 training codewords
        from oracle import oracle as O
        O.build()
        N, K = 256, 128
        m = 8
        fz = O.bec_frozen(N, K)
        idx = np.arange(256)
        u = I.info_bits(SEED + 5, idx, fz)
        x = O.encode(u)
        eb = I.uniform(SEED + 5, idx, 1.0, 4.0)
        llr = I.channel_llr(x, I.gaussian(SEED + 5, idx, N), I.sigma(eb, K / N))
        wts = np.full((T, m, N // 2), ALPHA)
        dout = np.ones(N)
        t0 = time.perf_counter()
        for c in range(len(idx)):
            O.wms_forward(fz, llr[c], wts)
            O.wms_backward(fz, llr[c], wts, dout)
        secs = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": len(idx) / secs, "unit": "codewords/s", "cores": 1, "kind": "oracle",
                                "sample": (f"{len(idx)} training codewords at N=256, T={T}: FP64 oracle forward and "
                                           f"adjoint, one thread, {secs:.1f} s")}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=1 << 20, help="codewords per step per GPU")
    ap.add_argument("--mode-steps", type=int, default=3, help="timed steps of each comparison mode")
    ap.add_argument("--only-main", action="store_true", help="skip the comparison modes")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--sweep-codewords", type=int, default=1000000)
    ap.add_argument("--workload", choices=["n1024", "mixed", "long", "wms", "sweep", "flooding", "readings",
                                           "quantized", "bitrev"],
                    default="n1024",
                    help="n1024: the (1024,512) headline; mixed: the mixed-length stream; long: N = 8192..32768 "
                         "on thread-block clusters; wms: learned weights; sweep: FER over Eb/N0; flooding: the "
                         "true flooding schedule against the sweep; readings: freezing order A against B; "
                         "quantized: 16-bit messages against binary32")
    ap.add_argument("--long-codewords", type=int, default=100000)
    ap.add_argument("--long-n", type=int, default=0, help="one code length of the long workload (default: all)")
    ap.add_argument("--long-ebn0", type=float, default=None, help="one Eb/N0 point of the long workload")
    ap.add_argument("--wms-steps", type=int, default=300)
    ap.add_argument("--wms-lr", type=float, default=0.005)
    ap.add_argument("--wms-k", type=int, default=1, help="checkpoint interval of the weighted min-sum training")
    ap.add_argument("--wms-eval", type=int, default=1 << 17)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    _device_constants()
    if args.workload == "mixed":
        return run_mixed(args)
    if args.workload == "wms":
        return run_wms(args)
    if args.workload == "long":
        return run_long(args)
    if args.workload == "flooding":
        return run_flooding(args)
    if args.workload == "readings":
        return run_readings(args)
    if args.workload == "quantized":
        return run_quantized(args)
    if args.workload == "sweep":
        return run_sweep(args)
    if args.workload == "bitrev":
        return run_bitrev(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
