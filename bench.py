"""Benchmark of the compressed-matrix hot path on GB300.

Default workload (one "step" = one pass of the whole hot path):
  8192 x 8192 int64 count matrices A and B, entries Poisson(lambda = 5)
  (seeds 1303 / 1304), x of length 8192 uniform over the signed 8-bit range,
  s = 7.  Step: pack A, pack B, pack x (width selection + SM pack), unpack A
  to int64, get 2^20 entries of A, C = A + B, D = 7 A, y = A x -- every result
  re-packed at its exact width.  Inputs are generated on the GPU by the
  library's counter-based generator (identical to the host generator used by
  the tests) and stay resident; dense A and B (512 MiB each) are larger than
  L2, so every step streams them from HBM.

Printed: one JSON line (rank 0).  `value` is the step's algorithmic bytes
(the one-pass traffic of each operation: dense int64 read and packed bytes
written for pack, the reverse for unpack, packed inputs plus packed result
for add and scale, packed A plus x and y for matvec, index, value and one
word per gathered entry for get) divided by the
device-timed step time, summed over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "compressed matvec GB/s (% HBM peak); packed matmul int-TOPS; batched vs plain"
N_ROWS = N_COLS = 8192
LAMBDA = 5.0
SCALE = 7
GET_COUNT = 1 << 20
SEED_A, SEED_B = 1303, 1304


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="ccm_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                p = [v.strip() for v in line.split(",")]
                if len(p) < 9:
                    continue
                try:
                    sm.append(float(p[1]))
                    smax.append(float(p[2]))
                except ValueError:
                    continue
                for name, v in zip(names, p[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
class Workload:
    """Device buffers and the step of the default workload (one rank)."""

    def __init__(self, ccm, torch, dev, seed_offset: int):
        import synth
        self.ccm, self.torch, self.dev = ccm, torch, dev
        n = N_ROWS * N_COLS
        self.n = n
        table = torch.from_numpy(synth.poisson_cdf_table(LAMBDA))
        sa, sb = SEED_A + seed_offset, SEED_B + seed_offset
        self.A = ccm.gen_poisson(n, sa, synth.STREAM_A, table, device=dev).view(N_ROWS, N_COLS)
        self.B = ccm.gen_poisson(n, sb, synth.STREAM_B, table, device=dev).view(N_ROWS, N_COLS)
        self.X = ccm.gen_uniform(N_COLS, sa, synth.STREAM_X, -128, 127, device=dev).view(N_COLS, 1)
        self.idx = ccm.gen_uniform(GET_COUNT, sa, synth.STREAM_INDEX, 0, n - 1, device=dev)
        self.seeds = (sa, sb)
        ba, sa = ccm.measure(self.A)
        bb, sb = ccm.measure(self.B)
        bx, sx = ccm.measure(self.X)
        L = ccm.lib()
        # outputs sized by the library's result-width bounds
        bc = L.ccm_bound_add(ba, sa, bb, sb)
        bd = L.ccm_bound_scale(ba, sa, SCALE)
        by = L.ccm_bound_matvec(ba, sa, bx, sx, N_COLS)
        self.pa = ccm.PackedMatrix(N_ROWS, N_COLS, ccm.words_for(N_ROWS, N_COLS, ba), dev)
        self.pb = ccm.PackedMatrix(N_ROWS, N_COLS, ccm.words_for(N_ROWS, N_COLS, bb), dev)
        self.px = ccm.PackedMatrix(N_COLS, 1, ccm.words_for(N_COLS, 1, bx), dev)
        self.pc = ccm.PackedMatrix(N_ROWS, N_COLS, ccm.words_for(N_ROWS, N_COLS, bc), dev)
        self.pd = ccm.PackedMatrix(N_ROWS, N_COLS, ccm.words_for(N_ROWS, N_COLS, bd), dev)
        self.py = ccm.PackedMatrix(N_ROWS, 1, ccm.words_for(N_ROWS, 1, by), dev)
        self.unp = torch.empty((N_ROWS, N_COLS), dtype=torch.int64, device=dev)
        self.got = torch.empty(GET_COUNT, dtype=torch.int64, device=dev)
        self.err = torch.zeros(2, dtype=torch.int32, device=dev)
        self.ws = ccm.workspace(ccm.OP_MATVEC, N_ROWS, N_COLS, 1, dev)
        self.ws_pa = ccm.workspace(ccm.OP_PACK, N_ROWS, N_COLS, self.pa.capacity, dev)
        self.ws_pb = ccm.workspace(ccm.OP_PACK, N_ROWS, N_COLS, self.pb.capacity, dev)
        self.ma, self.mb, self.mx = self.pa.c(), self.pb.c(), self.px.c()
        self.mc, self.md, self.my = self.pc.c(), self.pd.c(), self.py.c()
        self.profiled = ["pack", "unpack", "add", "scale", "matvec"]
        self.events = {k: [] for k in self.profiled}
        self.call_events = {k: [] for k in self.profiled}

    def event_pair(self):
        """Two timing events whose CUDA handles exist already (torch creates
        an event lazily at its first record, so record each once here)."""
        pair = []
        for _ in range(2):
            e = self.torch.cuda.Event(enable_timing=True)
            e.record()
            pair.append(e)
        return pair

    def step(self, profile: str = "", A=None, B=None, X=None):
        """One pass of the hot path through the C ABI (asynchronous)."""
        import ctypes
        ccm, L = self.ccm, self.ccm.lib()
        st = ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)
        A = self.A if A is None else A
        B = self.B if B is None else B
        X = self.X if X is None else X
        by = ctypes.byref

        # profile == "call": events on the stream before the first and after
        # the last launch of each profiled call (the stream is backed up with
        # queued steps, so they see device time, not host gaps).
        # profile == "kernel": the library hook brackets each call's main
        # kernel (that call then launches without programmatic dependent
        # launch, so the timed steps use "call" only).
        def prof(name):
            if profile == "kernel":
                e0, e1 = self.event_pair()
                ccm.profile_next(e0, e1)
                self.events[name].append((e0, e1))
            elif profile == "call":
                c0, c1 = self.event_pair()
                c0.record()
                self.call_events[name].append((c0, c1))

        def done(name):
            if profile == "call":
                self.call_events[name][-1][1].record()

        rc = []
        prof("pack")
        vp = ctypes.c_void_p
        rc.append(L.ccm_pack(vp(A.data_ptr()), ccm.I64, N_ROWS, N_COLS, by(self.ma),
                             vp(self.ws_pa.data_ptr()), self.ws_pa.numel(), st))
        done("pack")
        rc.append(L.ccm_pack(vp(B.data_ptr()), ccm.I64, N_ROWS, N_COLS, by(self.mb),
                             vp(self.ws_pb.data_ptr()), self.ws_pb.numel(), st))
        rc.append(L.ccm_pack(vp(X.data_ptr()), ccm.I64, N_COLS, 1, by(self.mx), None, 0, st))
        prof("unpack")
        rc.append(L.ccm_unpack(by(self.ma), ctypes.c_void_p(self.unp.data_ptr()), ccm.I64,
                               ctypes.c_void_p(self.err.data_ptr()), st))
        done("unpack")
        rc.append(L.ccm_get(by(self.ma), ctypes.c_void_p(self.idx.data_ptr()), GET_COUNT,
                            ctypes.c_void_p(self.got.data_ptr()),
                            ctypes.c_void_p(self.err.data_ptr() + 4), st))
        prof("add")
        rc.append(L.ccm_add(by(self.ma), by(self.mb), by(self.mc), None, 0, st))
        done("add")
        prof("scale")
        rc.append(L.ccm_scale(by(self.ma), SCALE, by(self.md), None, 0, st))
        done("scale")
        prof("matvec")
        rc.append(L.ccm_matvec(by(self.ma), by(self.mx), by(self.my),
                               ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), st))
        done("matvec")
        if any(rc):
            raise RuntimeError(f"C ABI returned {rc}")

    def widths(self):
        return {k: (p.header().width, p.header().is_signed) for k, p in
                (("A", self.pa), ("B", self.pb), ("x", self.px), ("C", self.pc), ("D", self.pd),
                 ("y", self.py))}

    def check(self):
        """Every output valid, and results consistent with the inputs."""
        torch = self.torch
        for p in (self.pa, self.pb, self.px, self.pc, self.pd, self.py):
            p._written()
            p.check()
        assert int(self.err[0].item()) == 0 and int(self.err[1].item()) == 0
        assert torch.equal(self.unp, self.A), "unpack(pack(A)) != A"
        assert torch.equal(self.got, self.A.view(-1)[self.idx]), "get mismatch"
        c = self.ccm.unpack(self.pc)
        assert torch.equal(c, self.A + self.B), "add mismatch"
        d = self.ccm.unpack(self.pd)
        assert torch.equal(d, self.A * SCALE), "scale mismatch"
        y = self.ccm.unpack(self.py).view(-1)
        # int64 matvec reference on the GPU (exact: |y| < 2^40)
        yr = (self.A.double() @ self.X.view(-1).double()).round().long()
        assert torch.equal(y, yr), "matvec mismatch"

    def step_bytes(self):
        """Algorithmic (one-pass) bytes of each operation in a step."""
        w = self.widths()
        n, b = self.n, w["A"][0]
        bb, bc, bd, bx, byw = w["B"][0], w["C"][0], w["D"][0], w["x"][0], w["y"][0]
        ops = {
            "pack": 8 * n + n * b / 8,                 # per matrix (A)
            "pack_B": 8 * n + n * bb / 8,
            "pack_x": 8 * N_COLS + N_COLS * bx / 8,
            "unpack": n * b / 8 + 8 * n,
            "get": GET_COUNT * (8 + 8 + 4),            # index, value, one word
            "add": n * (b + bb + bc) / 8,
            "scale": n * (b + bd) / 8,
            "matvec": n * b / 8 + N_COLS * bx / 8 + N_ROWS * byw / 8,
        }
        return ops


def kernel_traffic(kernel: str):
    """Per-launch DRAM bytes of `kernel` from the committed ncu summary, when
    the kernel source has not changed since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    import hashlib
    for line in open(path):
        p = line.split("#", 1)[0].split()
        if len(p) >= 4 and p[0] == kernel.replace(" ", ""):
            src_hash = hashlib.sha256()
            for f in p[3].split(","):
                src_hash.update(open(os.path.join(ROOT, f), "rb").read())
            if src_hash.hexdigest()[:16] == p[1]:
                return float(p[2])
    return None


def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_1303_0270_gb300 import ccm
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    ccm.lib()
    wl = Workload(ccm, torch, dev, seed_offset=1000 * rank)

    dist = None
    if world > 1:
        import torch.distributed as dist

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        wl.step()
    torch.cuda.synchronize()
    wl.check()
    widths = wl.widths()

    sampler = ClockSampler(local_rank)
    if rank == 0:
        sampler.start()
    barrier()
    launches0 = ccm.launch_count()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(args.steps):
        wl.step(profile="call")
    t1.record()
    barrier()
    launches = ccm.launch_count() - launches0
    ms = t0.elapsed_time(t1)
    clocks = sampler.stop() if rank == 0 else None
    # main-kernel times: the same steps again, each op's main kernel bracketed
    for _ in range(args.steps):
        wl.step(profile="kernel")
    torch.cuda.synchronize()
    if dist is not None:
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    wl.check()

    # per-kernel times of the profiled main kernels
    kern_ms = {k: statistics.mean(e0.elapsed_time(e1) for e0, e1 in v)
               for k, v in wl.events.items() if v}
    call_ms = {k: statistics.mean(e0.elapsed_time(e1) for e0, e1 in v)
               for k, v in wl.call_events.items() if v}
    ops = wl.step_bytes()
    step_bytes = sum(ops.values())
    ms_per_step = ms / args.steps
    value = world * step_bytes / (ms_per_step * 1e-3) / 1e9

    # end to end: host (pinned) inputs in, results back to host, every step
    e2e = run_e2e(wl, torch, args, barrier, dist, dev, world, step_bytes)

    if rank != 0:
        return None
    hbm, peak_kind = peaks()
    kernels = {"pack": "ge::k_pack_local<int64_t, 8>", "unpack": "ge::k_unpack_ge<int64_t, 8>",
               "add": "ge::k_ew_lanes<OpAdd> (+ k_ew spec/finish, which return at once)",
               "scale": "ge::k_ew_lanes<OpScale<true>> (+ k_ew spec/finish, which return at once)",
               "matvec": "mvs::k_mv<byte lanes, narrow>"}
    per_op = {}
    for k, t in kern_ms.items():
        gbs = ops[k] / (t * 1e-3) / 1e9
        per_op[k] = {"kernel": kernels[k], "ms": round(t, 5), "algorithmic_bytes": int(ops[k]),
                     "GB/s": round(gbs, 1), "frac_of_hbm": round(gbs / hbm, 3)}
        if k in call_ms:
            # the whole call: every launch of the operation, epilogues included
            gbc = ops[k] / (call_ms[k] * 1e-3) / 1e9
            per_op[k].update({"ms_call": round(call_ms[k], 5), "GB/s_call": round(gbc, 1),
                              "frac_of_hbm_call": round(gbc / hbm, 3)})
    def roofline(d):
        return {"bound": "hbm", "kernel": d["kernel"], "achieved": d["GB/s"], "peak": hbm,
                "unit": "GB/s", "frac": round(d["GB/s"] / hbm, 4),
                "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)",
                "traffic": kernel_traffic(d["kernel"]),
                "algorithmic_bytes_per_launch": d["algorithmic_bytes"]}
    dom = max(per_op, key=lambda k: per_op[k]["ms"])
    roof = roofline(per_op[dom])
    roof_mv = roofline(per_op["matvec"]) if "matvec" in per_op else None
    line = {
        "metric": METRIC, "value": round(value, 2), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic (counter-based SplitMix64, generated on the GPU)",
        "config": {"workload": "8192x8192 int64 Poisson(5) count matrices A, B; x 8192 signed "
                               "8-bit; step = pack A,B,x + unpack A + get 2^20 + A+B + 7A + Ax",
                   "rows": N_ROWS, "cols": N_COLS, "seeds": list(wl.seeds),
                   "widths": {k: v[0] for k, v in widths.items()},
                   "l2": "inputs larger than L2 (dense A, B 512 MiB each, re-read every step)",
                   "parallelism": f"replicas x{world} (independent problems)"},
        "step_bytes": int(step_bytes), "per_op": per_op,
        "matvec_GBps": per_op.get("matvec", {}).get("GB/s"),
        "eta1_vs_int64": round((64 - widths["A"][0]) / 64, 4),
        "roofline": roof, "roofline_matvec": roof_mv,
        # two events recorded back to back on the stream: the floor inside
        # every per-kernel time above (reported, not subtracted)
        "event_pair_floor_us": event_pair_floor(torch),
        "e2e": e2e, "gpu_launches": launches, "clocks": clocks,
    }
    # the metric's other two parts, measured in the same run (this rank's replica)
    line["matmul"] = matmul_measure(torch, ccm, dev, args.matmul_n, SEED_A, reps=10)
    line["batch"] = batch_measure(torch, ccm, dev, args.batch_count, SEED_A, steps=10, warmup=3)
    return line


def event_pair_floor(torch, reps: int = 50) -> float:
    ts = []
    for _ in range(reps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) * 1e3)
    return round(statistics.mean(ts), 2)


def batch_measure(torch, ccm, dev, count, seed, steps, warmup):
    """Batched matvec: `count` packed matrices, rows/cols log-uniform in
    [16, 2048), widths uniform in 1..24, values uniform over the signed b-bit
    range, x signed 8-bit; one persistent graph-captured launch (autotuned)
    against one ccm_matvec call per matrix on the same GPU.  Per batch: the
    mean over `steps` graph replays (inputs 2.7 GB, larger than L2)."""
    import synth
    from paper_1303_0270_gb300.batch import BatchMatvec
    rows, cols, widths = synth.batch_shapes(seed, count)
    maxn = int((rows * cols).max())
    dense = torch.empty(maxn, dtype=torch.int64, device=dev)
    xd = torch.empty(2048, dtype=torch.int64, device=dev)
    mats, xs = [], []
    packed_bytes = 0
    for i in range(count):
        r, c, b = int(rows[i]), int(cols[i]), int(widths[i])
        si = synth.batch_matrix_seed(seed, i)
        lo, hi = synth.signed_range(b)
        ccm.gen_uniform(r * c, si, synth.STREAM_A, lo, hi, out=dense[: r * c])
        pa = ccm.PackedMatrix(r, c, ccm.words_for(r, c, b), dev)
        ccm.pack_into(dense[: r * c].view(r, c), pa)
        ccm.gen_uniform(c, si, synth.STREAM_X, -128, 127, out=xd[:c])
        px = ccm.PackedMatrix(c, 1, ccm.words_for(c, 1, 8), dev)
        ccm.pack_into(xd[:c].view(c, 1), px)
        mats.append(pa)
        xs.append(px)
        packed_bytes += ccm.words_for(r, c, b) * 4
    del dense
    torch.cuda.synchronize()
    bm = BatchMatvec(mats, xs)
    tune = bm.autotune(reps=2)
    bm.capture()
    for _ in range(warmup):
        bm.run()
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(steps):
        bm.run()
    t1.record()
    torch.cuda.synchronize()
    ms_batch = t0.elapsed_time(t1) / steps
    # one launch sequence per matrix (ccm_matvec), same inputs
    ys = [ccm.PackedMatrix(m.rows, 1, bm.ys[i].capacity, dev) for i, m in enumerate(mats)]
    wss = torch.empty(ccm.workspace_bytes(ccm.OP_MATVEC, 2048, 2048, 1), dtype=torch.uint8,
                      device=dev)

    def plain():
        for a, x, y in zip(mats, xs, ys):
            ccm.matvec_into(a, x, y, ws=wss)
    plain()
    torch.cuda.synchronize()
    reps = max(1, min(3, steps))
    t0.record()
    for _ in range(reps):
        plain()
    t1.record()
    torch.cuda.synchronize()
    ms_plain = t0.elapsed_time(t1) / reps
    # results: identical words, every entry
    bad = 0
    for i in range(count):
        if bm.ys[i].header().status != 0 or not torch.equal(bm.ys[i].words(), ys[i].words()):
            bad += 1
    hbm, _ = peaks()
    gbs = packed_bytes / (ms_batch * 1e-3) / 1e9
    return {"workload": f"{count} packed matrices, rows/cols log-uniform [16, 2048), "
                        "widths U{1..24}, signed uniform values, x signed 8-bit",
            "packed_bytes": packed_bytes, "fields": int((rows * cols).sum()),
            "autotune": {k: tune[k] for k in ("unit_segments", "grid", "slots", "stage_bytes")
                         if k in tune},
            "ms": round(ms_batch, 4), "GB/s": round(gbs, 2), "frac_of_hbm": round(gbs / hbm, 4),
            "plain_ms": round(ms_plain, 3), "speedup_vs_plain": round(ms_plain / ms_batch, 2),
            "mismatches_vs_plain": bad, "timing": f"mean of {steps} graph replays, CUDA events"}


def run_batch(args, rank, world, local_rank):
    import torch

    from paper_1303_0270_gb300 import ccm
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    d = batch_measure(torch, ccm, dev, args.batch_count, SEED_A + 1000 * rank, args.steps,
                      args.warmup)
    return {
        "metric": METRIC, "workload": "batched matvec", "value": d["GB/s"], "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": d["ms"], "higher_is_better": True, "scaling": "weak",
        "dtype": "int64", "data": "synthetic", "config": {"workload": d["workload"]},
        "batch": d,
    }


def matmul_measure(torch, ccm, dev, n, seed_base, reps):
    """Packed matmul: A, B n x n uniform over the signed b-bit range, b in
    {4, 8, 12, 16}; exact int64 C re-packed at its width.  Tensor-core digit
    path (tcgen05, e4m3 digits, fp32 accumulators) against the CUDA-core
    decode-and-multiply path on the same inputs (results compared word for
    word).  Useful ops = 2 n^3 per matmul; the whole call includes the digit
    planes and C's re-pack."""
    import synth
    peaks_d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    fp8_peak = 2.0 * float(peaks_d["bf16_tflops"])  # measured bf16 x nominal fp8/bf16 ratio (2)
    dense = torch.empty(n * n, dtype=torch.int64, device=dev)
    ws = ccm.workspace(ccm.OP_MATMUL, n, n, n, dev)
    results = []
    for b in (4, 8, 12, 16):
        lo, hi = synth.signed_range(b)
        seed = seed_base + b
        ccm.gen_uniform(n * n, seed, synth.STREAM_A, lo, hi, out=dense)
        pa = ccm.pack_into(dense.view(n, n), ccm.PackedMatrix(n, n, ccm.words_for(n, n, b), dev))
        ccm.gen_uniform(n * n, seed, synth.STREAM_B, lo, hi, out=dense)
        pb = ccm.pack_into(dense.view(n, n), ccm.PackedMatrix(n, n, ccm.words_for(n, n, b), dev))
        cap = ccm.words_for(n, n, ccm.bound_matmul(pa, pb))
        ct = ccm.PackedMatrix(n, n, cap, dev)
        cc = ccm.PackedMatrix(n, n, cap, dev)
        timings = {}
        for name, path, out, nrep in (("tensor", ccm.MATMUL_TENSOR, ct, reps),
                                      ("cudacore", ccm.MATMUL_CUDACORE, cc, 2)):
            for _ in range(2):
                ccm.matmul_into(pa, pb, out, path=path, ws=ws)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            # whole calls: nrep calls queued back to back on the stream (the
            # device time per call, not the host's launch latency)
            e0.record()
            for _ in range(nrep):
                ccm.matmul_into(pa, pb, out, path=path, ws=ws)
            e1.record()
            e1.synchronize()
            tot = e0.elapsed_time(e1) / nrep
            # the MMA (or CUDA-core) kernel alone, one call at a time (the
            # library records the two events; recorded once here so that
            # torch accepts them)
            k0.record()
            k1.record()
            kern = 0.0
            for _ in range(nrep):
                ccm.profile_next(k0, k1)
                ccm.matmul_into(pa, pb, out, path=path, ws=ws)
                k1.synchronize()
                kern += k0.elapsed_time(k1)
            timings[name] = (tot, kern / nrep)
        same = (ct.check().width == cc.check().width and torch.equal(ct.words(), cc.words()))
        L = (b + 3) // 4
        useful = 2.0 * n ** 3
        t_all, t_mma = timings["tensor"]
        results.append({
            "b": b, "digits": L, "width_C": ct.width, "tensor_vs_cudacore_identical": bool(same),
            "tensor_ms": round(t_all, 4), "tensor_mma_kernel_ms": round(t_mma, 4),
            "useful_int_TOPS": round(useful / (t_all * 1e-3) / 1e12, 2),
            "mma_kernel_fp8_TFLOPS": round(L * L * useful / (t_mma * 1e-3) / 1e12, 1),
            "mma_frac_of_fp8_peak": round(L * L * useful / (t_mma * 1e-3) / 1e12 / fp8_peak, 4),
            "cudacore_ms": round(timings["cudacore"][0], 3),
            "cudacore_useful_int_TOPS": round(useful / (timings["cudacore"][0] * 1e-3) / 1e12, 3),
            "speedup_tensor_vs_cudacore": round(timings["cudacore"][0] / t_all, 2),
        })
        del pa, pb, ct, cc
    del dense, ws
    # reference point: a plain s8 x s8 -> s32 GEMM of the same size through
    # the vendor library (torch._int_mm -> cuBLASLt), the integer tensor rate
    # an int8-limb design would get on this GPU
    int8_tops = None
    try:
        a8 = torch.randint(-128, 128, (n, n), dtype=torch.int8, device=dev)
        b8 = torch.randint(-128, 128, (n, n), dtype=torch.int8, device=dev)
        for _ in range(3):
            torch._int_mm(a8, b8)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            torch._int_mm(a8, b8)
        e1.record()
        e1.synchronize()
        int8_tops = round(2.0 * n ** 3 / (e0.elapsed_time(e1) / 10 * 1e-3) / 1e12, 1)
    except RuntimeError:
        pass
    return {"n": n, "unit": "int-TOPS (useful)",
            "useful_int_TOPS_mean": round(statistics.mean(r["useful_int_TOPS"] for r in results), 2),
            "fp8_peak_TFLOPS": fp8_peak,
            "fp8_peak_source": "MEASURED_PEAKS bf16_tflops x 2 (nominal fp8/bf16 ratio)",
            "s8_gemm_library_TOPS": int8_tops,
            "s8_gemm_library": "torch._int_mm (cuBLASLt) s8 x s8 -> s32, same n, 10 launches",
            "timing": f"whole call: {reps} calls queued back to back, mean; MMA kernel: "
                      f"mean of {reps} calls; CUDA events",
            "results": results}


def run_matmul_bench(args, rank, world, local_rank):
    import torch

    from paper_1303_0270_gb300 import ccm
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    d = matmul_measure(torch, ccm, dev, args.matmul_n, SEED_A + 1000 * rank, args.steps)
    return {"metric": METRIC, "workload": "packed matmul", "unit": d["unit"],
            "value": d["useful_int_TOPS_mean"], "matmul": d}


def run_vlb_bench(args, rank, world, local_rank):
    """VLB (Method 2) against SM (Method 1) on two 8192 x 8192 matrices: the
    Poisson(5) count matrix of the default step (SM is smaller) and a heavy
    tailed one with bit lengths spread over 1..40 (VLB is smaller).  Times the
    encoder (dense int64 -> VLB stream + index), the decoder and the matvec on
    the VLB stream, with the SM pack and matvec beside them; y compared word
    for word between the two encodings."""
    import ctypes

    import torch

    import synth
    from paper_1303_0270_gb300 import ccm
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n_rows = n_cols = 8192
    n = n_rows * n_cols
    hbm, _ = peaks()
    table = torch.from_numpy(synth.poisson_cdf_table(LAMBDA))
    X = ccm.gen_uniform(n_cols, SEED_A, synth.STREAM_X, -128, 127, device=dev).view(n_cols, 1)
    px = ccm.pack(X)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def kernel_ms(fn, reps):
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record()
        k1.record()
        fn()
        torch.cuda.synchronize()
        ts = []
        for i in range(reps):
            flush.fill_(i & 255)  # inputs out of L2 between repetitions
            ccm.profile_next(k0, k1)
            fn()
            torch.cuda.synchronize()
            ts.append(k0.elapsed_time(k1))
        return statistics.mean(ts)

    results = []
    for name in ("poisson5", "heavy_tail_1_40"):
        if name == "poisson5":
            A = ccm.gen_poisson(n, SEED_A, synth.STREAM_A, table, device=dev).view(n_rows, n_cols)
        else:  # floor(2^(40 u)), u uniform: bit lengths spread evenly over 1..40
            U = ccm.gen_uniform(n, SEED_A, synth.STREAM_A, 0, (1 << 53) - 1, device=dev)
            A = torch.floor(torch.exp2(U.double() * (40.0 / 2 ** 53))).long().view(n_rows, n_cols)
            del U
        choice = ccm.choose(A)
        sm_b = choice["sm_width"]
        pa = ccm.PackedMatrix(n_rows, n_cols, ccm.words_for(n_rows, n_cols, sm_b), dev)
        ws_pack = ccm.workspace(ccm.OP_PACK, n_rows, n_cols, pa.capacity, dev)
        v = ccm.vlb_pack(A)
        vbytes = 4 * int(v.header().nwords)
        y_sm = ccm.PackedMatrix(n_rows, 1, ccm.words_for(n_rows, 1, 64), dev)
        y_v = ccm.PackedMatrix(n_rows, 1, ccm.words_for(n_rows, 1, 64), dev)
        ws_mv = ccm.workspace(ccm.OP_MATVEC, n_rows, n_cols, 1, dev)
        ws_vmv = ccm.workspace(ccm.OP_VLB_MATVEC, n_rows, n_cols, 0, dev)
        ws_v = torch.empty(max(ccm.workspace_bytes(ccm.OP_VLB, n_rows, n_cols, 0), 256),
                           dtype=torch.uint8, device=dev)
        dense_out = torch.empty_like(A)
        reps = max(args.steps, 3)
        L = ccm.lib()
        vp = ctypes.c_void_p

        def vlb_encode():
            L.ccm_vlb_pack(vp(A.data_ptr()), ccm.I64, n_rows, n_cols, vp(v.buf.data_ptr()),
                           vp(v.buf.data_ptr() + 4 * ccm.HEADER_WORDS), v.capacity,
                           vp(v.index.data_ptr()), vp(ws_v.data_ptr()), ws_v.numel(),
                           vp(torch.cuda.current_stream().cuda_stream))

        t = {
            "sm_pack": kernel_ms(lambda: ccm.pack_into(A, pa, ws=ws_pack), reps),
            "sm_matvec": kernel_ms(lambda: ccm.matvec_into(pa, px, y_sm, ws=ws_mv), reps),
            "vlb_encode": kernel_ms(vlb_encode, reps),
            "vlb_decode": kernel_ms(lambda: ccm.vlb_unpack(v, check=False), reps),
            "vlb_matvec": kernel_ms(lambda: ccm.vlb_matvec_into(v, px, y_v, ws=ws_vmv), reps),
        }
        same = (y_sm.check().width == y_v.check().width and
                torch.equal(y_sm.words(), y_v.words()))
        assert torch.equal(ccm.vlb_unpack(v), A), "VLB round trip"
        sm_bytes = n * sm_b / 8
        gbs = {"sm_pack": (8 * n + sm_bytes), "sm_matvec": sm_bytes,
               "vlb_encode": 8 * n + vbytes,  # the write pass (k_vlb_write): dense in, stream out
               "vlb_decode": vbytes + 8 * n, "vlb_matvec": vbytes}
        results.append({
            "matrix": name, "sm_bits_per_entry": sm_b,
            "vlb_bits_per_entry": round(8 * vbytes / n, 3), "vlb_prefix_bits": choice["vlb_prefix"],
            "choice": choice["choice"], "y_identical_sm_vs_vlb": bool(same),
            "kernel_ms": {k: round(val, 4) for k, val in t.items()},
            "GB/s": {k: round(gbs[k] / (t[k] * 1e-3) / 1e9, 1) for k in t},
        })
        del A, dense_out, v, pa
        torch.cuda.empty_cache()
    mv = results[1]["GB/s"]["vlb_matvec"]
    return {"metric": METRIC, "workload": "vlb codec", "unit": "GB/s",
            "value": mv, "value_is": "VLB matvec, heavy-tailed matrix, stream bytes / kernel time",
            "frac_of_hbm": round(mv / hbm, 4), "l2": "flushed (256 MiB write) before every repetition",
            "results": results}


def run_sweep_bench(args, rank, world, local_rank):
    """The width sweep of the 8192 x 8192 workload: for each b, A and B with
    entries uniform over the signed b-bit range (generated on the GPU), x
    signed 8-bit; pack (single pass), unpack, A + B, 7A and A x, each timed
    on its main kernel(s) with L2 flushed before every repetition, as GB/s of
    algorithmic bytes and as a fraction of the measured HBM peak."""
    import torch

    import synth
    from paper_1303_0270_gb300 import ccm
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    n_rows = n_cols = 8192
    n = n_rows * n_cols
    hbm, _ = peaks()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    X = ccm.gen_uniform(n_cols, SEED_A, synth.STREAM_X, -128, 127, device=dev).view(n_cols, 1)
    px = ccm.pack(X)
    A = torch.empty((n_rows, n_cols), dtype=torch.int64, device=dev)
    B = torch.empty_like(A)
    unp = torch.empty_like(A)
    reps = max(3, args.steps)

    def kernel_ms(fn):
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k0.record()
        k1.record()
        fn()
        torch.cuda.synchronize()
        ts = []
        for i in range(reps):
            flush.fill_(i & 255)
            ccm.profile_next(k0, k1)
            fn()
            torch.cuda.synchronize()
            ts.append(k0.elapsed_time(k1))
        return statistics.mean(ts)

    rows = []
    widths = [int(w) for w in args.sweep_widths.split(",")]
    for b in widths:
        lo, hi = synth.signed_range(b)
        ccm.gen_uniform(n, SEED_A + b, synth.STREAM_A, lo, hi, out=A.view(-1))
        ccm.gen_uniform(n, SEED_B + b, synth.STREAM_B, lo, hi, out=B.view(-1))
        pa = ccm.PackedMatrix(n_rows, n_cols, ccm.words_for(n_rows, n_cols, b), dev)
        pb = ccm.PackedMatrix(n_rows, n_cols, ccm.words_for(n_rows, n_cols, b), dev)
        ws = ccm.workspace(ccm.OP_PACK, n_rows, n_cols, pa.capacity, dev)
        ccm.pack_into(B, pb, ws=ws)
        pc = ccm.PackedMatrix(n_rows, n_cols, ccm.words_for(n_rows, n_cols, min(64, b + 2)), dev)
        pd = ccm.PackedMatrix(n_rows, n_cols, ccm.words_for(n_rows, n_cols, min(64, b + 4)), dev)
        py = ccm.PackedMatrix(n_rows, 1, ccm.words_for(n_rows, 1, 64), dev)
        wsm = ccm.workspace(ccm.OP_MATVEC, n_rows, n_cols, 1, dev)
        t = {"pack": kernel_ms(lambda: ccm.pack_into(A, pa, ws=ws)),
             "unpack": kernel_ms(lambda: ccm.unpack(pa, out=unp, check=False)),
             "add": kernel_ms(lambda: ccm.add_into(pa, pb, pc)),
             "scale": kernel_ms(lambda: ccm.scale_into(pa, SCALE, pd)),
             "matvec": kernel_ms(lambda: ccm.matvec_into(pa, px, py, ws=wsm))}
        assert pa.check().width == b and torch.equal(unp, A)
        bc, bd, by = pc.check().width, pd.check().width, py.check().width
        nb = {"pack": 8 * n + n * b / 8, "unpack": n * b / 8 + 8 * n,
              "add": n * (2 * b + bc) / 8, "scale": n * (b + bd) / 8,
              "matvec": n * b / 8 + n_cols + n_rows * by / 8}
        gbs = {k: nb[k] / (t[k] * 1e-3) / 1e9 for k in t}
        rows.append({"b": b, "ms": {k: round(v, 4) for k, v in t.items()},
                     "GB/s": {k: round(v, 1) for k, v in gbs.items()},
                     "frac_of_hbm": {k: round(v / hbm, 3) for k, v in gbs.items()}})
        del pa, pb, pc, pd, py, ws, wsm
        torch.cuda.empty_cache()
    mv = statistics.mean(r["GB/s"]["matvec"] for r in rows)
    return {"metric": METRIC, "workload": "width sweep", "unit": "GB/s", "value": round(mv, 1),
            "value_is": "mean matvec GB/s over the swept widths", "frac_of_hbm": round(mv / hbm, 4),
            "config": {"workload": "8192x8192, entries uniform over the signed b-bit range, "
                                   "x signed 8-bit, s = 7", "widths": widths,
                       "l2": "flushed (256 MiB write) before every repetition"},
            "results": rows}


def serve_measure(torch, dev, store_gb, budget_gb, requests, reps=3, seed_store=SEED_A,
                  seed_trace=SEED_B):
    """Serving (config 5): a store of packed matrices (dims log-uniform in
    [64, 8192), widths U{2..20}) resident on the GPU, a Poisson stream of
    requests (60 % matvec on a store matrix, 30 % pack of a new dense matrix,
    10 % matmul of two store matrices; every size log-uniform over 64..8192),
    admitted by memory and continuously batched.  An untimed pass of the
    whole trace first (every output size allocated once, every launch plan
    made), then `reps` runs each of: saturation (everything arrives at t = 0),
    50 % and 80 % of the median saturation rate; medians with min..max.
    Matvecs and packs run on high-priority streams, matmuls on low-priority
    ones.  Against it, one launch sequence per request on one stream for the
    same 80 % trace and at saturation."""
    from paper_1303_0270_gb300 import serve
    t0 = time.perf_counter()
    store, store_bytes = serve.build_store(seed_store, int(store_gb * (1 << 30)), 64, 8192,
                                           2, 20, dev)
    t_store = time.perf_counter() - t0
    budget = store_bytes + int(budget_gb * (1 << 30))

    def run(rate, batching=True, streams=4, heavy_streams=2):
        trace = serve.build_trace(seed_trace, store, requests, rate, dev)
        srv = serve.Server(store, mem_budget=budget, streams=streams, batching=batching,
                           heavy_streams=heavy_streams)
        torch.cuda.synchronize(dev)
        w0 = time.perf_counter()
        # results handed back and dropped as they complete, but for a sample
        # kept for the alone-vs-mix check
        st = srv.run(trace, keep_result=lambda r: r.rid % 64 == 0)
        wall = time.perf_counter() - w0
        return st.summary(wall), trace

    def spread(runs, key):
        v = sorted(r[key] for r in runs)
        return {"median": v[len(v) // 2], "min": v[0], "max": v[-1]}

    run(float("inf"))  # untimed: allocations and plans of every request size
    sats = [run(float("inf"))[0] for _ in range(reps)]
    rate_sat = spread(sats, "throughput_rps")["median"]
    out = {"store_bytes": store_bytes, "store_matrices": len(store),
           "store_build_s": round(t_store, 1), "requests_per_run": requests, "reps": reps,
           "mix": "60% matvec / 30% pack / 10% matmul, sizes log-uniform 64..8192",
           "mem_budget": budget, "streams": "4 high-priority (matvec, pack) + 2 low-priority "
                                             "(matmul)",
           "saturation_rps": spread(sats, "throughput_rps")}
    trace80 = None
    for frac in (0.5, 0.8):
        runs = []
        for _ in range(reps):
            summ, tr = run(frac * rate_sat)
            runs.append(summ)
            trace80 = tr if frac == 0.8 else trace80
        key = f"at_{int(frac * 100)}pct"
        out[key] = {"rate_rps": round(frac * rate_sat, 1),
                    "throughput_rps": spread(runs, "throughput_rps"),
                    "p50_ms": spread(runs, "p50_ms"), "p99_ms": spread(runs, "p99_ms"),
                    "p99_ms_by_kind": {k: spread(runs, f"p99_ms_{k}")
                                       for k in ("matvec", "pack", "matmul")
                                       if all(f"p99_ms_{k}" in r for r in runs)}}
    plain80, _ = run(0.8 * rate_sat, batching=False, streams=1, heavy_streams=0)
    plain_sat, _ = run(float("inf"), batching=False, streams=1, heavy_streams=0)
    out["plain_at_80pct"] = {k: plain80[k] for k in ("throughput_rps", "p50_ms", "p99_ms")}
    out["plain_saturation_rps"] = plain_sat["throughput_rps"]
    out["speedup_saturation_vs_plain"] = round(rate_sat / plain_sat["throughput_rps"], 2)
    # results: the same alone and in the mix (sample of the 80 % trace)
    bad = 0
    for r in trace80:
        if r.out is None:
            continue
        alone = serve.run_alone(store, r, dev)
        if not (torch.equal(r.out.words(), alone.words()) and
                r.out.header().width == alone.header().width):
            bad += 1
    out["mismatches_alone_vs_mix"] = bad
    return out


def run_serve_bench(args, rank, world, local_rank):
    import torch
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    d = serve_measure(torch, dev, args.store_gb, args.serve_budget_gb, args.serve_requests,
                      seed_store=SEED_A + rank)
    return {"metric": METRIC, "workload": "serving", "unit": "requests/s",
            "value": d["at_80pct"]["throughput_rps"]["median"], "n_gpus": world,
            "data": "synthetic", "serve": d}


def run_e2e(wl, torch, args, barrier, dist, dev, world, step_bytes):
    """Same step through the public API with host buffers: pinned host -> device
    copies of the dense inputs, the step, and device -> host copies of every
    result (unpacked A, the gathered entries, packed C, D and y).  Steps are
    pipelined over three streams (inputs of step k+1 copied in while step k
    computes and its results are copied out; two sets of device inputs and
    host outputs), so the per-step time is the copies' throughput, not their
    sum; every step still moves all its bytes in and out.  (Cutting the copies
    into chunks on more streams measured no faster.)"""
    hA = torch.empty_like(wl.A, device="cpu").pin_memory()
    hB = torch.empty_like(wl.B, device="cpu").pin_memory()
    hX = torch.empty_like(wl.X, device="cpu").pin_memory()
    hA.copy_(wl.A)
    hB.copy_(wl.B)
    hX.copy_(wl.X)
    dev_in = [(torch.empty_like(wl.A), torch.empty_like(wl.B), torch.empty_like(wl.X))
              for _ in range(2)]
    outs = [wl.unp, wl.got, wl.pc.buf, wl.pd.buf, wl.py.buf]
    houts = [[torch.empty_like(o, device="cpu").pin_memory() for o in outs] for _ in range(2)]
    h2d = hA.numel() * 8 + hB.numel() * 8 + hX.numel() * 8
    d2h = sum(o.numel() * o.element_size() for o in outs)
    s_in, s_comp, s_out = (torch.cuda.Stream(dev) for _ in range(3))
    ev = lambda: torch.cuda.Event()  # noqa: E731
    comp_done = [ev(), ev()]
    out_done = ev()
    started = [False, False]
    any_out = [False]

    def one(k):
        i = k % 2
        dA, dB, dX = dev_in[i]
        with torch.cuda.stream(s_in):
            if started[i]:
                s_in.wait_event(comp_done[i])  # step k-2 no longer reads these inputs
            dA.copy_(hA, non_blocking=True)
            dB.copy_(hB, non_blocking=True)
            dX.copy_(hX, non_blocking=True)
            in_done = ev()
            in_done.record(s_in)
        with torch.cuda.stream(s_comp):
            s_comp.wait_event(in_done)
            if any_out[0]:
                s_comp.wait_event(out_done)  # step k-1's results have left the device
            wl.step(A=dA, B=dB, X=dX)
            comp_done[i].record(s_comp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(comp_done[i])
            for h, o in zip(houts[i], outs):
                h.copy_(o, non_blocking=True)
            out_done.record(s_out)
        started[i] = True
        any_out[0] = True

    steps = max(3, min(args.steps, 10))
    for k in range(2):
        one(k)
    torch.cuda.synchronize(dev)
    barrier()
    t0 = time.perf_counter()
    for k in range(steps):
        one(k)
    torch.cuda.synchronize(dev)
    barrier()
    sec = (time.perf_counter() - t0) / steps
    if dist is not None:
        t = torch.tensor([sec], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        sec = float(t.item())
    assert torch.equal(houts[(steps - 1) % 2][0], hA), "e2e unpack mismatch"
    return {"value": round(world * step_bytes / sec / 1e9, 2), "unit": "GB/s",
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": round(sec * 1e3, 4), "steps": steps,
            "timing": "host wall clock around the pipelined copies and steps, synchronised"}


# ---------------------------------------------------------------------------
# the oracle, timed on the host cores
# ---------------------------------------------------------------------------
def oracle_sample(rows: int):
    """Rows 0..rows-1 of the same workload, through the oracle (one thread)."""
    import oracle
    import synth
    a = synth.count_matrix(SEED_A, synth.STREAM_A, rows, N_COLS, LAMBDA)
    b = synth.count_matrix(SEED_B, synth.STREAM_B, rows, N_COLS, LAMBDA)
    x = synth.uniform_int(SEED_A, synth.STREAM_X, N_COLS, -128, 127).reshape(-1, 1)
    idx = synth.uniform_int(SEED_A, synth.STREAM_INDEX, max(1, GET_COUNT * rows // N_ROWS), 0,
                            rows * N_COLS - 1)
    t0 = time.perf_counter()
    pa, pb, px = oracle.pack(a), oracle.pack(b), oracle.pack(x)
    ua = oracle.unpack(pa)
    g = oracle.get_flat(pa, idx[: min(idx.size, 4096)])
    pc = oracle.add(pa, pb)
    pd = oracle.scale(pa, SCALE)
    py = oracle.matvec(pa, px)
    sec = time.perf_counter() - t0
    n = rows * N_COLS
    bA, bB, bC, bD = pa.width, pb.width, pc.width, pd.width
    nbytes = (2 * 8 * n + n * (bA + bB) / 8 + 8 * N_COLS + (n * bA / 8 + 8 * n)
              + min(idx.size, 4096) * 20 + n * (bA + bB + bC) / 8 + n * (bA + bD) / 8
              + n * bA / 8 + N_COLS + rows * py.width / 8)
    assert np.array_equal(ua, a) and g.size > 0
    return sec, nbytes


def _oracle_worker(rows: int):
    return oracle_sample(rows)


def cpu_baseline_parallel(rows: int, procs: int):
    """The same oracle sample in `procs` processes at once (one row block per
    core, as an OpenMP loop over rows would split it): throughput of the
    oracle on all host cores.  Spawned processes (no fork of a CUDA parent)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(procs) as pool:
        pool.map(_oracle_worker, [64] * procs)  # imports and library loads, untimed
        t0 = time.perf_counter()
        res = pool.map(_oracle_worker, [rows] * procs)
        wall = time.perf_counter() - t0
    nb = sum(r[1] for r in res)
    return {"value": round(nb / wall / 1e9, 4), "unit": "GB/s", "cores": procs, "kind": "oracle",
            "sample": f"{procs} processes, each rows 0..{rows - 1} of the 8192x8192 workload "
                      f"(same operations as the one-core sample); {wall:.1f} s wall"}


def cpu_baseline(target_s: float = 12.0):
    sec, nb = oracle_sample(64)
    rows = int(min(N_ROWS, max(64, 64 * target_s / max(sec, 1e-3))))
    rows = max(64, rows // 64 * 64)
    sec, nb = oracle_sample(rows)
    return {"value": round(nb / sec / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
            "sample": f"rows 0..{rows - 1} of the 8192x8192 workload ({rows * N_COLS} entries): "
                      f"pack A,B,x, unpack A, get 4096, A+B, 7A, Ax; {sec:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    rows = 128
    for _ in range(args.warmup):
        oracle_sample(rows)
    secs, nbs = [], []
    for _ in range(args.steps):
        s, nb = oracle_sample(rows)
        secs.append(s)
        nbs.append(nb)
    sec = sum(secs) / len(secs)
    value = statistics.mean(nbs) / sec / 1e9
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(sec * 1e3, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int64", "data": "synthetic (same generator)",
        "config": {"workload": "8192x8192 int64 Poisson(5) count matrices A, B; x 8192 signed "
                               "8-bit; step = pack A,B,x + unpack A + get + A+B + 7A + Ax",
                   "sample_rows": rows},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"rows 0..{rows - 1} of the workload per step"},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ccm", choices=["ccm", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="step",
                    choices=["step", "batch", "matmul", "serve", "vlb", "sweep"])
    ap.add_argument("--sweep-widths", default="1,2,3,4,5,6,7,8,10,12,16,20,24,28,31,32")
    ap.add_argument("--store-gb", type=float, default=8.0)
    ap.add_argument("--serve-budget-gb", type=float, default=16.0)
    ap.add_argument("--serve-requests", type=int, default=20000)
    ap.add_argument("--matmul-n", type=int, default=4096)
    ap.add_argument("--batch-count", type=int, default=10000)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        line = run_reference(args, rank, world)
        if line is not None:
            print(json.dumps(line), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.workload in ("batch", "matmul", "serve", "vlb", "sweep"):
        fn = {"batch": run_batch, "matmul": run_matmul_bench, "serve": run_serve_bench,
              "vlb": run_vlb_bench, "sweep": run_sweep_bench}[args.workload]
        line = fn(args, rank, world, local_rank)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    line = run_gpu(args, rank, world, local_rank)
    if line is not None:
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline()
            procs = max(1, os.cpu_count() or 1)
            if procs > 1:
                # per process about as much work as the one-core sample
                rows1 = int(line["cpu_baseline"]["sample"].split("rows 0..")[1].split(" ")[0]) + 1
                line["cpu_baseline_all_cores"] = cpu_baseline_parallel(
                    max(64, rows1 // 64 * 64), procs)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
