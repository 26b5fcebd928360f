"""Serving: a streaming request loop over a store of packed matrices kept
resident on the GPU (the paper's streaming-analysis setting: data compressed
once, then operated on as it arrives, Introduction).

Requests (pack / matvec / matmul) arrive over time.  The loop admits a
request when a stream slot is free and its outputs and workspace fit the
memory budget; matvecs admitted together are continuously batched into one
persistent batched-matvec launch; packs and matmuls run on their own streams,
so the work of different requests overlaps on the device.  Completion is
observed through CUDA events (polled, never waited on with a spin in device
code); latency = completion - arrival on the host clock.  All arithmetic
runs in libccm's kernels; this module only schedules.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import torch

from . import ccm
from .batch import BatchMatvec


@dataclass
class Request:
    rid: int
    kind: str                 # "matvec" | "pack" | "matmul"
    arrival: float            # seconds from the start of the trace
    a: int = -1               # store index (matvec, matmul)
    b: int = -1               # store index (matmul)
    x: object = None          # packed x (matvec)
    dense: object = None      # dense int64 tensor (pack)
    out: object = None        # packed result
    admitted: float = -1.0
    done: float = -1.0
    event: object = None
    nbytes: int = 0
    recipe: tuple = None      # pack: how `dense` was generated (seed, stream, lo, hi)


@dataclass
class Stats:
    latencies: list = field(default_factory=list)
    kinds: list = field(default_factory=list)
    batches: int = 0
    batched_matvecs: int = 0
    max_inflight: int = 0
    peak_bytes: int = 0

    def summary(self, wall: float) -> dict:
        import numpy as np
        lat = np.array(self.latencies) * 1e3
        out = {"requests": len(lat), "wall_s": round(wall, 4),
               "throughput_rps": round(len(lat) / wall, 2) if wall > 0 else None,
               "p50_ms": round(float(np.percentile(lat, 50)), 4) if len(lat) else None,
               "p99_ms": round(float(np.percentile(lat, 99)), 4) if len(lat) else None,
               "mean_ms": round(float(lat.mean()), 4) if len(lat) else None,
               "batches": self.batches, "batched_matvecs": self.batched_matvecs,
               "max_inflight": self.max_inflight, "peak_bytes": self.peak_bytes}
        for k in ("matvec", "pack", "matmul"):
            sel = np.array([kk == k for kk in self.kinds])
            if sel.any():
                out[f"p50_ms_{k}"] = round(float(np.percentile(lat[sel], 50)), 4)
                out[f"p99_ms_{k}"] = round(float(np.percentile(lat[sel], 99)), 4)
        return out


class Server:
    """Continuous-batching loop over a resident store of packed matrices."""

    def __init__(self, store, mem_budget: int, streams: int = 4, batching: bool = True,
                 device=None, heavy_streams: int = 2):
        self.store = store                     # list of PackedMatrix (resident)
        self.device = device or store[0].device
        self.mem_budget = int(mem_budget)
        # matvecs and packs (sub-millisecond) on high-priority streams, matmuls
        # (up to ~10^2 ms at 8192^3) on low-priority ones: when SMs free up,
        # the short requests' blocks are scheduled first
        lo, hi = torch.cuda.Stream.priority_range() if hasattr(torch.cuda.Stream,
                                                                "priority_range") else (0, 0)
        self.light = list(range(streams))
        self.heavy = list(range(streams, streams + heavy_streams)) if heavy_streams else []
        self.streams = ([torch.cuda.Stream(self.device, priority=hi) for _ in self.light] +
                        [torch.cuda.Stream(self.device, priority=lo) for _ in self.heavy])
        self.busy = [None] * len(self.streams)  # what runs on each stream
        self.batching = batching
        self.used = sum(4 * (ccm.HEADER_WORDS + m.capacity) for m in store)

    # -- per-request resources ---------------------------------------------
    def _out_capacity(self, r: Request) -> int:
        """Output words: the library's result-width bound (matvec, matmul);
        64 bits per entry for a pack, whose width is only known once packed."""
        if r.kind == "matvec":
            a = self.store[r.a]
            return ccm.words_for(a.rows, 1, ccm.bound_matvec(a, r.x))
        if r.kind == "pack":
            rows, cols = r.dense.shape
            return ccm.words_for(rows, cols, 64)
        a, b = self.store[r.a], self.store[r.b]
        return ccm.words_for(a.rows, b.cols, ccm.bound_matmul(a, b))

    def _out_bytes(self, r: Request) -> int:
        cap = 4 * self._out_capacity(r) + 64
        if r.kind == "matvec":
            a = self.store[r.a]
            return cap + 16 * a.rows + 8 * a.cols + 512
        if r.kind == "pack":
            rows, cols = r.dense.shape
            return cap + ccm.workspace_bytes(ccm.OP_PACK, rows, cols, self._out_capacity(r))
        a, b = self.store[r.a], self.store[r.b]
        return cap + ccm.workspace_bytes(ccm.OP_MATMUL, a.rows, a.cols, b.cols)

    def _launch_single(self, r: Request, s: torch.cuda.Stream):
        with torch.cuda.stream(s):
            cap = self._out_capacity(r)
            if r.kind == "pack":
                rows, cols = r.dense.shape
                r.out = ccm.PackedMatrix(rows, cols, cap, self.device)
                ccm.pack_into(r.dense, r.out, stream=s)
            elif r.kind == "matmul":
                a, b = self.store[r.a], self.store[r.b]
                r.out = ccm.PackedMatrix(a.rows, b.cols, cap, self.device)
                ccm.matmul_into(a, b, r.out, stream=s)
            else:
                a = self.store[r.a]
                r.out = ccm.PackedMatrix(a.rows, 1, cap, self.device)
                ccm.matvec_into(a, r.x, r.out, stream=s)
            r.event = torch.cuda.Event()
            r.event.record(s)

    def _launch_batch(self, reqs, s: torch.cuda.Stream):
        mats = [self.store[r.a] for r in reqs]
        xs = [r.x for r in reqs]
        ys = [ccm.PackedMatrix(self.store[r_.a].rows, 1, self._out_capacity(r_), self.device)
              for r_ in reqs]
        with torch.cuda.stream(s):
            bm = BatchMatvec(mats, xs, ys, unit_segments=256)
            bm.launch(stream=s)
            ev = torch.cuda.Event()
            ev.record(s)
        for r, y in zip(reqs, ys):
            r.out = y
            r.event = ev
        return bm

    # -- the loop ----------------------------------------------------------
    def run(self, trace, stats: Stats | None = None, max_batch: int = 512,
            keep_result=None) -> Stats:
        """Serve the trace.  `keep_result(r)` says whether request r's result
        stays attached to it after completion (default: all); the others are
        dropped as they complete, as a server hands results back."""
        stats = stats or Stats()
        pending = deque(sorted(trace, key=lambda r: r.arrival))
        # one FIFO per kind: admission looks at the three heads only
        queues = {"matvec": deque(), "pack": deque(), "matmul": deque()}
        nwait = 0
        inflight = []          # (slot, [requests], keepalive)
        t0 = time.perf_counter()
        while pending or nwait or inflight:
            now = time.perf_counter() - t0
            while pending and pending[0].arrival <= now:
                r = pending.popleft()
                queues[r.kind].append(r)
                nwait += 1
            # retire finished work and free its slot and memory
            still = []
            for slot, reqs, keepalive in inflight:
                if reqs[0].event.query():
                    tdone = time.perf_counter() - t0
                    for r in reqs:
                        r.done = tdone
                        stats.latencies.append(r.done - r.arrival)
                        stats.kinds.append(r.kind)
                        self.used -= r.nbytes
                        if keep_result is not None and not keep_result(r):
                            r.out = None
                        r.event = None
                    self.busy[slot] = None
                else:
                    still.append((slot, reqs, keepalive))
            inflight = still
            # admit, earliest arrival first among the kinds whose slot class
            # has a free slot (a matmul waiting for a heavy slot does not hold
            # up the rest), while memory fits
            free = [i for i in self.light if self.busy[i] is None]
            free_heavy = [i for i in self.heavy if self.busy[i] is None]
            launched = False
            while nwait:
                head, pool = None, None
                for kind, q in queues.items():
                    if not q:
                        continue
                    heavy = kind == "matmul" and bool(self.heavy)
                    p = free_heavy if heavy else free
                    if p and (head is None or q[0].arrival < head.arrival):
                        head, pool = q[0], p
                if head is None:
                    break
                q = queues[head.kind]
                if self.batching and head.kind == "matvec":
                    group, need = [], 0
                    while q and len(group) < max_batch:
                        nb = self._out_bytes(q[0])
                        if self.used + need + nb > self.mem_budget:
                            break
                        r = q.popleft()
                        r.nbytes = nb
                        r.admitted = now
                        group.append(r)
                        need += nb
                    if not group:
                        break
                    nwait -= len(group)
                    self.used += need
                    slot = pool.pop(0)
                    keepalive = self._launch_batch(group, self.streams[slot])
                    self.busy[slot] = group
                    inflight.append((slot, group, keepalive))
                    stats.batches += 1
                    stats.batched_matvecs += len(group)
                else:
                    nb = self._out_bytes(head)
                    if self.used + nb > self.mem_budget:
                        break
                    q.popleft()
                    nwait -= 1
                    head.nbytes = nb
                    head.admitted = now
                    self.used += nb
                    slot = pool.pop(0)
                    self._launch_single(head, self.streams[slot])
                    self.busy[slot] = [head]
                    inflight.append((slot, [head], None))
                launched = True
            stats.max_inflight = max(stats.max_inflight, len(inflight))
            stats.peak_bytes = max(stats.peak_bytes, self.used)
            if not launched and not inflight and pending:
                # idle until the next arrival
                delay = pending[0].arrival - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(min(delay, 0.001))
        torch.cuda.synchronize(self.device)
        return stats


def run_alone(store, r: Request, device) -> "ccm.PackedMatrix":
    """The same request on its own (default stream, no batching)."""
    if r.kind == "pack":
        rows, cols = r.dense.shape
        out = ccm.PackedMatrix(rows, cols, ccm.words_for(rows, cols, 64), device)
        return ccm.pack_into(r.dense, out)
    if r.kind == "matmul":
        a, b = store[r.a], store[r.b]
        out = ccm.PackedMatrix(a.rows, b.cols, ccm.words_for(a.rows, b.cols,
                                                             ccm.bound_matmul(a, b)), device)
        return ccm.matmul_into(a, b, out)
    a = store[r.a]
    out = ccm.PackedMatrix(a.rows, 1, ccm.words_for(a.rows, 1, ccm.bound_matvec(a, r.x)), device)
    return ccm.matvec_into(a, r.x, out)


# ---------------------------------------------------------------------------
# Workload construction (store, request trace) shared by the bench and tests
# ---------------------------------------------------------------------------
def build_store(seed: int, target_bytes: int, lo: int, hi: int, wlo: int, whi: int, device,
                max_count: int = 100000):
    """A chain of packed matrices A_i (d_i x d_{i+1}), dims log-uniform in
    [lo, hi), widths uniform in [wlo, whi], values uniform over the signed
    b-bit range, until `target_bytes` of packed words; consecutive matrices
    multiply."""
    import synth
    dims = synth.log_uniform_sizes(seed, synth.STREAM_SHAPES, max_count + 1, lo, hi)
    widths = synth.uniform_int(seed, synth.STREAM_WIDTHS, max_count, wlo, whi)
    store, total = [], 0
    dense = None
    for i in range(max_count):
        r, c, b = int(dims[i]), int(dims[i + 1]), int(widths[i])
        nbytes = 4 * ccm.words_for(r, c, b)
        if store and total + nbytes > target_bytes:
            break
        if dense is None or dense.numel() < r * c:
            dense = torch.empty(max(r * c, hi * hi // 4), dtype=torch.int64, device=device)
        lo_v, hi_v = synth.signed_range(b)
        ccm.gen_uniform(r * c, synth.batch_matrix_seed(seed, i), synth.STREAM_A, lo_v, hi_v,
                        out=dense[: r * c])
        m = ccm.PackedMatrix(r, c, ccm.words_for(r, c, b), device)
        ccm.pack_into(dense[: r * c].view(r, c), m)
        # the generator inputs of this matrix (entries uniform in [lo, hi])
        m.recipe = (synth.batch_matrix_seed(seed, i), synth.STREAM_A, lo_v, hi_v)
        store.append(m)
        total += nbytes
    torch.cuda.synchronize(device)
    return store, total


def build_trace(seed: int, store, count: int, rate: float, device, mix=(0.6, 0.3, 0.1),
                pack_sizes=(64, 8192), matmul_max_dim: int = 8192):
    """`count` requests with Poisson(rate) arrivals (rate = inf: all at t = 0)
    mixing matvec / pack / matmul in the proportions `mix`.  Matvec uses a
    packed signed 8-bit x per store matrix; pack draws a dense matrix
    (dims log-uniform in pack_sizes) from a pool; matmul multiplies consecutive
    store matrices A_i A_{i+1} whose dims are at most matmul_max_dim.  Each
    x (attribute `recipe`) and each pack request (`Request.recipe`) records
    the generator inputs of its entries."""
    import numpy as np

    import synth
    u = synth.u53(synth.u64(seed, synth.STREAM_ARRIVALS, 0, count))
    gaps = -np.log1p(-u) / rate if np.isfinite(rate) else np.zeros(count)
    arrivals = np.cumsum(gaps)
    kinds_u = synth.u53(synth.u64(seed, synth.STREAM_KINDS, 0, count))
    pick = synth.u64(seed, synth.STREAM_INDEX, 0, count)
    xs = {}
    xd = torch.empty(max(m.cols for m in store), dtype=torch.int64, device=device)
    for i, m in enumerate(store):
        if m.cols not in xs:
            ccm.gen_uniform(m.cols, seed + i, synth.STREAM_X, -128, 127, out=xd[: m.cols])
            xs[m.cols] = ccm.pack(xd[: m.cols].view(-1, 1).clone())
            xs[m.cols].recipe = (seed + i, synth.STREAM_X, -128, 127)
    mm_ok = [i for i in range(len(store) - 1)
             if max(store[i].rows, store[i].cols, store[i + 1].cols) <= matmul_max_dim]
    pdims = synth.log_uniform_sizes(seed + 7, synth.STREAM_SHAPES, 16, pack_sizes[0], pack_sizes[1])
    pool, recipes = [], []
    for j in range(8):
        r, c = int(pdims[2 * j]), int(pdims[2 * j + 1])
        d = torch.empty(r * c, dtype=torch.int64, device=device)
        ccm.gen_uniform(r * c, seed + 100 + j, synth.STREAM_A, -(1 << 11), (1 << 11) - 1, out=d)
        pool.append(d.view(r, c))
        recipes.append((seed + 100 + j, synth.STREAM_A, -(1 << 11), (1 << 11) - 1))
    trace = []
    for k in range(count):
        p = int(pick[k])
        if kinds_u[k] < mix[0] or (kinds_u[k] >= mix[0] + mix[1] and not mm_ok):
            a = p % len(store)
            trace.append(Request(k, "matvec", float(arrivals[k]), a=a, x=xs[store[a].cols]))
        elif kinds_u[k] < mix[0] + mix[1]:
            trace.append(Request(k, "pack", float(arrivals[k]), dense=pool[p % len(pool)],
                                 recipe=recipes[p % len(pool)]))
        else:
            i = mm_ok[p % len(mm_ok)]
            trace.append(Request(k, "matmul", float(arrivals[k]), a=i, b=i + 1))
    torch.cuda.synchronize(device)
    return trace
