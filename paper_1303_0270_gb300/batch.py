"""Batched matvec: thousands of packed matrices of uneven shapes and widths
in one persistent launch (C ABI: ccm_batch_plan / ccm_batch_matvec), with an
autotuner for the work-unit size, the ring depth and the stage size (which
sets how many segments of 32 fields each lane decodes per stage), and
CUDA-graph replay.  Argument marshalling and orchestration only: the arithmetic runs in
libccm's kernels."""
from __future__ import annotations

import ctypes
import json
import os
import time

import torch

from . import ccm


class BatchMatvec:
    """y_i = A_i x_i for every (A_i, x_i) of a batch of packed matrices."""

    def __init__(self, mats, xs, ys=None, unit_segments: int = 256, grid: int = 0):
        if len(mats) != len(xs) or not mats:
            raise ValueError("need as many x as A, and at least one")
        self.mats, self.xs = list(mats), list(xs)
        self.device = self.mats[0].device
        if ys is None:
            ys = []
            for a, x in zip(self.mats, self.xs):
                bound = ccm.bound_matvec(a, x)
                ys.append(ccm.PackedMatrix(a.rows, 1, ccm.words_for(a.rows, 1, bound), self.device))
        self.ys = list(ys)
        n = len(self.mats)
        self.entries = (ccm.BatchEntry * n)()
        for i, (a, x, y) in enumerate(zip(self.mats, self.xs, self.ys)):
            self.entries[i].a, self.entries[i].x, self.entries[i].y = a.c(), x.c(), y.c()
        self.count = n
        self.grid = grid
        self.slots = 0  # ring slots per warp (0 = the library's default, else 2..4)
        self.stage_bytes = 0  # bytes of A per warp stage (0 = the library's default)
        self.graph = None
        L = ccm.lib()
        ws = L.ccm_batch_workspace_bytes(self.entries, n)
        self.ws = torch.empty(max(ws, 256), dtype=torch.uint8, device=self.device)
        self.plan = None
        self.info = ccm.BatchInfo()
        self.set_unit_segments(unit_segments)

    def set_unit_segments(self, unit_segments: int):
        L = ccm.lib()
        nbytes = L.ccm_batch_plan_bytes(self.entries, self.count, unit_segments)
        if self.plan is None or self.plan.numel() < nbytes:
            self.plan = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        torch.cuda.synchronize(self.device)
        ccm._check(L.ccm_batch_plan(self.entries, self.count, unit_segments,
                                    ctypes.c_void_p(self.plan.data_ptr()), self.plan.numel(),
                                    ctypes.byref(self.info)), "ccm_batch_plan")
        self.unit_segments = unit_segments
        self.graph = None

    def launch(self, stream=None):
        """Both launches of one batched matvec, asynchronous."""
        self.info.slots = self.slots
        self.info.stage_bytes = self.stage_bytes
        ccm._check(ccm.lib().ccm_batch_matvec(
            ctypes.c_void_p(self.plan.data_ptr()), ctypes.byref(self.info),
            ctypes.c_void_p(self.ws.data_ptr()), self.ws.numel(), int(self.grid),
            ccm._stream(stream)), "ccm_batch_matvec")
        for y in self.ys:
            y._written()

    def capture(self):
        """Capture the batched matvec in a CUDA graph (replayed by run())."""
        s = torch.cuda.Stream(self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            self.launch(stream=s)  # warm-up outside the graph
        torch.cuda.current_stream(self.device).wait_stream(s)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.launch(stream=torch.cuda.current_stream(self.device))
        self.graph = g
        return g

    def run(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()
        for y in self.ys:
            y._written()

    # -- autotuning ---------------------------------------------------------
    def signature(self) -> str:
        import hashlib
        h = hashlib.sha256()
        for a, x in zip(self.mats, self.xs):
            h.update(f"{a.rows},{a.cols},{a.capacity},{x.capacity};".encode())
        return h.hexdigest()[:24]

    def autotune(self, candidates=None, reps: int = 3, cache: str | None = None):
        """Time each (unit_segments, grid, ring slots, stage bytes) candidate
        on this batch and keep the fastest; results are cached by batch signature (in memory and, when
        `cache` or $CCM_AUTOTUNE_CACHE names a file, on disk)."""
        cache = cache or os.environ.get("CCM_AUTOTUNE_CACHE")
        key = self.signature()
        store = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                store = json.load(f)
        if key in store:
            us, grid = store[key]["unit_segments"], store[key]["grid"]
            self.grid = grid
            self.slots = store[key].get("slots", 0)
            self.stage_bytes = store[key].get("stage_bytes", 0)
            if us != self.unit_segments:
                self.set_unit_segments(us)
            return store[key]
        if candidates is None:
            # work-unit size x ring depth x stage bytes (segments per lane
            # per stage: about stage_bytes / (128 b)), one resident wave
            candidates = [(us, 0, k, sb) for us in (256, 1024, 4096) for k in (2, 3, 4)
                          for sb in (768, 1536, 3072)]
        best = None
        results = []
        for cand in candidates:
            us, grid = cand[0], cand[1]
            slots = cand[2] if len(cand) > 2 else 0
            stage = cand[3] if len(cand) > 3 else 0
            if us != self.unit_segments or self.plan is None:
                self.set_unit_segments(us)
            self.grid = grid
            self.slots = slots
            self.stage_bytes = stage
            try:
                self.launch()
            except ccm.CCMError:
                continue  # (ring too large for shared memory at this width bound)
            self.launch()
            torch.cuda.synchronize(self.device)
            times = []
            for _ in range(reps):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                self.launch()
                e1.record()
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            t = min(times)
            res = {"unit_segments": us, "grid": grid, "slots": slots, "stage_bytes": stage,
                   "ms": t}
            results.append(res)
            if best is None or t < best["ms"]:
                best = dict(res)
        self.set_unit_segments(best["unit_segments"])
        self.grid = best["grid"]
        self.slots = best["slots"]
        self.stage_bytes = best["stage_bytes"]
        best["tried"] = results
        store[key] = best
        if cache:
            tmp = cache + f".{os.getpid()}"
            with open(tmp, "w") as f:
                json.dump(store, f)
            os.replace(tmp, cache)
        return best
