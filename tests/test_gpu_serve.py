"""Serving loop: continuous batching over a resident store; every result is
the same (word for word, header included) alone and in the mix."""
import numpy as np
import pytest

from gpu_util import device, lib_ccm, torch, words_np

pytestmark = pytest.mark.gpu


def test_results_identical_alone_and_in_the_mix():
    ccm = lib_ccm()
    from paper_1303_0270_gb300 import serve
    dev = device()
    store, _ = serve.build_store(1303, 64 << 20, 64, 600, 2, 20, dev, max_count=40)
    trace = serve.build_trace(1304, store, 300, float("inf"), dev, matmul_max_dim=600)
    kinds = {r.kind for r in trace}
    assert kinds == {"matvec", "pack", "matmul"}
    srv = serve.Server(store, mem_budget=1 << 34, streams=4)
    stats = srv.run(trace)
    s = stats.summary(1.0)
    assert s["requests"] == len(trace)
    assert stats.batched_matvecs > stats.batches  # matvecs really were batched
    for r in trace:
        alone = serve.run_alone(store, r, dev)
        h1, h2 = r.out.header(), alone.header()
        assert h1.status == 0 and h2.status == 0, r
        assert (h1.width, h1.is_signed, h1.nwords) == (h2.width, h2.is_signed, h2.nwords), r
        assert np.array_equal(words_np(r.out), words_np(alone)), (r.rid, r.kind)


def test_admission_by_memory():
    ccm = lib_ccm()
    from paper_1303_0270_gb300 import serve
    dev = device()
    store, nbytes = serve.build_store(7, 8 << 20, 64, 300, 2, 12, dev, max_count=12)
    trace = serve.build_trace(8, store, 60, float("inf"), dev, mix=(1.0, 0.0, 0.0))
    # a budget just above the store: only a few requests fit at a time
    budget = srv_used = sum(4 * (ccm.HEADER_WORDS + m.capacity) for m in store)
    one = serve.Server(store, mem_budget=budget + (1 << 20), streams=4)
    stats = one.run(trace)
    assert len(stats.latencies) == 60
    assert stats.peak_bytes <= budget + (1 << 20)
