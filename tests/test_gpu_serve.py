"""Serving loop: continuous batching over a resident store.  Every served
result equals the oracle's (word for word, header included) on the same
inputs, regenerated on the host from their generator recipes, and equals the
same request run alone."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import assert_same_packed, device, lib_ccm, torch, words_np

pytestmark = pytest.mark.gpu


def _dense(recipe, rows, cols):
    seed, stream, lo, hi = recipe
    return synth.uniform_int(seed, stream, rows * cols, lo, hi).reshape(rows, cols)


def _oracle_result(store, r, cache):
    """The oracle's packed result of request r, from host-generated inputs."""
    if r.kind == "pack":
        key = ("pack", r.recipe, tuple(r.dense.shape))
        if key not in cache:
            cache[key] = oracle.pack(_dense(r.recipe, *r.dense.shape))
    elif r.kind == "matvec":
        a = store[r.a]
        key = ("matvec", r.a, r.x.recipe)
        if key not in cache:
            da = _dense(a.recipe, a.rows, a.cols)
            dx = _dense(r.x.recipe, a.cols, 1)
            cache[key] = oracle.pack(oracle.matvec_dense(da, dx.ravel()).reshape(a.rows, 1))
    else:
        a, b = store[r.a], store[r.b]
        key = ("matmul", r.a, r.b)
        if key not in cache:
            da, db = _dense(a.recipe, a.rows, a.cols), _dense(b.recipe, b.rows, b.cols)
            try:
                c = oracle.matmul_dense_f64(da, db)
            except ValueError:  # magnitudes beyond the float64-exact range
                c = oracle.matmul_dense(da, db)
            cache[key] = oracle.pack(c)
    return cache[key]


def test_results_match_oracle_alone_and_in_the_mix():
    ccm = lib_ccm()
    from paper_1303_0270_gb300 import serve
    dev = device()
    # sizes up to 2048 (packs and matmuls above 1024 included), widths 2..20
    store, _ = serve.build_store(1303, 96 << 20, 64, 2048, 2, 20, dev, max_count=24)
    trace = serve.build_trace(1304, store, 300, float("inf"), dev, pack_sizes=(64, 2048),
                              matmul_max_dim=2048)
    kinds = {r.kind for r in trace}
    assert kinds == {"matvec", "pack", "matmul"}
    assert max(max(r.dense.shape) for r in trace if r.kind == "pack") > 1024
    assert max(store[r.a].rows for r in trace if r.kind == "matmul") > 1024
    srv = serve.Server(store, mem_budget=1 << 36, streams=4)
    stats = srv.run(trace)
    s = stats.summary(1.0)
    assert s["requests"] == len(trace)
    assert stats.batched_matvecs > stats.batches  # matvecs really were batched
    cache = {}
    for r in trace:
        assert_same_packed(r.out, _oracle_result(store, r, cache), f"served {r.kind} {r.rid}")
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
