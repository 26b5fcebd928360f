"""Helpers for the GPU parity tests: move seeded inputs to the GPU and compare
packed results with the oracle word for word (header fields included)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def device():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def lib_ccm():
    from paper_1303_0270_gb300 import build, ccm
    build.build()
    ccm.lib()
    return ccm


def to_dev(a: np.ndarray, dtype=np.int64):
    return torch.from_numpy(np.ascontiguousarray(a.astype(dtype))).to(device())


def words_np(p) -> np.ndarray:
    return p.words().cpu().numpy().view(np.uint32)


def assert_same_packed(p, o, what=""):
    """GPU packed matrix `p` equals oracle Packed `o`: shape, width, sign,
    word count and every word (padding included)."""
    h = p.header()
    assert h.status == 0, f"{what}: status {h.status}"
    assert h.magic == 0x314D4343
    assert (h.rows, h.cols) == (o.rows, o.cols), what
    assert (h.width, h.is_signed) == (o.width, o.is_signed), \
        f"{what}: width {h.width}/{h.is_signed} vs oracle {o.width}/{o.is_signed}"
    assert h.nwords == o.words.size, what
    w = words_np(p)
    if not np.array_equal(w, o.words):
        bad = np.nonzero(w != o.words)[0]
        raise AssertionError(f"{what}: {bad.size} words differ, first at {bad[:5]}: "
                             f"{w[bad[:5]]} vs {o.words[bad[:5]]}")
