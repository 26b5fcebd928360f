"""Python binding of libccm (include/ccm.h): argument marshalling only.

Every step of every operation runs in the CUDA kernels of libccm.so; PyTorch
only supplies device memory (one int32 tensor per packed matrix holding the
64-byte header followed by the words) and the current CUDA stream.  There is
no CPU fallback: importing this module without a built libccm.so raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

OK, E_INVAL, E_SHAPE, E_WIDTH, E_OVERFLOW, E_CAPACITY, E_RANGE, E_CUDA, E_TIMEOUT, E_INPUT = (
    0, -1, -2, -3, -4, -5, -6, -7, -8, -9)
I32, I64 = 0, 1
OP_MATVEC, OP_MATMUL, OP_PACK, OP_VLB, OP_VLB_MATVEC = 1, 2, 3, 4, 5
VLB_MAGIC = 0x31564343
VLB_INDEX_STRIDE = 64
MATMUL_AUTO, MATMUL_TENSOR, MATMUL_CUDACORE = 0, 1, 2
MAGIC = 0x314D4343
HEADER_WORDS = 16  # 64 bytes


class CCMError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {status_str(status)} ({status})" if what else status_str(status))


class Header(ctypes.Structure):
    _fields_ = [("magic", ctypes.c_uint32), ("width", ctypes.c_int32),
                ("is_signed", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rows", ctypes.c_uint64), ("cols", ctypes.c_uint64),
                ("nwords", ctypes.c_uint64), ("stat_or", ctypes.c_uint64),
                ("stat_neg", ctypes.c_uint32), ("reserved0", ctypes.c_uint32),
                ("reserved1", ctypes.c_uint64)]


class Matrix(ctypes.Structure):
    _fields_ = [("hdr", ctypes.c_void_p), ("words", ctypes.c_void_p),
                ("capacity", ctypes.c_uint64), ("rows", ctypes.c_uint64),
                ("cols", ctypes.c_uint64)]


class BatchEntry(ctypes.Structure):
    _fields_ = [("a", Matrix), ("x", Matrix), ("y", Matrix)]


class BatchInfo(ctypes.Structure):
    _fields_ = [("count", ctypes.c_uint32), ("units", ctypes.c_uint32),
                ("y_rows", ctypes.c_uint64), ("unit_segments", ctypes.c_uint32),
                ("max_cols", ctypes.c_uint32), ("plan_bytes", ctypes.c_uint64),
                ("max_width", ctypes.c_uint32), ("slots", ctypes.c_uint32),
                ("x_ints", ctypes.c_uint64), ("stage_bytes", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


assert ctypes.sizeof(Header) == 64

_lib = None

# Every exported symbol of include/ccm.h with its (argtypes, restype).
_vp, _u64, _i64, _i32, _sz = (ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int64, ctypes.c_int,
                              ctypes.c_size_t)
_MP = ctypes.POINTER(Matrix)
SIGNATURES = {
    "ccm_words_for": ([_u64, _u64, _i32], _u64),
    "ccm_status_str": ([_i32], ctypes.c_char_p),
    "ccm_version": ([], _i32),
    "ccm_measure": ([_vp, _i32, _u64, _u64, _vp, _vp], _i32),
    "ccm_pack": ([_vp, _i32, _u64, _u64, _MP, _vp, _sz, _vp], _i32),
    "ccm_unpack": ([_MP, _vp, _i32, _vp, _vp], _i32),
    "ccm_get": ([_MP, _vp, _u64, _vp, _vp, _vp], _i32),
    "ccm_add": ([_MP, _MP, _MP, _vp, _sz, _vp], _i32),
    "ccm_scale": ([_MP, _i64, _MP, _vp, _sz, _vp], _i32),
    "ccm_matvec": ([_MP, _MP, _MP, _vp, _sz, _vp], _i32),
    "ccm_matmul": ([_MP, _MP, _MP, _i32, _vp, _sz, _vp], _i32),
    "ccm_workspace_bytes": ([_i32, _u64, _u64, _u64], _sz),
    "ccm_header_read": ([_vp, ctypes.POINTER(Header), _vp], _i32),
    "ccm_gen_uniform": ([_vp, _u64, _u64, _u64, _u64, _i64, _i64, _vp], _i32),
    "ccm_gen_poisson": ([_vp, _u64, _u64, _u64, _u64, _vp, ctypes.c_uint32, _vp], _i32),
    "ccm_batch_plan_bytes": ([ctypes.POINTER(BatchEntry), _i32, ctypes.c_uint32], _sz),
    "ccm_batch_workspace_bytes": ([ctypes.POINTER(BatchEntry), _i32], _sz),
    "ccm_batch_plan": ([ctypes.POINTER(BatchEntry), _i32, ctypes.c_uint32, _vp, _sz,
                        ctypes.POINTER(BatchInfo)], _i32),
    "ccm_batch_matvec": ([_vp, ctypes.POINTER(BatchInfo), _vp, _sz, _i32, _vp], _i32),
    "ccm_matvec_static": ([_MP, _MP, _MP, _vp], _i32),
    "ccm_vlb_index_entries": ([_u64, _u64], _u64),
    "ccm_vlb_pack": ([_vp, _i32, _u64, _u64, _vp, _vp, _u64, _vp, _vp, _sz, _vp], _i32),
    "ccm_vlb_unpack": ([_vp, _vp, _u64, _vp, _u64, _u64, _vp, _i32, _vp, _vp], _i32),
    "ccm_matvec2": ([_MP, _MP, _MP, _MP, _MP, _vp, _sz, _vp], _i32),
    "ccm_vlb_matvec": ([_vp, _vp, _u64, _vp, _u64, _u64, _MP, _MP, _vp, _sz, _vp], _i32),
    "ccm_bound_add": ([_i32, _i32, _i32, _i32], _i32),
    "ccm_bound_scale": ([_i32, _i32, _i64], _i32),
    "ccm_bound_matvec": ([_i32, _i32, _i32, _i32, _u64], _i32),
    "ccm_bound_matmul": ([_i32, _i32, _i32, _i32, _u64], _i32),
    "ccm_repack": ([_MP, _i32, _i32, _MP, _u64, _vp], _i32),
    "ccm_launch_count": ([], _u64),
    "ccm_profile_next": ([_vp, _vp], _i32),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """The loaded libccm.so; raises when it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"libccm.so is not built ({path}); run __graft_entry__.build() "
                               "or python -m paper_1303_0270_gb300.build")
        L = ctypes.CDLL(path)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def launch_count() -> int:
    """Kernels libccm has launched in this process."""
    return int(lib().ccm_launch_count())


def profile_next(start: "torch.cuda.Event", stop: "torch.cuda.Event"):
    """Bracket the main kernel of the next ccm_* call with these two events."""
    _check(lib().ccm_profile_next(ctypes.c_void_p(start.cuda_event),
                                  ctypes.c_void_p(stop.cuda_event)), "ccm_profile_next")


def status_str(status: int) -> str:
    return lib().ccm_status_str(int(status)).decode()


def _check(status: int, what: str):
    if status != OK:
        raise CCMError(status, what)


def _stream(stream=None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def words_for(rows: int, cols: int, width: int) -> int:
    return int(lib().ccm_words_for(rows, cols, width))


class PackedMatrix:
    """A matrix in SM form on the GPU: one int32 tensor = header + words."""

    def __init__(self, rows: int, cols: int, capacity: int, device=None):
        self.rows, self.cols = int(rows), int(cols)
        self.capacity = int(capacity)
        dev = torch.device(device) if device is not None else torch.device("cuda")
        self.buf = torch.empty(HEADER_WORDS + self.capacity, dtype=torch.int32, device=dev)
        self._host = None  # cached host copy of the header, valid until the next write

    @property
    def device(self):
        return self.buf.device

    @property
    def hdr_ptr(self) -> int:
        return self.buf.data_ptr()

    @property
    def words_ptr(self) -> int:
        return self.buf.data_ptr() + 4 * HEADER_WORDS

    def c(self) -> Matrix:
        return Matrix(self.hdr_ptr, self.words_ptr, self.capacity, self.rows, self.cols)

    def _written(self):
        self._host = None

    def header(self, stream=None) -> Header:
        """Synchronous read of the device header (cached until the next write)."""
        if self._host is None:
            h = Header()
            _check(lib().ccm_header_read(ctypes.c_void_p(self.hdr_ptr), ctypes.byref(h),
                                         _stream(stream)), "ccm_header_read")
            self._host = h
        return self._host

    @property
    def width(self) -> int:
        return self.header().width

    @property
    def is_signed(self) -> int:
        return self.header().is_signed

    @property
    def status(self) -> int:
        return self.header().status

    @property
    def nwords(self) -> int:
        return int(self.header().nwords)

    def check(self) -> "PackedMatrix":
        h = self.header()
        _check(h.status, "packed matrix")
        return self

    def words(self) -> torch.Tensor:
        """The data words (with padding) as a uint32-valued int32 view."""
        return self.buf[HEADER_WORDS:HEADER_WORDS + self.nwords]

    def header_tensor(self) -> torch.Tensor:
        return self.buf[:HEADER_WORDS]



def _as_dense(t: torch.Tensor):
    if t.dtype not in (torch.int32, torch.int64):
        raise TypeError("dense input must be int32 or int64")
    if not t.is_cuda:
        raise ValueError("dense input must be a CUDA tensor")
    t = t.contiguous()
    if t.dim() == 1:
        rows, cols = t.shape[0], 1
    elif t.dim() == 2:
        rows, cols = t.shape
    else:
        raise ValueError("dense input must be 1-D or 2-D")
    return t, int(rows), int(cols), (I64 if t.dtype == torch.int64 else I32)


def measure(t: torch.Tensor, stream=None) -> tuple[int, int]:
    """(width, is_signed) of a dense matrix by the width rule (synchronous)."""
    t, rows, cols, dt = _as_dense(t)
    hdr = torch.empty(HEADER_WORDS, dtype=torch.int32, device=t.device)
    _check(lib().ccm_measure(ctypes.c_void_p(t.data_ptr()), dt, rows, cols,
                             ctypes.c_void_p(hdr.data_ptr()), _stream(stream)), "ccm_measure")
    h = Header()
    _check(lib().ccm_header_read(ctypes.c_void_p(hdr.data_ptr()), ctypes.byref(h),
                                 _stream(stream)), "ccm_header_read")
    _check(h.status, "ccm_measure")
    return h.width, h.is_signed


def pack_into(t: torch.Tensor, out: PackedMatrix, stream=None, ws: torch.Tensor | None = None,
              single_pass: bool = True) -> PackedMatrix:
    """Asynchronous SM pack of a dense CUDA tensor into a preallocated matrix
    (single pass over the dense data when a workspace applies)."""
    t, rows, cols, dt = _as_dense(t)
    m = out.c()
    if ws is None and single_pass:
        nb = workspace_bytes(OP_PACK, rows, cols, out.capacity)
        ws = torch.empty(nb, dtype=torch.uint8, device=t.device) if nb else None
    wsp = ctypes.c_void_p(ws.data_ptr()) if ws is not None else None
    _check(lib().ccm_pack(ctypes.c_void_p(t.data_ptr()), dt, rows, cols, ctypes.byref(m),
                          wsp, ws.numel() if ws is not None else 0, _stream(stream)), "ccm_pack")
    out._written()
    return out


def pack(t: torch.Tensor, capacity: int | None = None, stream=None) -> PackedMatrix:
    """SM compression of a dense int32/int64 CUDA tensor.  Without `capacity`
    the width is measured first (one synchronisation) and the words sized
    exactly."""
    t, rows, cols, _ = _as_dense(t)
    if capacity is None:
        b, _ = measure(t, stream)
        capacity = words_for(rows, cols, b)
    out = PackedMatrix(rows, cols, capacity, t.device)
    return pack_into(t, out, stream)


def unpack(a: PackedMatrix, dtype=torch.int64, out: torch.Tensor | None = None, stream=None,
           check: bool = True) -> torch.Tensor:
    dt = I64 if dtype == torch.int64 else I32
    if out is None:
        out = torch.empty((a.rows, a.cols), dtype=dtype, device=a.device)
    err = torch.empty(1, dtype=torch.int32, device=a.device)
    m = a.c()
    _check(lib().ccm_unpack(ctypes.byref(m), ctypes.c_void_p(out.data_ptr()), dt,
                            ctypes.c_void_p(err.data_ptr()), _stream(stream)), "ccm_unpack")
    if check:
        _check(int(err.item()), "ccm_unpack")
    return out


def get(a: PackedMatrix, idx: torch.Tensor, stream=None, check: bool = True) -> torch.Tensor:
    """Entries at flat row-major indices i*cols + j (int64 CUDA tensor)."""
    idx = idx.to(device=a.device, dtype=torch.int64).contiguous()
    out = torch.empty(idx.numel(), dtype=torch.int64, device=a.device)
    err = torch.empty(1, dtype=torch.int32, device=a.device)
    m = a.c()
    _check(lib().ccm_get(ctypes.byref(m), ctypes.c_void_p(idx.data_ptr()), idx.numel(),
                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(err.data_ptr()),
                         _stream(stream)), "ccm_get")
    if check:
        _check(int(err.item()), "ccm_get")
    return out


def _bound(status: int, what: str) -> int:
    if status < 0:
        raise CCMError(status, what)
    return int(status)


def bound_add(a: PackedMatrix, b: PackedMatrix) -> int:
    """Width that holds every possible A + B (ccm_bound_add)."""
    return _bound(lib().ccm_bound_add(a.width, a.is_signed, b.width, b.is_signed),
                  "ccm_bound_add")


def bound_scale(a: PackedMatrix, s: int) -> int:
    return _bound(lib().ccm_bound_scale(a.width, a.is_signed, int(s)), "ccm_bound_scale")


def bound_matvec(a: PackedMatrix, x: PackedMatrix) -> int:
    return _bound(lib().ccm_bound_matvec(a.width, a.is_signed, x.width, x.is_signed, a.cols),
                  "ccm_bound_matvec")


def bound_matmul(a: PackedMatrix, b: PackedMatrix) -> int:
    return _bound(lib().ccm_bound_matmul(a.width, a.is_signed, b.width, b.is_signed, a.cols),
                  "ccm_bound_matmul")


def add_into(a: PackedMatrix, b: PackedMatrix, c: PackedMatrix, stream=None) -> PackedMatrix:
    ma, mb, mc = a.c(), b.c(), c.c()
    _check(lib().ccm_add(ctypes.byref(ma), ctypes.byref(mb), ctypes.byref(mc), None, 0,
                         _stream(stream)), "ccm_add")
    c._written()
    return c


def add(a: PackedMatrix, b: PackedMatrix, capacity: int | None = None, stream=None):
    if capacity is None:
        capacity = words_for(a.rows, a.cols, bound_add(a, b))
    return add_into(a, b, PackedMatrix(a.rows, a.cols, capacity, a.device), stream)


def scale_into(a: PackedMatrix, s: int, c: PackedMatrix, stream=None) -> PackedMatrix:
    ma, mc = a.c(), c.c()
    _check(lib().ccm_scale(ctypes.byref(ma), int(s), ctypes.byref(mc), None, 0, _stream(stream)),
           "ccm_scale")
    c._written()
    return c


def scale(a: PackedMatrix, s: int, capacity: int | None = None, stream=None):
    if capacity is None:
        capacity = words_for(a.rows, a.cols, bound_scale(a, s))
    return scale_into(a, s, PackedMatrix(a.rows, a.cols, capacity, a.device), stream)


def repack_into(a: PackedMatrix, width: int, is_signed: int, out: PackedMatrix,
                row_offset: int = 0, stream=None) -> PackedMatrix:
    """a's fields at `width` (and sign mode) into rows [row_offset, +a.rows)
    of out; every other word of out is zero (ccm_repack)."""
    ma, mo = a.c(), out.c()
    _check(lib().ccm_repack(ctypes.byref(ma), int(width), int(is_signed), ctypes.byref(mo),
                            int(row_offset), _stream(stream)), "ccm_repack")
    out._written()
    return out


def workspace_bytes(op: int, m: int, k: int, n: int) -> int:
    return int(lib().ccm_workspace_bytes(op, m, k, n))


def workspace(op: int, m: int, k: int, n: int, device) -> torch.Tensor:
    return torch.empty(max(workspace_bytes(op, m, k, n), 256), dtype=torch.uint8, device=device)


def matvec_into(a: PackedMatrix, x: PackedMatrix, y: PackedMatrix, ws: torch.Tensor | None = None,
                stream=None) -> PackedMatrix:
    if ws is None:
        ws = workspace(OP_MATVEC, a.rows, a.cols, 1, a.device)
    ma, mx, my = a.c(), x.c(), y.c()
    _check(lib().ccm_matvec(ctypes.byref(ma), ctypes.byref(mx), ctypes.byref(my),
                            ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)),
           "ccm_matvec")
    y._written()
    return y


def matvec(a: PackedMatrix, x: PackedMatrix, capacity: int | None = None, stream=None):
    if capacity is None:
        capacity = words_for(a.rows, 1, bound_matvec(a, x))
    return matvec_into(a, x, PackedMatrix(a.rows, 1, capacity, a.device), stream=stream)


def matvec2_into(a: PackedMatrix, x: PackedMatrix, b: PackedMatrix, z: PackedMatrix,
                 y: PackedMatrix, ws: torch.Tensor | None = None, stream=None) -> PackedMatrix:
    """y = A x + B z, both products summed before y is packed once."""
    if ws is None:
        ws = workspace(OP_MATVEC, a.rows, max(a.cols, b.cols), 1, a.device)
    ma, mx, mb, mz, my = a.c(), x.c(), b.c(), z.c(), y.c()
    _check(lib().ccm_matvec2(ctypes.byref(ma), ctypes.byref(mx), ctypes.byref(mb),
                             ctypes.byref(mz), ctypes.byref(my), ctypes.c_void_p(ws.data_ptr()),
                             ws.numel(), _stream(stream)), "ccm_matvec2")
    y._written()
    return y


def matvec2(a: PackedMatrix, x: PackedMatrix, b: PackedMatrix, z: PackedMatrix,
            capacity: int | None = None, stream=None) -> PackedMatrix:
    if capacity is None:
        capacity = words_for(a.rows, 1, 64)
    return matvec2_into(a, x, b, z, PackedMatrix(a.rows, 1, capacity, a.device), stream=stream)


def matvec_chain(a: PackedMatrix, b: PackedMatrix, x: PackedMatrix, stream=None) -> PackedMatrix:
    """y = A (B x): the intermediate t = B x stays on the GPU, packed at its
    own exact width, and is the x of the second product (no host round trip)."""
    t = matvec(b, x, stream=stream)
    return matvec(a, t, stream=stream)


def matmul_into(a: PackedMatrix, b: PackedMatrix, c: PackedMatrix, path: int = MATMUL_AUTO,
                ws: torch.Tensor | None = None, stream=None) -> PackedMatrix:
    if ws is None:
        ws = workspace(OP_MATMUL, a.rows, a.cols, b.cols, a.device)
    ma, mb, mc = a.c(), b.c(), c.c()
    _check(lib().ccm_matmul(ctypes.byref(ma), ctypes.byref(mb), ctypes.byref(mc), int(path),
                            ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)),
           "ccm_matmul")
    c._written()
    return c


def matmul(a: PackedMatrix, b: PackedMatrix, path: int = MATMUL_AUTO,
           capacity: int | None = None, stream=None):
    if capacity is None:
        capacity = words_for(a.rows, b.cols, bound_matmul(a, b))
    return matmul_into(a, b, PackedMatrix(a.rows, b.cols, capacity, a.device), path, stream=stream)


def gen_uniform(count: int, seed: int, stream_id: int, lo: int, hi: int, start: int = 0,
                out: torch.Tensor | None = None, device="cuda", stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(count, dtype=torch.int64, device=device)
    _check(lib().ccm_gen_uniform(ctypes.c_void_p(out.data_ptr()), count, seed, stream_id, start,
                                 lo, hi, _stream(stream)), "ccm_gen_uniform")
    return out


def gen_poisson(count: int, seed: int, stream_id: int, table: torch.Tensor, start: int = 0,
                out: torch.Tensor | None = None, device="cuda", stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(count, dtype=torch.int64, device=device)
    table = table.to(device=out.device, dtype=torch.float64).contiguous()
    _check(lib().ccm_gen_poisson(ctypes.c_void_p(out.data_ptr()), count, seed, stream_id, start,
                                 ctypes.c_void_p(table.data_ptr()), table.numel(),
                                 _stream(stream)), "ccm_gen_poisson")
    return out


# ---------------------------------------------------------------------------
# VLB (Method 2): header + words + offset index, in one int32 buffer + index.
# ---------------------------------------------------------------------------
class VlbMatrix:
    def __init__(self, rows: int, cols: int, capacity: int, device=None):
        self.rows, self.cols, self.capacity = int(rows), int(cols), int(capacity)
        dev = torch.device(device) if device is not None else torch.device("cuda")
        self.buf = torch.empty(HEADER_WORDS + self.capacity, dtype=torch.int32, device=dev)
        n_index = int(lib().ccm_vlb_index_entries(self.rows, self.cols))
        self.index = torch.empty(n_index, dtype=torch.int64, device=dev)

    @property
    def device(self):
        return self.buf.device

    def header(self, stream=None) -> Header:
        h = Header()
        _check(lib().ccm_header_read(ctypes.c_void_p(self.buf.data_ptr()), ctypes.byref(h),
                                     _stream(stream)), "ccm_header_read")
        return h

    def words(self) -> torch.Tensor:
        return self.buf[HEADER_WORDS:HEADER_WORDS + int(self.header().nwords)]


def vlb_measure(t: torch.Tensor, stream=None) -> Header:
    """k, total bits and word count of the VLB stream of a dense matrix
    (synchronous), without writing it."""
    t, rows, cols, dt = _as_dense(t)
    hdr = torch.empty(HEADER_WORDS, dtype=torch.int32, device=t.device)
    ws = torch.empty(max(workspace_bytes(OP_VLB, rows, cols, 0), 256), dtype=torch.uint8,
                     device=t.device)
    _check(lib().ccm_vlb_pack(ctypes.c_void_p(t.data_ptr()), dt, rows, cols,
                              ctypes.c_void_p(hdr.data_ptr()), None, 0, None,
                              ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)),
           "ccm_vlb_pack")
    h = Header()
    _check(lib().ccm_header_read(ctypes.c_void_p(hdr.data_ptr()), ctypes.byref(h),
                                 _stream(stream)), "ccm_header_read")
    return h


def vlb_pack(t: torch.Tensor, capacity: int | None = None, stream=None) -> VlbMatrix:
    t, rows, cols, dt = _as_dense(t)
    if capacity is None:
        h = vlb_measure(t, stream)
        _check(h.status, "ccm_vlb_pack")
        capacity = int(h.nwords)
    out = VlbMatrix(rows, cols, capacity, t.device)
    ws = torch.empty(max(workspace_bytes(OP_VLB, rows, cols, 0), 256), dtype=torch.uint8,
                     device=t.device)
    _check(lib().ccm_vlb_pack(ctypes.c_void_p(t.data_ptr()), dt, rows, cols,
                              ctypes.c_void_p(out.buf.data_ptr()),
                              ctypes.c_void_p(out.buf.data_ptr() + 4 * HEADER_WORDS), capacity,
                              ctypes.c_void_p(out.index.data_ptr()),
                              ctypes.c_void_p(ws.data_ptr()), ws.numel(), _stream(stream)),
           "ccm_vlb_pack")
    return out


def vlb_unpack(v: VlbMatrix, dtype=torch.int64, stream=None, check: bool = True) -> torch.Tensor:
    out = torch.empty((v.rows, v.cols), dtype=dtype, device=v.device)
    err = torch.empty(1, dtype=torch.int32, device=v.device)
    _check(lib().ccm_vlb_unpack(ctypes.c_void_p(v.buf.data_ptr()),
                                ctypes.c_void_p(v.buf.data_ptr() + 4 * HEADER_WORDS), v.capacity,
                                ctypes.c_void_p(v.index.data_ptr()), v.rows, v.cols,
                                ctypes.c_void_p(out.data_ptr()), I64 if dtype == torch.int64 else I32,
                                ctypes.c_void_p(err.data_ptr()), _stream(stream)), "ccm_vlb_unpack")
    if check and v.rows * v.cols:
        _check(int(err.item()), "ccm_vlb_unpack")
    return out


def vlb_matvec_into(v: VlbMatrix, x: PackedMatrix, y: PackedMatrix,
                    ws: torch.Tensor | None = None, stream=None) -> PackedMatrix:
    """y = A x with A in VLB form (decoded entry by entry as it is used)."""
    if ws is None:
        ws = workspace(OP_VLB_MATVEC, v.rows, v.cols, 0, v.device)
    mx, my = x.c(), y.c()
    _check(lib().ccm_vlb_matvec(ctypes.c_void_p(v.buf.data_ptr()),
                                ctypes.c_void_p(v.buf.data_ptr() + 4 * HEADER_WORDS), v.capacity,
                                ctypes.c_void_p(v.index.data_ptr()), v.rows, v.cols,
                                ctypes.byref(mx), ctypes.byref(my), ctypes.c_void_p(ws.data_ptr()),
                                ws.numel(), _stream(stream)), "ccm_vlb_matvec")
    y._written()
    return y


def vlb_matvec(v: VlbMatrix, x: PackedMatrix, capacity: int | None = None,
               stream=None) -> PackedMatrix:
    if capacity is None:
        capacity = words_for(v.rows, 1, 64)
    y = PackedMatrix(v.rows, 1, capacity, v.device)
    return vlb_matvec_into(v, x, y, stream=stream)


def choose(t: torch.Tensor, stream=None) -> dict:
    """SM or VLB for this matrix: the bits each encoding needs (SM: n*b,
    Eq. 15; VLB: sum of k + L_i, Eq. 16), measured on the GPU."""
    t2, rows, cols, _ = _as_dense(t)
    b, _ = measure(t2, stream)
    v = vlb_measure(t2, stream)
    sm_bits = rows * cols * b
    vlb_bits = int(v.stat_or) if v.status == OK else None
    best = "sm" if vlb_bits is None or sm_bits <= vlb_bits else "vlb"
    return {"sm_bits": sm_bits, "vlb_bits": vlb_bits, "choice": best, "sm_width": b,
            "vlb_prefix": int(v.width) if v.status == OK else None}
