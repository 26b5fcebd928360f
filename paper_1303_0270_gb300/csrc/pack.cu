// pack.cu -- SM compression and decompression kernels (Methods, Method 1):
// width selection + pack of dense int32/int64 matrices, unpack, element
// access, and the elementwise operations whose results are re-packed by the
// same engine (add, scale).
#include "ew_kernels.cuh"
#include "async_copy.cuh"
#include "cta_pack.cuh"
#include "kernels.h"
#include "pack_engine.cuh"

namespace ccm {

int width_bound(uint64_t capacity, uint64_t n) {
  if (n == 0) return 64;
  return (int)umin(capacity * 32 / n, 64);
}

int bitlen_host(uint64_t v) {
  int l = 0;
  for (; v; v >>= 1) ++l;
  return l;
}

namespace {

// Width class of the group-engine kernels for a width bound (0: none, use
// the run-time-width kernels).
int ew_class(int bmax) { return bmax <= 8 ? 8 : bmax <= 16 ? 16 : bmax <= 32 ? 32 : 0; }

void launch_ew(int cls, const ge::EwCall& c, cudaStream_t st) {
  int launched;
  switch (cls) {
    case 8: launched = ge::launch_ew_class<8>(c, st); break;
    case 16: launched = ge::launch_ew_class<16>(c, st); break;
    default: launched = ge::launch_ew_class<32>(c, st); break;
  }
  note_launch(launched);
}

}  // namespace

int num_sms() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  static int cached_dev = -1, cached = 0;
  if (dev != cached_dev) {
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cached = sms > 0 ? sms : 1;
    cached_dev = dev;
  }
  return cached;
}

int max_smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  static int cached_dev = -1, cached = 0;
  if (dev != cached_dev) {
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cached = v > 0 ? v : 48 * 1024;
    cached_dev = dev;
  }
  return cached;
}

__global__ void k_init(InitArgs a) {
  ax::grid_dep_launch();  // a programmatically launched successor may start now
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int st = CCM_OK;
    if (a.in0) st = check_input(a.in0, a.in0_rows, a.in0_cols, a.in0_capacity);
    if (st == CCM_OK && a.in1) st = check_input(a.in1, a.in1_rows, a.in1_cols, a.in1_capacity);
    ccm_header* o = a.out;
    o->magic = CCM_MAGIC;
    o->width = 0;
    o->is_signed = 0;
    o->status = st;
    o->rows = a.out_rows;
    o->cols = a.out_cols;
    o->nwords = 0;
    o->stat_or = 0;
    o->stat_neg = 0;
    o->reserved0 = 0;
    o->reserved1 = 0;
  }
  if (a.zero_ptr) {
    uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.zero_count; i += stride)
      a.zero_ptr[i] = 0;
  }
}

// Validates one more pair of inputs against an already initialised output:
// the first invalid header's status goes to the output header.
__global__ void k_check(InitArgs a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    int st = CCM_OK;
    if (a.in0) st = check_input(a.in0, a.in0_rows, a.in0_cols, a.in0_capacity);
    if (st == CCM_OK && a.in1) st = check_input(a.in1, a.in1_rows, a.in1_cols, a.in1_capacity);
    if (st != CCM_OK) set_status(a.out, st);
  }
}

void launch_check(const ccm_matrix& p, const ccm_matrix& q, ccm_header* out, cudaStream_t st) {
  InitArgs ia{};
  ia.out = out;
  ia.in0 = p.hdr;
  ia.in0_rows = p.rows;
  ia.in0_cols = p.cols;
  ia.in0_capacity = p.capacity;
  ia.in1 = q.hdr;
  ia.in1_rows = q.rows;
  ia.in1_cols = q.cols;
  ia.in1_capacity = q.capacity;
  k_check<<<1, 32, 0, st>>>(ia);
  note_launch();
}

void launch_init(const InitArgs& a, cudaStream_t st) {
  int grid = 1;
  if (a.zero_ptr && a.zero_count > 256)
    grid = (int)umin((a.zero_count + 255) / 256, (uint64_t)num_sms() * 4);
  k_init<<<grid, 256, 0, st>>>(a);
  note_launch();
}

// ---------------------------------------------------------------------------
// pack / measure
// ---------------------------------------------------------------------------
// Finalises the header of a measure-only call (no words): width, sign, nwords.
__global__ void k_measure_finish(ccm_header* out, uint64_t n) {
  if (out->status != CCM_OK) return;
  int b = width_from_stats(out->stat_or, out->stat_neg);
  out->width = b;
  out->is_signed = out->stat_neg ? 1 : 0;
  out->nwords = words_for(n, b);
}

void run_measure(const void* dense, int dtype, uint64_t rows, uint64_t cols, ccm_header* hdr,
                 cudaStream_t st) {
  InitArgs ia{};
  ia.out = hdr;
  ia.out_rows = rows;
  ia.out_cols = cols;
  launch_init(ia, st);
  uint64_t n = rows * cols;
  if (n) {
    profile_begin(st);
    if (dtype == CCM_I64)
      launch_stats(ProdDenseI64{(const int64_t*)dense}, hdr, n, st);
    else
      launch_stats(ProdDenseI32{(const int32_t*)dense}, hdr, n, st);
    profile_end(st);
  }
  k_measure_finish<<<1, 1, 0, st>>>(hdr, n);
  note_launch();
}

size_t pack_workspace(uint64_t rows, uint64_t cols, uint64_t capacity) {
  const uint64_t n = rows * cols;
  const int cls = ew_class(width_bound(capacity, n));
  return (cls && n) ? ge::pack_ws_bytes(n, cls) : 0;
}

// A small dense input (n <= kSmallPack entries) packed in one launch by
// vec_pack_ctas(n) CTAs (cta_pack.cuh): each reads all the entries for the
// width statistics (Eq. 1) and packs its own 16 groups of 32 fields; CTA 0
// writes the whole header.  The general path's three launches (header,
// statistics, pack) cost more than the work here.
constexpr uint64_t kSmallPack = 16384;

template <typename T>
__global__ void __launch_bounds__(kVecThreads) k_pack_small(const T* __restrict__ src,
                                                            uint64_t rows, uint64_t cols,
                                                            ccm_header* out, uint32_t* words,
                                                            uint64_t capacity) {
  __shared__ VecPackSmem sm;
  const uint32_t mm = (uint32_t)(rows * cols);  // 1 .. kSmallPack
  const uint32_t g0 = blockIdx.x * kVecGroupsPerCta;
  uint64_t orv;
  uint32_t neg;
  vec_stats_stage([&](uint32_t i) { return (int64_t)src[i]; }, mm, g0, sm, orv, neg);
  const int b = width_from_stats(orv, neg);
  const uint64_t nw = words_for(mm, b), dw = data_words(mm, b);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out->magic = CCM_MAGIC;
    out->width = b;
    out->is_signed = neg ? 1 : 0;
    out->status = nw > capacity ? CCM_E_CAPACITY : CCM_OK;
    out->rows = rows;
    out->cols = cols;
    out->nwords = nw;
    out->stat_or = orv;
    out->stat_neg = neg;
    out->reserved0 = 0;
    out->reserved1 = 0;
  }
  if (nw > capacity) return;
  vec_pack_groups(sm, mm, g0, b, words, dw, nw);
}

void run_pack(const void* dense, int dtype, uint64_t rows, uint64_t cols, const ccm_matrix& out,
              void* ws, size_t ws_bytes, cudaStream_t st) {
  uint64_t n = rows * cols;
  if (n && n <= kSmallPack) {
    const uint32_t g = vec_pack_ctas(n);
    profile_begin(st);
    if (dtype == CCM_I64)
      k_pack_small<int64_t><<<g, kVecThreads, 0, st>>>((const int64_t*)dense, rows, cols,
                                                      out.hdr, out.words, out.capacity);
    else
      k_pack_small<int32_t><<<g, kVecThreads, 0, st>>>((const int32_t*)dense, rows, cols,
                                                      out.hdr, out.words, out.capacity);
    profile_end(st);
    note_launch();
    return;
  }
  InitArgs ia{};
  ia.out = out.hdr;
  ia.out_rows = rows;
  ia.out_cols = cols;
  launch_init(ia, st);
  const int cls = ew_class(width_bound(out.capacity, n));
  // (the single pass stages the dense tiles with 16-byte copies: it needs a
  // 16-byte aligned input; an input aligned only to its element size takes
  // the two-pass path below, which reads it element by element)
  const bool aligned16 = reinterpret_cast<uintptr_t>(dense) % 16 == 0;
  if (cls && n && ws && ws_bytes >= ge::pack_ws_bytes(n, cls) && aligned16) {
    // single pass over the dense input: local-width tiles, then re-code
    ge::EwCall c{};
    c.kind = dtype == CCM_I64 ? ge::EwKind::LocalI64 : ge::EwKind::LocalI32;
    c.dense = dense;
    c.out = out.hdr;
    c.words = out.words;
    c.capacity = out.capacity;
    c.rows = rows;
    c.cols = cols;
    c.ws = ws;
    c.slot_class = cls;
    // the widest width the output's capacity holds: the speculative width
    c.spec = width_bound(out.capacity, n);
    if (c.spec > cls) c.spec = 0;
    // (starts while the header is initialised, unless this call is timed)
    c.pdl = profile_armed() ? 0 : 1;
    profile_begin(st);
    launch_ew(cls, c, st);
    profile_end(st);
    c.kind = ge::EwKind::Repack;
    launch_ew(cls, c, st);
    return;
  }
  if (cls && n) {
    if (dtype == CCM_I64)
      launch_stats(ProdDenseI64{(const int64_t*)dense}, out.hdr, n, st);
    else
      launch_stats(ProdDenseI32{(const int32_t*)dense}, out.hdr, n, st);
    ge::EwCall c{};
    c.kind = dtype == CCM_I64 ? ge::EwKind::PackI64 : ge::EwKind::PackI32;
    c.dense = dense;
    c.out = out.hdr;
    c.words = out.words;
    c.capacity = out.capacity;
    c.rows = rows;
    c.cols = cols;
    profile_begin(st);
    launch_ew(cls, c, st);
    profile_end(st);
  } else if (dtype == CCM_I64) {
    ProdDenseI64 p{(const int64_t*)dense};
    if (n) launch_stats(p, out.hdr, n, st);
    profile_begin(st);
    launch_pack(p, out.hdr, out.words, out.capacity, n, st);
    profile_end(st);
  } else {
    ProdDenseI32 p{(const int32_t*)dense};
    if (n) launch_stats(p, out.hdr, n, st);
    profile_begin(st);
    launch_pack(p, out.hdr, out.words, out.capacity, n, st);
    profile_end(st);
  }
}

// ---------------------------------------------------------------------------
// unpack: every field, sign/zero extended, to int64 or int32.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) k_unpack(const ccm_header* h, const uint32_t* __restrict__ w,
                                                uint64_t rows, uint64_t cols, uint64_t capacity,
                                                T* __restrict__ out, int32_t* err) {
  int st = check_input(h, rows, cols, capacity);
  const int b = h->width, sgn = h->is_signed;
  if (st == CCM_OK && sizeof(T) == 4 && (sgn ? b > 32 : b > 31)) st = CCM_E_WIDTH;
  if (st != CCM_OK) {
    if (err && blockIdx.x == 0 && threadIdx.x == 0) *err = st;
    return;
  }
  if (err && blockIdx.x == 0 && threadIdx.x == 0) *err = CCM_OK;
  const uint64_t n = rows * cols;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = (T)decode_field(w, i, b, sgn);
}

void run_unpack(const ccm_matrix& a, void* dense, int dtype, int32_t* err, cudaStream_t st) {
  uint64_t n = a.rows * a.cols;
  const int cls = ew_class(width_bound(a.capacity, n));
  if (cls && n) {
    ge::EwCall c{};
    c.kind = dtype == CCM_I64 ? ge::EwKind::UnpackI64 : ge::EwKind::UnpackI32;
    c.dense = dense;
    c.out = a.hdr;
    c.words = a.words;
    c.capacity = a.capacity;
    c.rows = a.rows;
    c.cols = a.cols;
    c.err = err;
    profile_begin(st);
    launch_ew(cls, c, st);
    profile_end(st);
    return;
  }
  int grid = (int)umin(umax((n + 255) / 256, 1), (uint64_t)num_sms() * 16);
  profile_begin(st);
  if (dtype == CCM_I64)
    k_unpack<int64_t><<<grid, 256, 0, st>>>(a.hdr, a.words, a.rows, a.cols, a.capacity,
                                            (int64_t*)dense, err);
  else
    k_unpack<int32_t><<<grid, 256, 0, st>>>(a.hdr, a.words, a.rows, a.cols, a.capacity,
                                            (int32_t*)dense, err);
  profile_end(st);
  note_launch();
}

// ---------------------------------------------------------------------------
// get: element access by flat row-major index.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_get(const ccm_header* h, const uint32_t* __restrict__ w,
                                             uint64_t rows, uint64_t cols, uint64_t capacity,
                                             const uint64_t* __restrict__ idx, uint64_t count,
                                             int64_t* __restrict__ out, int32_t* err) {
  int st = check_input(h, rows, cols, capacity);
  if (err && blockIdx.x == 0 && threadIdx.x == 0 && st != CCM_OK) *err = st;
  if (st != CCM_OK) return;
  const int b = h->width, sgn = h->is_signed;
  const uint64_t n = rows * cols;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  int bad = 0;
  for (uint64_t k = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count; k += stride) {
    uint64_t e = idx[k];
    if (e < n) {
      out[k] = decode_field(w, e, b, sgn);
    } else {
      out[k] = 0;
      bad = 1;
    }
  }
  if (err && bad) atomicCAS(err, CCM_OK, CCM_E_RANGE);
}

__global__ void k_set_i32(int32_t* p, int32_t v) { *p = v; }

void run_get(const ccm_matrix& a, const uint64_t* idx, uint64_t count, int64_t* out, int32_t* err,
             cudaStream_t st) {
  if (err) {
    k_set_i32<<<1, 1, 0, st>>>(err, CCM_OK);
    note_launch();
  }
  if (!count) return;
  int grid = (int)umin((count + 255) / 256, (uint64_t)num_sms() * 8);
  profile_begin(st);
  k_get<<<grid, 256, 0, st>>>(a.hdr, a.words, a.rows, a.cols, a.capacity, idx, count, out,
                              err);
  profile_end(st);
  note_launch();
}

// ---------------------------------------------------------------------------
// add / scale
// ---------------------------------------------------------------------------
void run_add(const ccm_matrix& a, const ccm_matrix& b, const ccm_matrix& c, void* /*ws*/,
             size_t /*ws_bytes*/, cudaStream_t st) {
  InitArgs ia{};
  ia.out = c.hdr;
  ia.in0 = a.hdr;
  ia.in1 = b.hdr;
  ia.in0_rows = a.rows;
  ia.in0_cols = a.cols;
  ia.in0_capacity = a.capacity;
  ia.in1_rows = b.rows;
  ia.in1_cols = b.cols;
  ia.in1_capacity = b.capacity;
  ia.out_rows = c.rows;
  ia.out_cols = c.cols;
  launch_init(ia, st);
  uint64_t n = c.rows * c.cols;
  const int cls = ew_class(max(max(width_bound(a.capacity, n), width_bound(b.capacity, n)),
                               width_bound(c.capacity, n)));
  if (cls && n) {
    ge::EwCall e{};
    e.ha = a.hdr;
    e.wa = a.words;
    e.hb = b.hdr;
    e.wb = b.words;
    e.out = c.hdr;
    e.words = c.words;
    e.capacity = c.capacity;
    e.rows = c.rows;
    e.cols = c.cols;
    // one pass at the width the input ranges give, then the finish (a second
    // pass only when the exact width is smaller)
    e.kind = ge::EwKind::AddSpec;
    profile_begin(st);
    launch_ew(cls, e, st);
    e.kind = ge::EwKind::AddPack;
    e.spec = 1;
    launch_ew(cls, e, st);
    profile_end(st);
    return;
  }
  // No width class holds the output bound.  With inputs of at most 32 bits
  // the lane pass may still write the sum (up to 33 bits) first; the
  // run-time passes then return at once.
  ProdAdd p{{a.hdr, a.words, 0, 0}, {b.hdr, b.words, 0, 0}};
  const int in_bound = max(width_bound(a.capacity, n), width_bound(b.capacity, n));
  const int lanes = n && in_bound <= 32;
  profile_begin(st);
  if (lanes) {
    const ge::OpAdd op{ge::PackedIn{a.hdr, a.words, 0, 0, 0}, ge::PackedIn{b.hdr, b.words, 0, 0, 0}};
    ge::launch_lanes_add(op, c.hdr, c.words, c.capacity, n, in_bound, st);
    note_launch();
  }
  if (n) launch_stats(p, c.hdr, n, st, lanes);
  launch_pack(p, c.hdr, c.words, c.capacity, n, st, lanes);
  profile_end(st);
}

void run_scale(const ccm_matrix& a, int64_t s, const ccm_matrix& c, void* /*ws*/,
               size_t /*ws_bytes*/, cudaStream_t st) {
  InitArgs ia{};
  ia.out = c.hdr;
  ia.in0 = a.hdr;
  ia.in0_rows = a.rows;
  ia.in0_cols = a.cols;
  ia.in0_capacity = a.capacity;
  ia.out_rows = c.rows;
  ia.out_cols = c.cols;
  launch_init(ia, st);
  uint64_t n = c.rows * c.cols;
  const int cls = ew_class(max(width_bound(a.capacity, n), width_bound(c.capacity, n)));
  if (cls && n) {
    ge::EwCall e{};
    e.ha = a.hdr;
    e.wa = a.words;
    e.s = s;
    e.out = c.hdr;
    e.words = c.words;
    e.capacity = c.capacity;
    e.rows = c.rows;
    e.cols = c.cols;
    e.kind = ge::EwKind::ScaleSpec;
    profile_begin(st);
    launch_ew(cls, e, st);
    e.kind = ge::EwKind::ScalePack;
    e.spec = 1;
    launch_ew(cls, e, st);
    profile_end(st);
    return;
  }
  // No width class holds the output bound: the lane pass may still write
  // s A (up to 36 bits) first for 1 <= |s| < 2^5; the run-time passes then
  // return at once.
  ProdScale p{{a.hdr, a.words, 0, 0}, s};
  const int in_bound = width_bound(a.capacity, n);
  const int lanes = n && in_bound <= 32 && s != 0 && s > -32 && s < 32;
  profile_begin(st);
  if (lanes) {
    const ge::OpScale<true> op{ge::PackedIn{a.hdr, a.words, 0, 0, 0}, s};
    ge::launch_lanes_scale(op, c.hdr, c.words, c.capacity, n, in_bound, st);
    note_launch();
  }
  if (n) launch_stats(p, c.hdr, n, st, lanes);
  launch_pack(p, c.hdr, c.words, c.capacity, n, st, lanes);
  profile_end(st);
}

void run_pack_scratch32(const int32_t* vals, const ccm_matrix& out, cudaStream_t st) {
  const uint64_t n = out.rows * out.cols;
  const int cls = ew_class(width_bound(out.capacity, n));
  if (cls && n && reinterpret_cast<uintptr_t>(vals) % 16 == 0) {
    // the producer merged the statistics: one pass at the exact width (the
    // staged single-pass kernel, spec < 0), then the header
    ge::EwCall c{};
    c.kind = ge::EwKind::LocalI32;
    c.dense = vals;
    c.out = out.hdr;
    c.words = out.words;
    c.capacity = out.capacity;
    c.rows = out.rows;
    c.cols = out.cols;
    c.slot_class = cls;
    c.spec = -1;
    launch_ew(cls, c, st);
    c.kind = ge::EwKind::Repack;
    launch_ew(cls, c, st);
    return;
  }
  launch_pack(ProdDenseI32{vals}, out.hdr, out.words, out.capacity, n, st);
}

// Pack an int64 result held in device scratch (matvec / matmul epilogue).
void run_pack_scratch(const int64_t* vals, const ccm_matrix& out, cudaStream_t st,
                      bool stats_done) {
  ProdDenseI64 p{vals};
  uint64_t n = out.rows * out.cols;
  const int cls = ew_class(width_bound(out.capacity, n));
  if (cls && n) {
    if (!stats_done) launch_stats(p, out.hdr, n, st);
    ge::EwCall c{};
    c.kind = ge::EwKind::PackI64;
    c.dense = vals;
    c.out = out.hdr;
    c.words = out.words;
    c.capacity = out.capacity;
    c.rows = out.rows;
    c.cols = out.cols;
    launch_ew(cls, c, st);
    return;
  }
  if (n && !stats_done) launch_stats(p, out.hdr, n, st);
  launch_pack(p, out.hdr, out.words, out.capacity, n, st);
}

}  // namespace ccm
