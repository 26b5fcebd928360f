// ew_kernels.cuh -- elementwise kernels on the group engine: SM pack of dense
// int32/int64 data, unpack, and the add / scale operations whose results are
// re-packed at their own width.  Each is instantiated per width class
// (ew8.cu, ew16.cu, ew32.cu); the host picks the class from the widths the
// buffer capacities allow.
//
// A result is packed in two launches: a statistics pass (OR of the folded
// values and the any-negative flag, merged into the output header: the width
// rule of Eq. 1 with the two's complement reading) and a pack pass that reads
// the width back from the header and writes the fields.  Operations on
// packed inputs recompute their values in the pack pass instead of keeping
// them: re-reading b-bit inputs costs less than writing and reading int64.
#pragma once

#include "group_engine.cuh"
#include "pack_engine.cuh"

namespace ccm {
namespace ge {

struct PackedIn {
  const ccm_header* h;
  const uint32_t* __restrict__ w;
  int b, sgn;
  uint64_t dw;
  __device__ __forceinline__ void init(uint64_t n) {
    b = h->width;
    sgn = h->is_signed;
    dw = data_words(n, b);
  }
};

template <typename T>
struct OpDense {
  const T* __restrict__ p;
  __device__ __forceinline__ void init(uint64_t) {}
  template <int BMAX>
  __device__ __forceinline__ void produce(uint32_t* buf, uint64_t tile, uint32_t nt, int lane,
                                          int64_t (&v)[32], int&) const {
    T* tb = reinterpret_cast<T*>(buf);
    stage_dense<T>(tb, p, tile * kTile, nt, lane);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 32; ++k) v[k] = (int64_t)tb[33 * lane + k];
    __syncwarp();
  }
};

struct OpAdd {
  PackedIn a, b;
  __device__ __forceinline__ void init(uint64_t n) {
    a.init(n);
    b.init(n);
  }
  template <int BMAX>
  __device__ __forceinline__ void produce(uint32_t* buf, uint64_t tile, uint32_t, int lane,
                                          int64_t (&v)[32], int& ovf) const {
    stage_packed(buf, a.w, tile, a.b, a.dw, lane);
    __syncwarp();
    decode_dispatch<BMAX>(a.b, a.sgn, buf, lane, [&](int k, int64_t x) { v[k] = x; });
    __syncwarp();
    stage_packed(buf, b.w, tile, b.b, b.dw, lane);
    __syncwarp();
    decode_dispatch<BMAX>(b.b, b.sgn, buf, lane,
                          [&](int k, int64_t x) { v[k] = add_checked(v[k], x, ovf); });
    __syncwarp();
  }
};

struct OpScale {
  PackedIn a;
  int64_t s;
  __device__ __forceinline__ void init(uint64_t n) { a.init(n); }
  template <int BMAX>
  __device__ __forceinline__ void produce(uint32_t* buf, uint64_t tile, uint32_t, int lane,
                                          int64_t (&v)[32], int& ovf) const {
    stage_packed(buf, a.w, tile, a.b, a.dw, lane);
    __syncwarp();
    const int64_t sc = s;
    decode_dispatch<BMAX>(a.b, a.sgn, buf, lane,
                          [&](int k, int64_t x) { v[k] = mul_checked(x, sc, ovf); });
    __syncwarp();
  }
};

// Statistics (PACK = false) or pack (PACK = true) pass of an operation.
template <class Op, int BMAX, bool PACK>
__global__ void __launch_bounds__(kThreads) k_ew(Op op, ccm_header* out, uint32_t* words,
                                                 uint64_t capacity, uint64_t n) {
  __shared__ __align__(16) uint32_t s_buf[kWarps][kBufWords];
  int b = 0, sgn = 0;
  if constexpr (PACK) {
    if (!resolve_output(out, words, capacity, n, b, sgn)) return;
  } else {
    if (out->status != CCM_OK) return;
  }
  op.init(n);
  const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  uint32_t* buf = s_buf[warp];
  const uint64_t dw = PACK ? data_words(n, b) : 0;
  const uint32_t mask = b >= 32 ? 0xffffffffu : ((1u << b) - 1u);
  const uint64_t ntiles = (n + kTile - 1) / kTile;
  const uint64_t gwarps = (uint64_t)gridDim.x * kWarps;
  uint64_t orv = 0;
  uint32_t neg = 0;
  int ovf = 0;
  for (uint64_t tile = (uint64_t)blockIdx.x * kWarps + warp; tile < ntiles; tile += gwarps) {
    const uint32_t nt = (uint32_t)umin((uint64_t)kTile, n - tile * kTile);
    int64_t v[32];
    op.template produce<BMAX>(buf, tile, nt, lane, v, ovf);
    if ((uint32_t)(32 * lane + 32) > nt) {
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if ((uint32_t)(32 * lane + k) >= nt) v[k] = 0;
    }
    if constexpr (!PACK) {
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        orv |= fold(v[k]);
        neg |= (uint32_t)(v[k] < 0);
      }
    } else {
      uint32_t u[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) u[k] = (uint32_t)v[k] & mask;
      encode_dispatch<BMAX>(b, u, buf, lane);
      __syncwarp();
      store_packed(buf, words, tile, b, dw, lane);
      __syncwarp();
    }
  }
  if constexpr (!PACK) {
    orv = warp_or64(orv);
    neg = __reduce_or_sync(0xffffffffu, neg);
    ovf = (int)__reduce_or_sync(0xffffffffu, (uint32_t)ovf);
    if (lane == 0) {
      if (orv) atomicOr(reinterpret_cast<unsigned long long*>(&out->stat_or), (unsigned long long)orv);
      if (neg) atomicOr(&out->stat_neg, 1u);
      if (ovf) set_status(out, CCM_E_OVERFLOW);
    }
  }
}

// Unpack: decode every group and write the values densely (int64 or int32).
template <typename T, int BMAX>
__global__ void __launch_bounds__(kThreads) k_unpack_ge(const ccm_header* h,
                                                        const uint32_t* __restrict__ w,
                                                        uint64_t rows, uint64_t cols,
                                                        uint64_t capacity, T* __restrict__ out,
                                                        int32_t* err) {
  __shared__ __align__(16) uint32_t s_buf[kWarps][kBufWords];
  int st = check_input(h, rows, cols, capacity);
  const int b = h->width, sgn = h->is_signed;
  if (st == CCM_OK && sizeof(T) == 4 && (sgn ? b > 32 : b > 31)) st = CCM_E_WIDTH;
  if (err && blockIdx.x == 0 && threadIdx.x == 0) *err = st;
  if (st != CCM_OK) return;
  const uint64_t n = rows * cols;
  const uint64_t dw = data_words(n, b);
  const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  uint32_t* buf = s_buf[warp];
  T* tb = reinterpret_cast<T*>(buf);
  const uint64_t ntiles = (n + kTile - 1) / kTile;
  const uint64_t gwarps = (uint64_t)gridDim.x * kWarps;
  for (uint64_t tile = (uint64_t)blockIdx.x * kWarps + warp; tile < ntiles; tile += gwarps) {
    const uint32_t nt = (uint32_t)umin((uint64_t)kTile, n - tile * kTile);
    stage_packed(buf, w, tile, b, dw, lane);
    __syncwarp();
    int64_t v[32];
    decode_dispatch<BMAX>(b, sgn, buf, lane, [&](int k, int64_t x) { v[k] = x; });
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 32; ++k) tb[33 * lane + k] = (T)v[k];
    __syncwarp();
    store_dense<T>(tb, out, tile * kTile, nt, lane);
    __syncwarp();
  }
}

// What the host asks one class to run.
enum class EwKind { PackI64, PackI32, AddStats, AddPack, ScaleStats, ScalePack, UnpackI64, UnpackI32 };

struct EwCall {
  EwKind kind;
  const void* dense;      // PackI64 / PackI32 source, Unpack destination
  const ccm_header* ha;   // packed inputs
  const uint32_t* wa;
  const ccm_header* hb;
  const uint32_t* wb;
  int64_t s;              // scale factor
  ccm_header* out;        // output header (pack/stats) or input header (unpack)
  uint32_t* words;        // output words, or input words (unpack)
  uint64_t capacity;
  uint64_t rows, cols;
  int32_t* err;           // unpack status
};

inline int ew_grid(uint64_t n) {
  uint64_t tiles = (n + kTile - 1) / kTile;
  uint64_t want = (tiles + kWarps - 1) / kWarps;
  return (int)umin(umax(want, 1), (uint64_t)num_sms() * 12);
}

template <int C>
void launch_ew_class(const EwCall& c, cudaStream_t st) {
  const uint64_t n = c.rows * c.cols;
  const int g = ew_grid(n);
  PackedIn a{c.ha, c.wa, 0, 0, 0}, b{c.hb, c.wb, 0, 0, 0};
  switch (c.kind) {
    case EwKind::PackI64:
      k_ew<OpDense<int64_t>, C, true><<<g, kThreads, 0, st>>>(
          OpDense<int64_t>{(const int64_t*)c.dense}, c.out, c.words, c.capacity, n);
      break;
    case EwKind::PackI32:
      k_ew<OpDense<int32_t>, C, true><<<g, kThreads, 0, st>>>(
          OpDense<int32_t>{(const int32_t*)c.dense}, c.out, c.words, c.capacity, n);
      break;
    case EwKind::AddStats:
      k_ew<OpAdd, C, false><<<g, kThreads, 0, st>>>(OpAdd{a, b}, c.out, nullptr, 0, n);
      break;
    case EwKind::AddPack:
      k_ew<OpAdd, C, true><<<g, kThreads, 0, st>>>(OpAdd{a, b}, c.out, c.words, c.capacity, n);
      break;
    case EwKind::ScaleStats:
      k_ew<OpScale, C, false><<<g, kThreads, 0, st>>>(OpScale{a, c.s}, c.out, nullptr, 0, n);
      break;
    case EwKind::ScalePack:
      k_ew<OpScale, C, true><<<g, kThreads, 0, st>>>(OpScale{a, c.s}, c.out, c.words, c.capacity, n);
      break;
    case EwKind::UnpackI64:
      k_unpack_ge<int64_t, C><<<g, kThreads, 0, st>>>(c.out, c.words, c.rows, c.cols, c.capacity,
                                                      (int64_t*)c.dense, c.err);
      break;
    case EwKind::UnpackI32:
      k_unpack_ge<int32_t, C><<<g, kThreads, 0, st>>>(c.out, c.words, c.rows, c.cols, c.capacity,
                                                      (int32_t*)c.dense, c.err);
      break;
  }
}

}  // namespace ge
}  // namespace ccm
