// ccm_device.cuh -- device-side building blocks shared by the libccm kernels.
//
// Bit stream (Methods, Method 1; Eq. 3): field e of a matrix packed at width
// b occupies bits [e*b, (e+1)*b) of an LSB-first stream of 32-bit words.  A
// run of 32 consecutive fields therefore spans exactly b whole words and
// always starts on a word boundary -- the "group" every kernel tiles by.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "ccm.h"

namespace ccm {

constexpr int kWarp = 32;
constexpr int kTileFields = 1024;  // one warp tile = 32 groups of 32 fields

// Largest field count of one matrix: every bit offset n*64 then fits uint64.
constexpr uint64_t kMaxFields = 1ull << 57;

__host__ __device__ __forceinline__ uint64_t umin(uint64_t a, uint64_t b) { return a < b ? a : b; }

// rows*cols neither wraps nor exceeds kMaxFields.
__host__ __device__ __forceinline__ bool shape_ok(uint64_t rows, uint64_t cols) {
  return rows == 0 || cols == 0 || rows <= kMaxFields / cols;
}
__host__ __device__ __forceinline__ uint64_t umax(uint64_t a, uint64_t b) { return a > b ? a : b; }

struct Stats {
  uint64_t orv;  // OR of folded values
  uint32_t neg;  // any value < 0
};

__device__ __forceinline__ int bitlen64(uint64_t v) { return v ? 64 - __clzll((long long)v) : 0; }

// The width rule: Eq. 1 on non-negative data, its two's complement reading
// otherwise.  `orv` is the OR over entries of (a >= 0 ? a : ~a), whose bit
// length is the largest bit length of those terms.
__host__ __device__ __forceinline__ int width_from_stats(uint64_t orv, uint32_t neg) {
#ifdef __CUDA_ARCH__
  int len = bitlen64(orv);
#else
  int len = 0;
  for (uint64_t v = orv; v; v >>= 1) ++len;
#endif
  if (neg) return len + 1;
  return len > 1 ? len : 1;
}

__device__ __forceinline__ uint64_t fold(int64_t v) { return (uint64_t)(v ^ (v >> 63)); }

__host__ __device__ __forceinline__ uint64_t field_mask(int b) {
  return b >= 64 ? ~0ull : ((1ull << b) - 1ull);
}

__host__ __device__ __forceinline__ uint64_t words_for(uint64_t n, int b) {
  if (b < 1 || b > 64 || n == 0) return 0;
  uint64_t data = (n * (uint64_t)b + 31) >> 5;
  return (data + 3) & ~3ull;
}

__host__ __device__ __forceinline__ uint64_t data_words(uint64_t n, int b) {
  return (n * (uint64_t)b + 31) >> 5;
}

// Sign- or zero-extend the low b bits of `bits`.
__device__ __forceinline__ int64_t extend(uint64_t bits, int b, int sgn) {
  if (b >= 64) return (int64_t)bits;
  if (sgn) {
    int sh = 64 - b;
    return (int64_t)(bits << sh) >> sh;
  }
  return (int64_t)(bits & ((1ull << b) - 1ull));
}

// Positions of the sign bits of the 32 fields of a B-bit group (B words)
// that fall in word i of the group: XOR-ing them turns two's complement
// fields into offset binary (u = a + 2^(B-1)).
__host__ __device__ constexpr uint32_t group_sign_bits(int B, int i) {
  uint32_t m = 0;
  for (int e = 0; e < 32; ++e) {
    const int p = e * B + B - 1;
    if ((p >> 5) == i) m |= 1u << (p & 31);
  }
  return m;
}

// Field e of a stream at runtime width b (1..64), straight from global
// memory.  Touches only words that hold bits of the field.
__device__ __forceinline__ int64_t decode_field(const uint32_t* __restrict__ w, uint64_t e, int b,
                                                int sgn) {
  uint64_t p = e * (uint64_t)b;
  uint64_t wi = p >> 5;
  int s = (int)(p & 31);
  uint64_t bits = (uint64_t)__ldg(w + wi) >> s;
  int have = 32 - s;
  if (have < b) {
    bits |= (uint64_t)__ldg(w + wi + 1) << have;
    have += 32;
    if (have < b) bits |= (uint64_t)__ldg(w + wi + 2) << have;
  }
  return extend(bits, b, sgn);
}

// The first 32 bytes of a header (magic, width, sign, status, rows, cols),
// read with two 16-byte loads issued together: one memory round trip.
struct HeaderView {
  uint32_t magic;
  int width, is_signed, status;
  uint64_t rows, cols;
};

__device__ __forceinline__ HeaderView load_header(const ccm_header* h) {
  const uint4* p = reinterpret_cast<const uint4*>(h);
  const uint4 q0 = p[0], q1 = p[1];
  HeaderView v;
  v.magic = q0.x;
  v.width = (int)q0.y;
  v.is_signed = (int)q0.z;
  v.status = (int)q0.w;
  v.rows = ((uint64_t)q1.y << 32) | q1.x;
  v.cols = ((uint64_t)q1.w << 32) | q1.z;
  return v;
}

// A valid input header: magic set, no error, width in range, the expected
// shape, and words that fit the caller's buffer (so no read can leave it).
// Returns CCM_OK or the status to pass on.
__device__ __forceinline__ int check_header(const HeaderView& h, uint64_t rows, uint64_t cols,
                                            uint64_t capacity) {
  if (h.magic != CCM_MAGIC) return CCM_E_INPUT;
  if (h.status != CCM_OK) return h.status;
  if (h.width < 1 || h.width > 64) return CCM_E_INPUT;
  if (h.rows != rows || h.cols != cols) return CCM_E_INPUT;
  if (words_for(rows * cols, h.width) > capacity) return CCM_E_INPUT;
  return CCM_OK;
}

__device__ __forceinline__ int check_input(const ccm_header* h, uint64_t rows, uint64_t cols,
                                           uint64_t capacity) {
  return check_header(load_header(h), rows, cols, capacity);
}

__device__ __forceinline__ void set_status(ccm_header* h, int code) {
  atomicCAS(reinterpret_cast<int*>(&h->status), CCM_OK, code);
}

__device__ __forceinline__ uint64_t warp_or64(uint64_t v) {
  uint32_t lo = __reduce_or_sync(0xffffffffu, (uint32_t)v);
  uint32_t hi = __reduce_or_sync(0xffffffffu, (uint32_t)(v >> 32));
  return ((uint64_t)hi << 32) | lo;
}

// Exact int64 add / multiply with overflow detection.
__device__ __forceinline__ int64_t add_checked(int64_t a, int64_t b, int& ovf) {
  int64_t s = (int64_t)((uint64_t)a + (uint64_t)b);
  ovf |= (int)((((a ^ s) & (b ^ s)) >> 63) & 1);
  return s;
}

__device__ __forceinline__ int64_t mul_checked(int64_t a, int64_t b, int& ovf) {
  int64_t lo = (int64_t)((uint64_t)a * (uint64_t)b);
  int64_t hi = __mul64hi(a, b);
  ovf |= (int)(hi != (lo >> 63));
  return lo;
}

}  // namespace ccm
