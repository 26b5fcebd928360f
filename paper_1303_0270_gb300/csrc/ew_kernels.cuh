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
//
// Add and scale first try one pass: the input headers bound the result to a
// range (for add, the sum of the two ranges; for scale, s times the range
// of A) and so to a width b_spec; the statistics pass also writes every
// field at b_spec.  When the exact width turns out to be b_spec -- the usual
// case: the bound is reached as soon as one pair of entries is near its
// extremes -- the pack pass only finalises the header; otherwise it re-packs
// at the exact width as above.
//
// Memory-level parallelism: a warp loads the words of its next tile into
// registers (16-byte loads) while it decodes the current one, so every warp
// keeps one tile of every input in flight.
#pragma once

#include <type_traits>

#include "async_copy.cuh"
#include "group_engine.cuh"
#include "pack_engine.cuh"

namespace ccm {
namespace ge {

// Words of one packed input tile held in registers: Q 16-byte vectors per
// lane cover the 32*b <= 8*BMAX... words of a tile for b <= BMAX.
template <int BMAX>
struct TileRegs {
  static constexpr int Q = (BMAX + 3) / 4;  // uint4 per lane: 32*BMAX words / 4 / 32
  uint4 r[Q];
};

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
  // Global -> registers: uint4 index lane + 32 j of the tile (zero past the end).
  template <int BMAX>
  __device__ __forceinline__ void load(TileRegs<BMAX>& t, uint64_t tile, int lane) const {
    const uint64_t w0 = tile * (uint64_t)(32 * b);
    const int nq = 8 * b;  // uint4 per tile
    const bool whole = w0 + 32 * (uint64_t)b <= dw;
#pragma unroll
    for (int j = 0; j < TileRegs<BMAX>::Q; ++j) {
      const int q = lane + 32 * j;
      uint4 v = make_uint4(0, 0, 0, 0);
      if (q < nq) {
        if (whole) {
          v = __ldg(reinterpret_cast<const uint4*>(w + w0) + q);
        } else {
          const uint64_t g = w0 + 4 * (uint64_t)q;
          if (g < dw) v.x = __ldg(w + g);
          if (g + 1 < dw) v.y = __ldg(w + g + 1);
          if (g + 2 < dw) v.z = __ldg(w + g + 2);
          if (g + 3 < dw) v.w = __ldg(w + g + 3);
        }
      }
      t.r[j] = v;
    }
  }
  // Global -> shared in plain word order for the lane pass at compile-time
  // width B (= b): the data words of tile `tile`, rounded up to 16 bytes
  // (the canonical zero padding of the stream), by one bulk copy that lane 0
  // issues on `bar`; the warp zeroes the rest of the buffer first.  Returns
  // the bytes the copy brings (all lanes).
  template <int B>
  __device__ __forceinline__ uint32_t fill_tile(uint64_t tile, uint32_t* buf, uint64_t* bar,
                                                int lane) const;
  // Registers -> shared staging layout.
  template <int BMAX>
  __device__ __forceinline__ void stage(const TileRegs<BMAX>& t, uint32_t* buf, int lane) const {
    const int nq = 8 * b;
#pragma unroll
    for (int j = 0; j < TileRegs<BMAX>::Q; ++j) {
      const int q = lane + 32 * j;
      if (q < nq) {
        const int w = 4 * q;
        buf[stage_pos(w, b)] = t.r[j].x;
        buf[stage_pos(w + 1, b)] = t.r[j].y;
        buf[stage_pos(w + 2, b)] = t.r[j].z;
        buf[stage_pos(w + 3, b)] = t.r[j].w;
      }
    }
  }
};

constexpr int kRegion = kBufWords / 2;  // 1056 words: one packed tile of width <= 32

// The values a b-bit field can hold (b <= 63).
__device__ __forceinline__ int64_t range_lo(int b, int sgn) { return sgn ? -(1ll << (b - 1)) : 0; }
__device__ __forceinline__ int64_t range_hi(int b, int sgn) {
  return sgn ? (1ll << (b - 1)) - 1 : (1ll << b) - 1;
}
// The width (Eq. 1, two's complement when lo < 0) of the values [lo, hi].
__device__ __forceinline__ int range_width(int64_t lo, int64_t hi) {
  const int h = bitlen64((uint64_t)(hi > 0 ? hi : 0));
  if (lo >= 0) return h > 1 ? h : 1;
  const int l = bitlen64((uint64_t)~lo);
  return 1 + (h > l ? h : l);
}

// cp.async helpers (16 bytes, zero-filled past `bytes`; commit; wait).
__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, uint32_t bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit_ge() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait1_ge() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait0_ge() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait2_ge() {
  asm volatile("cp.async.wait_group 2;\n" ::: "memory");
}

template <int B>
__device__ __forceinline__ uint32_t PackedIn::fill_tile(uint64_t tile, uint32_t* buf,
                                                       uint64_t* bar, int lane) const {
  constexpr uint32_t TW = 32 * B;
  const uint64_t w0 = tile * (uint64_t)TW;
  const uint32_t valid = (uint32_t)umin((uint64_t)TW, dw - w0);  // tile < ntiles: w0 < dw
  const uint32_t cw = (valid + 3u) & ~3u;
  if (cw < TW)  // the last tile: zero words past the copy (fields past n read 0)
    for (uint32_t i = cw + lane; i < TW; i += 32) buf[i] = 0;
  if (lane == 0) ax::bulk_g2s(buf, w + w0, 4 * cw, bar);
  return 4 * cw;
}

// NW consecutive shared words from word w0 (w0 a multiple of the vector
// width chosen: 4 words when NW % 4 == 0, else 2 when even, else 1).
template <int NW>
__device__ __forceinline__ void lds_words(const uint32_t* buf, int w0, uint32_t* w) {
  if constexpr (NW % 4 == 0) {
#pragma unroll
    for (int i = 0; i < NW / 4; ++i) {
      const uint4 v = *reinterpret_cast<const uint4*>(buf + w0 + 4 * i);
      w[4 * i] = v.x, w[4 * i + 1] = v.y, w[4 * i + 2] = v.z, w[4 * i + 3] = v.w;
    }
  } else if constexpr (NW % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NW / 2; ++i) {
      const uint2 v = *reinterpret_cast<const uint2*>(buf + w0 + 2 * i);
      w[2 * i] = v.x, w[2 * i + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int i = 0; i < NW; ++i) w[i] = buf[w0 + i];
  }
}

template <int NW>
__device__ __forceinline__ void sts_words(uint32_t* buf, int w0, const uint32_t* w) {
  if constexpr (NW % 4 == 0) {
#pragma unroll
    for (int i = 0; i < NW / 4; ++i)
      *reinterpret_cast<uint4*>(buf + w0 + 4 * i) =
          make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
  } else if constexpr (NW % 2 == 0) {
#pragma unroll
    for (int i = 0; i < NW / 2; ++i)
      *reinterpret_cast<uint2*>(buf + w0 + 2 * i) = make_uint2(w[2 * i], w[2 * i + 1]);
  } else {
#pragma unroll
    for (int i = 0; i < NW; ++i) buf[w0 + i] = w[i];
  }
}

// ---------------------------------------------------------------------------
// Operations.  produce() hands every field value of the lane's group to
// sink(k, value) as Val<BMAX> (int32 when the class bounds every value below
// 2^31, int64 otherwise); loads for the next tile are issued by prefetch().
// Fields past the end of the matrix need no masking: they decode from the
// zero bits above the last field (a packed matrix is canonical) or from the
// zero fill of words past the end, and give 0 in every operation.
// ---------------------------------------------------------------------------
// Results of 33..36 bits (the sum of two 32-bit operands, a scaled 32-bit
// one) take one 64-bit value per field; narrower ones the slot form below.

// Field c (B <= 32 bits) of a lane's group, zero-extended to 64 bits.
template <int B>
__device__ __forceinline__ uint64_t spread64(const uint32_t* w, int c) {
  const int bit = B * c, wi = bit >> 5, sh = bit & 31;
  const uint32_t x = sh + B <= 32 ? (w[wi] >> sh) : __funnelshift_r(w[wi], w[wi + 1], sh);
  return (uint64_t)(B >= 32 ? x : (x & ((1u << B) - 1u)));
}

// A result r in offset binary at width BS = 33..36 (r = c + 2^(BS-1)):
// c >= 0 exactly when bit BS - 1 is set; returns the two's complement bits
// of c (r ^ 2^(BS-1)) and ORs the folded value (c >= 0 ? c : ~c, the bits
// below BS - 1) into `orb`, the sign into `neg`.
template <int BS>
__device__ __forceinline__ uint64_t offset_out64(uint64_t r, uint64_t& orb, uint32_t& neg) {
  constexpr uint64_t lo = (1ull << (BS - 1)) - 1ull, top = 1ull << (BS - 1);
  const uint64_t pos = (r >> (BS - 1)) & 1ull;  // c >= 0
  orb |= (r ^ lo ^ (pos * lo)) & lo;
  neg |= (uint32_t)(pos ^ 1ull);
  return r ^ top;
}

// Slot form of the lane pass (results of BS <= 32 bits): KS = 32 / BS
// fields of a lane's group side by side in one 32-bit word, field j in bits
// [j BS, j BS + BS), so that the sum (or the scaled value) of a word of
// slots is one add (one multiply-add) and lands already packed at width BS.
// expand_slots moves K consecutive B-bit fields (bits [j B, j B + B)) into
// the slots: log2 K steps, highest first, each moving the fields whose index
// has bit p set by p (BS - B) bits with one AND and one multiply-add,
// x + (x & m) (2^d - 1) = (x & ~m) + ((x & m) << d), which runs on the FMA
// pipe beside the integer one.
__host__ __device__ constexpr int slot_fields(int bs) { return 32 / bs; }

__host__ __device__ constexpr uint32_t slot_ones(int bs, int k) {
  uint32_t m = 0;
  for (int j = 0; j < k; ++j) m |= 1u << (j * bs);
  return m;
}

// Bits of the fields moved at step p (their positions before the step).
__host__ __device__ constexpr uint32_t slot_move_mask(int b, int g, int k, int p) {
  uint32_t m = 0;
  for (int j = 0; j < k; ++j)
    if (j & p) m |= ((1u << b) - 1u) << (j * b + (j & ~(2 * p - 1)) * g);
  return m;
}

__host__ __device__ constexpr int top_pow2(int v) {
  int p = v >= 1 ? 1 : 0;
  while (p && p * 2 <= v) p *= 2;
  return p;
}

template <int B, int G, int K, int P>
__device__ __forceinline__ uint32_t expand_steps(uint32_t x) {
  if constexpr (P == 0) {
    return x;
  } else {
    constexpr uint32_t m = slot_move_mask(B, G, K, P);
    constexpr uint32_t f = (1u << (P * G)) - 1u;
    return expand_steps<B, G, K, P / 2>((x & m) * f + x);
  }
}

// Fields c K .. c K + K - 1 of a lane's B-bit group (words w, w[B] = 0) in
// slots of B + G bits.
template <int B, int G, int K>
__device__ __forceinline__ uint32_t expand_slots(const uint32_t* w, int first) {
  const int bit = B * first, wi = bit >> 5, sh = bit & 31;
  const uint32_t x = sh + K * B <= 32 ? (w[wi] >> sh) : __funnelshift_r(w[wi], w[wi + 1], sh);
  return expand_steps<B, G, K, top_pow2(K - 1)>(x & ((1u << (K * B)) - 1u));  // K B < 32
}

// offset_out for K slots of BS bits.
template <int BS, int K>
__device__ __forceinline__ uint32_t offset_out_slots(uint32_t r, uint32_t& orb, uint32_t& neg) {
  constexpr uint32_t ones = slot_ones(BS, K);
  constexpr uint32_t lo1 = (1u << (BS - 1)) - 1u;
  constexpr uint32_t lo = lo1 * ones;
  constexpr uint32_t top = (1u << (BS - 1)) * ones;
  const uint32_t pos = ((r >> (BS - 1)) & ones) * lo1;  // slots with c >= 0
  orb |= (r ^ lo ^ pos) & lo;
  neg |= ~r & top;
  return r ^ top;
}

// Bytes fill_tile brings for tile `tile` of input x at width B.
template <int B>
__device__ __forceinline__ uint32_t lanes_fill_bytes(const PackedIn& x, uint64_t tile) {
  const uint64_t w0 = tile * (uint64_t)(32 * B);
  return 4 * (((uint32_t)umin((uint64_t)(32 * B), x.dw - w0) + 3u) & ~3u);
}

struct OpAdd {
  PackedIn a, b;
  template <int BMAX>
  using Val = typename std::conditional<(BMAX <= 16), int32_t, int64_t>::type;
  template <int BMAX>
  struct Regs {
    TileRegs<BMAX> ra, rb;
  };
  __device__ __forceinline__ void init(uint64_t n) {
    a.init(n);
    b.init(n);
  }
  // Width of [lo_a + lo_b, hi_a + hi_b] (widths of at most 32 bits here).
  __device__ __forceinline__ int spec_width() const {
    const int64_t lo = range_lo(a.b, a.sgn) + range_lo(b.b, b.sgn);
    const int64_t hi = range_hi(a.b, a.sgn) + range_hi(b.b, b.sgn);
    return range_width(lo, hi);
  }
  // Lanes apply when both operands have the same width B <= 31 and sign
  // mode: the sum then needs B + 1 bits (the speculative width) and fits a
  // lane of 8, 16 or 32 bits.  Returns B (0: not applicable).
  __device__ __forceinline__ int lanes_width(int bs) const {
    return (a.sgn == b.sgn && a.b == b.b && a.b <= 32 && bs == a.b + 1) ? a.b : 0;
  }
  static constexpr int kLaneGrow = 1;  // BS = B + 1
  // Lane mode: 0 unsigned operands, 1 signed (offset binary in and out).
  __device__ __forceinline__ int lanes_mode() const { return a.sgn; }
  // Mask of the sign-bit XOR on the inputs in mode 1 (all of them here).
  __device__ __forceinline__ uint32_t lanes_in_xor() const { return ~0u; }
  struct LaneConst {};
  template <int B, int BS, int MODE>
  __device__ __forceinline__ LaneConst lanes_const() const {
    return {};
  }
  struct SlotConst {};
  template <int B, int BS, int KS, int KL, int MODE>
  __device__ __forceinline__ SlotConst slots_const() const {
    return {};
  }
  // Fields first .. first + K - 1 in slot form: the sums, with the
  // statistics (offset binary for signed operands, as in lanes_k).
  template <int B, int BS, int K, bool LAST, int MODE>
  __device__ __forceinline__ uint32_t slots_k(const uint32_t* wa, const uint32_t* wb, int first,
                                              uint32_t& orb, uint32_t& neg,
                                              const SlotConst&) const {
    const uint32_t r = expand_slots<B, BS - B, K>(wa, first) + expand_slots<B, BS - B, K>(wb, first);
    if constexpr (MODE == 0) {
      orb |= r;
      return r;
    } else {
      return offset_out_slots<BS, K>(r, orb, neg);
    }
  }
  // Field c of the lane's group when the sum has 33 bits (B = 32): the sum
  // in a 64-bit value with the statistics of the result.  Signed inputs
  // arrive in offset binary (u = a + 2^(B-1)), so u_a + u_b = c + 2^B is the
  // sum in offset binary at width B + 1.
  template <int B, int BS, int MODE>
  __device__ __forceinline__ uint64_t lanes_k(const uint32_t* wa, const uint32_t* wb, int c,
                                              uint64_t& orb, uint32_t& neg,
                                              const LaneConst&) const {
    const uint64_t sum = spread64<B>(wa, c) + spread64<B>(wb, c);
    if constexpr (MODE == 0) {
      orb |= sum;
      return sum;
    } else {
      return offset_out64<BS>(sum, orb, neg);
    }
  }
  static constexpr bool kTwoInputs = true;
  // tile `tile` of both inputs into plain-order shared buffers, one bulk
  // copy each on `bar` (lane 0 arms it with the bytes of both)
  template <int B>
  __device__ __forceinline__ void lanes_fill(uint64_t tile, uint32_t* bufa, uint32_t* bufb,
                                             uint64_t* bar, int lane) const {
    if (lane == 0) ax::mbar_expect_tx(bar, 2 * lanes_fill_bytes<B>(a, tile));
    a.template fill_tile<B>(tile, bufa, bar, lane);
    b.template fill_tile<B>(tile, bufb, bar, lane);
  }
  template <int BMAX>
  __device__ __forceinline__ void prefetch(Regs<BMAX>& r, uint64_t tile, int lane) const {
    a.load(r.ra, tile, lane);
    b.load(r.rb, tile, lane);
  }
  template <int BMAX, class Sink>
  __device__ __forceinline__ void produce(const Regs<BMAX>& r, uint32_t* buf, int lane,
                                          int& ovf, Sink&& sink) const {
    using V = Val<BMAX>;
    uint32_t* ba = buf;
    uint32_t* bb = buf + kRegion;
    a.stage(r.ra, ba, lane);
    b.stage(r.rb, bb, lane);
    __syncwarp();
    V va[32];
    decode_dispatch<BMAX>(a.b, a.sgn, ba, lane, [&](int k, int64_t x) { va[k] = (V)x; });
    decode_dispatch<BMAX>(b.b, b.sgn, bb, lane, [&](int k, int64_t x) {
      if constexpr (BMAX <= 16)
        sink(k, (V)(va[k] + (V)x));  // |sum| < 2^17
      else
        sink(k, (V)add_checked((int64_t)va[k], x, ovf));
    });
    __syncwarp();
  }
};

// SMALL: the host checked |s| < 2^15, so in the classes up to 16 bits every
// product stays below 2^31 and is computed in 32 bits.
template <bool SMALL>
struct OpScale {
  PackedIn a;
  int64_t s;
  template <int BMAX>
  using Val = typename std::conditional<(SMALL && BMAX <= 16), int32_t, int64_t>::type;
  template <int BMAX>
  struct Regs {
    TileRegs<BMAX> ra;
  };
  __device__ __forceinline__ void init(uint64_t n) { a.init(n); }
  // Width of s times the range of A (65 when that leaves int64).
  __device__ __forceinline__ int spec_width() const {
    __int128 lo = (__int128)range_lo(a.b, a.sgn) * s, hi = (__int128)range_hi(a.b, a.sgn) * s;
    if (lo > hi) {
      const __int128 t = lo;
      lo = hi;
      hi = t;
    }
    const __int128 lim = (__int128)1 << 62;
    if (lo < -lim || hi >= lim) return 65;
    return range_width((int64_t)lo, (int64_t)hi);
  }
  // Lanes apply for 1 <= |s| < 2^5, A of at most 32 bits and a speculative
  // width BS = B + D with 1 <= D <= kLaneGrow (every result then fits its
  // BS-bit slot, or its 64-bit value), except 1-bit signed A with s < 0
  // (values {-1, 0}: a non-negative result range, not the signed one mode 1
  // writes).  Returns B (0: not applicable).
  static constexpr int kLaneGrow = 4;
  __device__ __forceinline__ int lanes_width(int bs) const {
    const int64_t t = s < 0 ? -s : s;
    if (t < 1 || t >= 32 || a.b > 32 || bs - a.b < 1 || bs - a.b > kLaneGrow) return 0;
    if (a.sgn && a.b == 1 && s < 0) return 0;
    return a.b;
  }
  // Lane mode: 0 unsigned A and s > 0 (unsigned result); 1 signed A, or
  // unsigned A and s < 0 (offset binary out; the sign-bit XOR on the input
  // only for signed A).
  __device__ __forceinline__ int lanes_mode() const { return (a.sgn || s < 0) ? 1 : 0; }
  __device__ __forceinline__ uint32_t lanes_in_xor() const { return a.sgn ? ~0u : 0u; }
  // With t = |s| and v = u (s > 0) or its B-bit complement (s < 0), where u
  // is A's field in offset binary (signed) or plain (unsigned), the result
  // in offset binary at width BS is r = t v + P for one constant P >= 0:
  //   signed, s > 0:   c = t u - t 2^(B-1),        P = 2^(BS-1) - t 2^(B-1)
  //   signed, s < 0:   c = t v - t (2^(B-1) - 1),  P = 2^(BS-1) - t (2^(B-1) - 1)
  //   unsigned, s < 0: c = t v - t (2^B - 1),      P = 2^(BS-1) - t (2^B - 1)
  // (mode 0: r = t a, P = 0; mode 1: the other three).  BS is the width of s times A's range, so every
  // r lies in [0, 2^BS): one multiply and one add per word of slots (per
  // 64-bit value for BS > 32), no carry from one slot into the next.
  struct LaneConst {  // the 64-bit values (BS = 33..36)
    uint32_t t, cmask;  // |s|; the complement mask (s < 0)
    uint64_t p;         // P
  };
  template <int B, int BS, int MODE>
  __device__ __forceinline__ LaneConst lanes_const() const {
    constexpr uint64_t lob = (1ull << B) - 1ull;
    const uint32_t t = (uint32_t)(s < 0 ? -s : s);
    if constexpr (MODE == 0) {
      return {t, 0u, 0ull};
    } else {
      const uint64_t half = 1ull << (BS - 1);
      const uint64_t p = !a.sgn ? half - t * lob
                         : s > 0 ? half - t * (1ull << (B - 1))
                                 : half - t * ((1ull << (B - 1)) - 1ull);
      return {t, s < 0 ? (uint32_t)lob : 0u, p};
    }
  }
  // Slot form: t, the complement masks and P per word of KS slots (the
  // chunks) and of KL slots (the last chunk of a group).
  struct SlotConst {
    uint32_t t, cm_k, cm_l, p_k, p_l;
  };
  template <int B, int BS, int KS, int KL, int MODE>
  __device__ __forceinline__ SlotConst slots_const() const {
    constexpr uint32_t lob = B >= 32 ? ~0u : (1u << B) - 1u;
    const uint32_t t = (uint32_t)(s < 0 ? -s : s);
    if constexpr (MODE == 0 || BS > 32) {  // (BS > 32: the 64-bit lanes, not slots)
      return {t, 0u, 0u, 0u, 0u};
    } else {
      const uint32_t half = 1u << (BS - 1);
      const uint32_t p = !a.sgn ? half - t * lob
                         : s > 0 ? half - t * (1u << (B - 1))
                                 : half - t * ((1u << (B - 1)) - 1u);
      const bool c = s < 0;
      return {t, c ? lob * slot_ones(BS, KS) : 0u, c ? lob * slot_ones(BS, KL) : 0u,
              p * slot_ones(BS, KS), p * slot_ones(BS, KL)};
    }
  }
  template <int B, int BS, int K, bool LAST, int MODE>
  __device__ __forceinline__ uint32_t slots_k(const uint32_t* wa, const uint32_t*, int first,
                                              uint32_t& orb, uint32_t& neg,
                                              const SlotConst& kc) const {
    const uint32_t v = expand_slots<B, BS - B, K>(wa, first);
    if constexpr (MODE == 0) {
      const uint32_t r = v * kc.t;
      orb |= r;
      return r;
    } else {
      const uint32_t cm = LAST ? kc.cm_l : kc.cm_k, p = LAST ? kc.p_l : kc.p_k;
      return offset_out_slots<BS, K>((v ^ cm) * kc.t + p, orb, neg);
    }
  }
  // Field c of the lane's group scaled, for BS = 33..36 (a 64-bit value).
  template <int B, int BS, int MODE>
  __device__ __forceinline__ uint64_t lanes_k(const uint32_t* wa, const uint32_t*, int c,
                                              uint64_t& orb, uint32_t& neg,
                                              const LaneConst& kc) const {
    const uint64_t v = spread64<B>(wa, c);
    if constexpr (MODE == 0) {
      const uint64_t r = v * kc.t;
      orb |= r;
      return r;
    } else {
      return offset_out64<BS>((v ^ kc.cmask) * kc.t + kc.p, orb, neg);
    }
  }
  static constexpr bool kTwoInputs = false;
  template <int B>
  __device__ __forceinline__ void lanes_fill(uint64_t tile, uint32_t* bufa, uint32_t*,
                                             uint64_t* bar, int lane) const {
    if (lane == 0) ax::mbar_expect_tx(bar, lanes_fill_bytes<B>(a, tile));
    a.template fill_tile<B>(tile, bufa, bar, lane);
  }
  template <int BMAX>
  __device__ __forceinline__ void prefetch(Regs<BMAX>& r, uint64_t tile, int lane) const {
    a.load(r.ra, tile, lane);
  }
  template <int BMAX, class Sink>
  __device__ __forceinline__ void produce(const Regs<BMAX>& r, uint32_t* buf, int lane,
                                          int& ovf, Sink&& sink) const {
    using V = Val<BMAX>;
    a.stage(r.ra, buf, lane);
    __syncwarp();
    const int64_t sc = s;
    decode_dispatch<BMAX>(a.b, a.sgn, buf, lane, [&](int k, int64_t x) {
      if constexpr (sizeof(V) == 4)
        sink(k, (V)((int32_t)x * (int32_t)sc));
      else
        sink(k, mul_checked(x, sc, ovf));
    });
    __syncwarp();
  }
};

// Pass of add / scale: statistics (kStats), pack at the width the header's
// statistics give (kPack), or statistics plus every field written at the
// speculative width (kSpec).  kPack with `spec` set follows a kSpec launch
// and returns after the header when the exact width is the speculative one.
constexpr int kStats = 0, kPack = 1, kSpec = 2;

// The speculative pass on lanes, a kernel of its own (few registers, buffers
// sized to the operands: many warps per SM) launched before k_ew<..., kSpec>:
// when the operands qualify (Op::lanes_width, decided from the headers), it
// does the pass and marks the output header (reserved1 = 1) so that the
// general kSpec launch returns at once; otherwise it returns and the general
// pass runs.  Input width B, output width BS (slot form for BS <= 32, one
// 64-bit value per field above) and sign mode are compile-time.  Per tile
// the inputs are staged in plain word order through a ring of bulk copies
// (one per input tile, issued by lane 0 on the slot's mbarrier, waits
// bounded); each lane reads its group's B words with the widest aligned
// vector (signed inputs: XOR of the sign bits), forms the results a word of
// slots at a time (one add, or one multiply-add, for 32 / BS fields), ORs the
// statistics, places each word at its bit offset among its BS output words
// and stores those; the warp then writes the output tile with 16-byte
// stores.
__host__ __device__ constexpr int lane_stages(int B) { return B <= 8 ? 3 : 2; }

// Shared words per warp of the pass at input width b and output width bs
// with `inputs` operands: the ring, then the output tile.
__host__ __device__ constexpr uint32_t lane_body_words(int b, int bs, int inputs) {
  return (uint32_t)(lane_stages(b) * inputs * 32 * b + 32 * bs);
}

// Shared words per warp for input widths up to bmax and output widths up to
// `grow` bits wider.
__host__ __device__ constexpr uint32_t lane_warp_words(int bmax, int inputs, int grow) {
  uint32_t m = 0;
  for (int b = 1; b <= bmax; ++b) {
    const uint32_t v = lane_body_words(b, b + grow, inputs);
    if (v > m) m = v;
  }
  return m;
}

template <class Op, int B, int BS, int L, int MODE>
__device__ __noinline__ void lanes_body(const Op& op, ccm_header* out, uint32_t* words,
                                        uint64_t n, uint32_t* sbuf, uint64_t* bar) {
  constexpr int S = lane_stages(B);
  constexpr int TW = 32 * B;  // words of an input tile
  constexpr int NI = Op::kTwoInputs ? 2 : 1;
  // slot form (BS <= 32): KS fields per chunk, NC chunks, KL in the last
  constexpr int KS = L == 64 ? 1 : slot_fields(BS);
  constexpr int NC = (32 + KS - 1) / KS, KL = 32 - (NC - 1) * KS;
  const typename Op::LaneConst kc = op.template lanes_const<B, BS, MODE>();
  const typename Op::SlotConst sc = op.template slots_const<B, BS, KS, KL, MODE>();
  const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  const uint64_t dw = data_words(n, BS);
  const uint64_t ntiles = (n + kTile - 1) / kTile;
  const uint64_t gwarps = (uint64_t)gridDim.x * kWarps;
  const uint64_t tile0 = (uint64_t)blockIdx.x * kWarps + warp;
  // per warp: S slots of (A tile[, B tile]), then the output tile
  uint32_t* obuf = sbuf + S * NI * TW;
  auto slot_a = [&](uint32_t k) { return sbuf + (k % S) * NI * TW; };
  uint64_t orb = 0;     // (the 64-bit path)
  uint32_t orb32 = 0;   // (slot form)
  uint32_t neg = 0;
  // bulk-copy ring: the next S - 1 tiles in flight while tile k is decoded,
  // slot k % S completing phase (k / S) & 1 of its mbarrier
  if (lane == 0) {
    for (int i = 0; i < S; ++i) ax::mbar_init(&bar[i], 1);
    ax::mbar_init_fence();
  }
  __syncwarp();
#pragma unroll
  for (uint32_t k = 0; k < S - 1; ++k) {
    const uint64_t t = tile0 + k * gwarps;
    if (t < ntiles) op.template lanes_fill<B>(t, slot_a(k), slot_a(k) + TW, &bar[k], lane);
  }
  uint32_t k = 0;
  bool ok = true;
  for (;; ++k) {
    const uint64_t tile = tile0 + k * gwarps;
    if (tile >= ntiles) break;
    const uint64_t tn = tile + (S - 1) * gwarps;
    if (tn < ntiles) {  // slot of tile k - 1: read by every lane before the last __syncwarp
      if (lane == 0) ax::fence_proxy_async_smem();
      op.template lanes_fill<B>(tn, slot_a(k + S - 1), slot_a(k + S - 1) + TW,
                                &bar[(k + S - 1) % S], lane);
    }
    if (!ax::mbar_wait(&bar[k % S], (k / S) & 1)) {
      ok = false;
      break;
    }
    __syncwarp();
    const uint32_t* bufa = slot_a(k);
    uint32_t wa[B + 1], wb[B + 1];
    lds_words<B>(bufa, lane * B, wa);
    wa[B] = 0;
    if constexpr (Op::kTwoInputs) {
      lds_words<B>(bufa + TW, lane * B, wb);
      wb[B] = 0;
    }
    if constexpr (MODE == 1) {  // signed operands: offset binary
      const uint32_t xs = op.lanes_in_xor();
#pragma unroll
      for (int i = 0; i < B; ++i) {
        wa[i] ^= group_sign_bits(B, i) & xs;
        if constexpr (Op::kTwoInputs) wb[i] ^= group_sign_bits(B, i) & xs;
      }
    }
    uint32_t ow[BS + 1];
#pragma unroll
    for (int i = 0; i <= BS; ++i) ow[i] = 0;
    if constexpr (L == 64) {
#pragma unroll
      for (int c = 0; c < 32; ++c) {  // one field of 33..36 bits: up to three words
        const uint64_t r = op.template lanes_k<B, BS, MODE>(wa, wb, c, orb, neg, kc);
        const int bit = BS * c, wi = bit >> 5, sh = bit & 31;
        ow[wi] |= (uint32_t)(r << sh);
        if (sh + BS > 32) ow[wi + 1] |= (uint32_t)(r >> (32 - sh));
        if (sh + BS > 64) ow[wi + 2] |= (uint32_t)(r >> (64 - sh));
      }
    } else {
      // slot form: KS fields per chunk (KL in the last), each chunk's word of
      // slots placed at its bit offset with a shift-add and a high multiply
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        uint32_t r;
        if (c == NC - 1)
          r = op.template slots_k<B, BS, KL, true, MODE>(wa, wb, c * KS, orb32, neg, sc);
        else
          r = op.template slots_k<B, BS, KS, false, MODE>(wa, wb, c * KS, orb32, neg, sc);
        const int bit = KS * BS * c, wi = bit >> 5, sh = bit & 31;
        ow[wi] += r << sh;
        if (sh + KS * BS > 32) ow[wi + 1] += __umulhi(r, 1u << sh);  // r >> (32 - sh)
      }
    }
    sts_words<BS>(obuf, lane * BS, ow);
    __syncwarp();
    const uint64_t w0 = tile * (uint64_t)(32 * BS);
    if (w0 + 32 * BS <= dw) {
      uint4* dst = reinterpret_cast<uint4*>(words + w0);
#pragma unroll
      for (int j = 0; j < (8 * BS + 31) / 32; ++j) {
        const int q = lane + 32 * j;
        if (q < 8 * BS) dst[q] = *reinterpret_cast<const uint4*>(obuf + 4 * q);
      }
    } else {
      const int tw = (int)(dw > w0 ? dw - w0 : 0);
      for (int w = lane; w < tw; w += 32) words[w0 + w] = obuf[w];
    }
    __syncwarp();
  }
  if (!ok) {  // a copy that never landed: report it, and wait (bounded) for the rest
    if (lane == 0) set_status(out, CCM_E_TIMEOUT);
    for (uint32_t j = 0; j < S; ++j)
      if (tile0 + (k + j) * gwarps < ntiles) ax::mbar_wait(&bar[(k + j) % S], ((k + j) / S) & 1);
    return;
  }
  uint64_t o;
  if constexpr (L == 64) {
    o = warp_or64(orb);
  } else {
    constexpr uint32_t slot = BS >= 32 ? ~0u : (1u << BS) - 1u;
    uint32_t o32 = 0;
#pragma unroll
    for (int j = 0; j < KS; ++j) o32 |= (orb32 >> (j * BS)) & slot;
    o = __reduce_or_sync(0xffffffffu, o32);
  }
  const uint32_t ng = __reduce_or_sync(0xffffffffu, neg);
  if (lane == 0) {
    if (o) atomicOr(reinterpret_cast<unsigned long long*>(&out->stat_or), (unsigned long long)o);
    if (ng) atomicOr(&out->stat_neg, 1u);
  }
}

// Calls lanes_body for the run-time (b, bs, mode).  Add: B <= 32 with
// BS = B + 1; scale: B <= 32 with BS = B + D, 1 <= D <= kLaneGrow.  L = 64:
// one 64-bit value per field (BS > 32); L = 32: the slot form.
template <class Op, int B, int BS>
__device__ __forceinline__ void lanes_modes(const Op& op, int mode, ccm_header* out,
                                            uint32_t* words, uint64_t n, uint32_t* sbuf,
                                            uint64_t* bar) {
  constexpr int L = BS > 32 ? 64 : 32;
  if (mode == 0)
    lanes_body<Op, B, BS, L, 0>(op, out, words, n, sbuf, bar);
  else
    lanes_body<Op, B, BS, L, 1>(op, out, words, n, sbuf, bar);
}

template <class Op, int B, int D = 1>
__device__ __forceinline__ void lanes_grow(const Op& op, int d, int mode, ccm_header* out,
                                           uint32_t* words, uint64_t n, uint32_t* sbuf,
                                           uint64_t* bar) {
  if constexpr (D <= Op::kLaneGrow) {
    if (d == D)
      lanes_modes<Op, B, B + D>(op, mode, out, words, n, sbuf, bar);
    else
      lanes_grow<Op, B, D + 1>(op, d, mode, out, words, n, sbuf, bar);
  }
}

template <class Op, int B = 1>
__device__ __forceinline__ void lanes_dispatch(const Op& op, int b, int bs, int mode,
                                               ccm_header* out, uint32_t* words, uint64_t n,
                                               uint32_t* sbuf, uint64_t* bar) {
  if constexpr (B <= 32) {
    if (b == B)
      lanes_grow<Op, B>(op, bs - B, mode, out, words, n, sbuf, bar);
    else
      lanes_dispatch<Op, B + 1>(op, b, bs, mode, out, words, n, sbuf, bar);
  }
}

// `warp_words`: shared words per warp (lane_warp_words of the host's width
// bound); the dynamic shared memory is kWarps times that.
template <class Op>
__global__ void __launch_bounds__(kThreads) k_ew_lanes(Op op, ccm_header* out, uint32_t* words,
                                                       uint64_t capacity, uint64_t n,
                                                       uint32_t warp_words) {
  extern __shared__ __align__(16) uint32_t s_lanes[];
  __shared__ uint64_t s_lane_bar[kWarps][3];
  if (out->status != CCM_OK) return;
  op.init(n);
  const int bs = op.spec_width();
  int B = (bs <= 32 + Op::kLaneGrow && words_for(n, bs) <= capacity) ? op.lanes_width(bs) : 0;
  if (B && lane_body_words(B, bs, Op::kTwoInputs ? 2 : 1) > warp_words)
    B = 0;  // (buffers sized for narrower inputs)
  if (!B) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out->reserved1 = 1;  // the lane pass wrote the result ...
    out->reserved0 = bs;  // ... at this (speculative) width
  }
  lanes_dispatch<Op>(op, B, bs, op.lanes_mode(), out, words, n,
                     s_lanes + (threadIdx.x / kWarp) * warp_words,
                     s_lane_bar[threadIdx.x / kWarp]);
}

// Host launchers (ew_lanes.cu).
// `bmax`: the host's bound on the input width (from the buffer capacities).
void launch_lanes_add(const OpAdd& op, ccm_header* out, uint32_t* words, uint64_t capacity,
                      uint64_t n, int bmax, cudaStream_t st);
void launch_lanes_scale(const OpScale<true>& op, ccm_header* out, uint32_t* words,
                        uint64_t capacity, uint64_t n, int bmax, cudaStream_t st);

template <class Op, int BMAX, int MODE>
__global__ void __launch_bounds__(kThreads) k_ew(Op op, ccm_header* out, uint32_t* words,
                                                 uint64_t capacity, uint64_t n, int spec) {
  using V = typename Op::template Val<BMAX>;
  using U = typename std::make_unsigned<V>::type;
  constexpr int kSignShift = 8 * sizeof(V) - 1;
  __shared__ __align__(16) uint32_t s_buf[kWarps][kBufWords];
  // after a lane pass or a speculative pass this kernel is launched with
  // programmatic dependent launch: wait for that kernel before reading the
  // header it wrote (a no-op for a normal launch)
  ax::grid_dep_wait();
  int b = 0, sgn = 0;
  if constexpr (MODE == kPack) {
    if (!resolve_output(out, words, capacity, n, b, sgn)) return;
    op.init(n);
    if (spec) {
      const int bs = op.spec_width();
      if (bs <= BMAX && words_for(n, bs) <= capacity && bs == b) return;  // already written
    }
  } else {
    if (out->status != CCM_OK) return;
    if (MODE == kSpec && out->reserved1) return;  // k_ew_lanes did the pass
    op.init(n);
    if constexpr (MODE == kSpec) {
      const int bs = op.spec_width();
      if (bs <= BMAX && words_for(n, bs) <= capacity) b = bs;  // else statistics only
    }
  }
  const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  uint32_t* buf = s_buf[warp];

  const uint64_t dw = b ? data_words(n, b) : 0;
  const uint32_t mask = b >= 32 ? 0xffffffffu : ((1u << b) - 1u);
  const uint64_t ntiles = (n + kTile - 1) / kTile;
  const uint64_t gwarps = (uint64_t)gridDim.x * kWarps;
  U orv = 0;  // OR of (v >= 0 ? v : ~v)
  V negv = 0;  // OR of the values: negative iff some value is
  int ovf = 0;
  uint64_t tile = (uint64_t)blockIdx.x * kWarps + warp;
  typename Op::template Regs<BMAX> cur, nxt;
  if (tile < ntiles) op.template prefetch<BMAX>(cur, tile, lane);
  for (; tile < ntiles; tile += gwarps) {
    if (tile + gwarps < ntiles) op.template prefetch<BMAX>(nxt, tile + gwarps, lane);
    if (MODE == kStats || (MODE == kSpec && b == 0)) {
      op.template produce<BMAX>(cur, buf, lane, ovf, [&](int, V v) {
        orv |= (U)(v ^ (v >> kSignShift));
        negv |= v;
      });
    } else {
      uint32_t u[32];
      op.template produce<BMAX>(cur, buf, lane, ovf, [&](int k, V v) {
        u[k] = (uint32_t)v & mask;
        if constexpr (MODE == kSpec) {
          orv |= (U)(v ^ (v >> kSignShift));
          negv |= v;
        }
      });
      encode_dispatch<BMAX>(b, u, buf, lane);
      __syncwarp();
      store_packed(buf, words, tile, b, dw, lane);
      __syncwarp();
    }
    cur = nxt;
  }
  if constexpr (MODE != kPack) {
    uint64_t o = warp_or64((uint64_t)orv);
    uint32_t neg = __reduce_or_sync(0xffffffffu, (uint32_t)(negv < 0));
    ovf = (int)__reduce_or_sync(0xffffffffu, (uint32_t)ovf);
    if (lane == 0) {
      if (o) atomicOr(reinterpret_cast<unsigned long long*>(&out->stat_or), (unsigned long long)o);
      if (neg) atomicOr(&out->stat_neg, 1u);
      if (ovf) set_status(out, CCM_E_OVERFLOW);
    }
  }
}

// Pack pass of a dense int32/int64 matrix (its statistics come from k_stats).
template <typename T, int BMAX>
__global__ void __launch_bounds__(kThreads) k_pack_dense(const T* __restrict__ src,
                                                         ccm_header* out, uint32_t* words,
                                                         uint64_t capacity, uint64_t n) {
  __shared__ __align__(16) uint32_t s_buf[kWarps][kBufWords];
  int b, sgn;
  if (!resolve_output(out, words, capacity, n, b, sgn)) return;
  const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  uint32_t* buf = s_buf[warp];
  T* tb = reinterpret_cast<T*>(buf);
  const uint64_t dw = data_words(n, b);
  const uint32_t mask = b >= 32 ? 0xffffffffu : ((1u << b) - 1u);
  const uint64_t ntiles = (n + kTile - 1) / kTile;
  const uint64_t gwarps = (uint64_t)gridDim.x * kWarps;
  for (uint64_t tile = (uint64_t)blockIdx.x * kWarps + warp; tile < ntiles; tile += gwarps) {
    const uint32_t nt = (uint32_t)umin((uint64_t)kTile, n - tile * kTile);
    stage_dense<T>(tb, src, tile * kTile, nt, lane);
    __syncwarp();
    uint32_t u[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) u[k] = (uint32_t)tb[33 * lane + k] & mask;
    __syncwarp();
    encode_dispatch<BMAX>(b, u, buf, lane);
    __syncwarp();
    store_packed(buf, words, tile, b, dw, lane);
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// Single-pass pack of a dense matrix (with workspace).  k_pack_local reads
// every dense tile once: it takes the tile's own width b_loc (the width rule
// on the tile's 1024 values), packs the tile at b_loc into its workspace slot
// (32*BMAX words) and merges the tile statistics into the output header.
// Since the matrix width is the largest tile width, b_loc <= b and every
// slot fits.  k_repack then re-codes each slot from b_loc to b (packed bytes
// only, mostly from L2).  Dense traffic: one read instead of two.
//
// Speculative width: the output's capacity bounds b by b_spec (the widest
// width whose words fit).  With b_spec given, every tile is also packed at
// b_spec straight into its final place in the output; if the matrix width
// turns out to be b_spec -- certain as soon as one tile's own width is
// b_spec -- the output is complete after this one pass and k_repack only
// writes the header.  A tile whose width is b_spec sets a flag in the output
// header (reserved1); tiles that see the flag skip their workspace slot,
// which only a narrower matrix needs.  Without the flag every tile keeps
// its slot, so a narrower matrix is re-coded from the slots as above.
// ---------------------------------------------------------------------------
// Dense int64 tiles are double-buffered with 16-byte cp.async (zero fill past
// the end): the next tile is in flight while the warp packs the current one.
// Shared layout: element f at f + 2*(f/32) (keeps 16-byte alignment; the
// lane's 16-byte reads of its 32 elements are conflict-free).
constexpr int kDensePad = kTile + 2 * (kTile / 32);  // int64 slots per staged tile

// Relaxed loads and stores at GPU scope (the speculation flag: written by
// some warps, read by all; no ordering needed beyond eventual visibility).
__device__ __forceinline__ uint64_t ld_relaxed_gpu(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p));
  return v;
}
__device__ __forceinline__ void st_relaxed_gpu(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;\n" ::"l"(p), "l"(v));
}

__device__ __forceinline__ void issue_dense_tile(int64_t* dst, const int64_t* __restrict__ src,
                                                 uint64_t base, uint32_t nt, int lane) {
#pragma unroll 4
  for (int j = 0; j < kTile / 2 / 32; ++j) {
    const uint32_t f = 2 * (lane + 32 * j);
    const uint32_t valid = f + 2 <= nt ? 16u : (f < nt ? 8u : 0u);
    cp_async16_zfill(dst + f + 2 * (f >> 5), src + base + (valid ? f : 0), valid);
  }
}

// The int32 form: element f at f + 4*(f/32) (16-byte aligned chunks of four;
// a lane's 16-byte reads of its 32 elements are conflict-free).
constexpr int kDensePad32 = kTile + 4 * (kTile / 32);  // int32 slots per staged tile

__device__ __forceinline__ void issue_dense_tile(int32_t* dst, const int32_t* __restrict__ src,
                                                 uint64_t base, uint32_t nt, int lane) {
#pragma unroll 4
  for (int j = 0; j < kTile / 4 / 32; ++j) {
    const uint32_t f = 4 * (lane + 32 * j);
    const uint32_t valid = f + 4 <= nt ? 16u : (f < nt ? 4u * (nt - f) : 0u);
    cp_async16_zfill(dst + f + 4 * (f >> 5), src + base + (valid ? f : 0), valid);
  }
}

template <typename T, int BMAX>
__global__ void __launch_bounds__(kThreads) k_pack_local(const T* __restrict__ src,
                                                         ccm_header* out,
                                                         uint32_t* __restrict__ slots,
                                                         uint32_t slot_words,
                                                         uint8_t* __restrict__ tile_width,
                                                         uint64_t n, uint32_t* words,
                                                         int b_spec) {
  // dynamic: kWarps x 2 buffers x kStageWords uint32 words
  constexpr int kStageWords = sizeof(T) == 8 ? 2 * kDensePad : kDensePad32;
  extern __shared__ __align__(16) uint32_t s_dyn[];
  const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  uint32_t* buf0 = s_dyn + warp * 2 * kStageWords;
  const uint64_t ntiles = (n + kTile - 1) / kTile;
  const uint64_t gwarps = (uint64_t)gridDim.x * kWarps;
  uint64_t tile = (uint64_t)blockIdx.x * kWarps + warp;
  // the first dense tile is requested before the header is looked at: with
  // a programmatic launch this overlaps the header's initialisation
  if (tile < ntiles)
    issue_dense_tile(reinterpret_cast<T*>(buf0), src, tile * kTile,
                     (uint32_t)umin((uint64_t)kTile, n - tile * kTile), lane);
  cp_async_commit_ge();
  ax::grid_dep_wait();
  if (out->status != CCM_OK) {
    cp_async_wait0_ge();
    return;
  }
  // b_spec < 0: the statistics are already in the header (an epilogue merged
  // them): the width is exact and every tile goes straight to its place
  const bool exact = b_spec < 0;
  if (exact) b_spec = width_from_stats(out->stat_or, out->stat_neg);
  uint64_t g_or = 0;
  uint32_t g_neg = 0;
  int cur = 0;
  // the speculation flag as this warp last saw it (sticky once set, so a
  // warp stops reading it after the first time it finds it set)
  bool known = exact;
  for (; tile < ntiles; tile += gwarps) {
    const uint32_t nt = (uint32_t)umin((uint64_t)kTile, n - tile * kTile);
    // (read before the tile's wait so that its latency hides behind it)
    if (b_spec && !known) known = ld_relaxed_gpu(&out->reserved1) != 0;
    int64_t v[32];
    {
      const uint64_t next = tile + gwarps;
      if (next < ntiles)
        issue_dense_tile(reinterpret_cast<T*>(buf0 + (cur ^ 1) * kStageWords), src, next * kTile,
                         (uint32_t)umin((uint64_t)kTile, n - next * kTile), lane);
      cp_async_commit_ge();
      cp_async_wait1_ge();
      __syncwarp();
      if constexpr (sizeof(T) == 8) {
        const int64_t* tb = reinterpret_cast<const int64_t*>(buf0 + cur * kStageWords);
#pragma unroll
        for (int k = 0; k < 32; k += 2) {
          const longlong2 p = *reinterpret_cast<const longlong2*>(tb + 34 * lane + k);
          v[k] = p.x;
          v[k + 1] = p.y;
        }
      } else {
        const int32_t* tb = reinterpret_cast<const int32_t*>(buf0 + cur * kStageWords);
#pragma unroll
        for (int k = 0; k < 32; k += 4) {
          const int4 p = *reinterpret_cast<const int4*>(tb + 36 * lane + k);
          v[k] = p.x;
          v[k + 1] = p.y;
          v[k + 2] = p.z;
          v[k + 3] = p.w;
        }
      }
      __syncwarp();
    }
    uint32_t* buf = buf0 + cur * kStageWords;  // the consumed tile's buffer stages the output
    cur ^= 1;
    uint64_t orv = 0;
    uint32_t neg = 0;
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      orv |= fold(v[k]);
      neg |= (uint32_t)(v[k] < 0);
    }
    orv = warp_or64(orv);
    neg = __reduce_or_sync(0xffffffffu, neg);
    g_or |= orv;
    g_neg |= neg;
    const int bl = width_from_stats(orv, neg);
    const bool fits = bl <= BMAX && 32 * bl <= (int)slot_words;
    // the slot is needed unless the matrix width is known to be b_spec
    bool slot = true;
    if (b_spec) {
      if (!exact && bl == b_spec && !known && lane == 0) st_relaxed_gpu(&out->reserved1, 1ull);
      slot = !(known || bl == b_spec);
      known = known || bl == b_spec;
    }
    // up to two encodes of the tile, one code path: at b_spec into the
    // output, then at b_loc into the slot (b_loc <= b_spec, so masking the
    // same registers again only narrows them)
    uint32_t u[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) u[k] = (uint32_t)v[k];
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const int w = pass == 0 ? b_spec : bl;
      if (pass == 0 ? !(b_spec && bl <= b_spec) : !(fits && slot)) continue;
      const uint32_t mask = w >= 32 ? 0xffffffffu : ((1u << w) - 1u);
#pragma unroll
      for (int k = 0; k < 32; ++k) u[k] &= mask;
      encode_dispatch<BMAX>(w, u, buf, lane);
      __syncwarp();
      if (pass == 0) {
        // the tile at b_spec in its final place (the low b_spec bits of a
        // value that fits b_spec bits, signed or not)
        store_packed(buf, words, tile, w, data_words(n, w), lane);
      } else {
        uint4* dst = reinterpret_cast<uint4*>(slots + tile * (uint64_t)slot_words);
        for (int q = lane; q < 8 * w; q += 32) {
          const int wq = 4 * q;
          dst[q] = make_uint4(buf[stage_pos(wq, w)], buf[stage_pos(wq + 1, w)],
                              buf[stage_pos(wq + 2, w)], buf[stage_pos(wq + 3, w)]);
        }
      }
      __syncwarp();
    }
    if (lane == 0 && tile_width) tile_width[tile] = fits ? (uint8_t)(bl | (neg ? 0x80 : 0)) : 0xFF;
  }
  cp_async_wait0_ge();
  if (lane == 0) {
    if (g_or) atomicOr(reinterpret_cast<unsigned long long*>(&out->stat_or), (unsigned long long)g_or);
    if (g_neg) atomicOr(&out->stat_neg, 1u);
  }
}

// k_repack: a warp takes K tiles at a time (tiles t, t + G, ..., G the
// grid's warp count) and issues all their loads before it re-codes any: the
// K width bytes first, then the K slots' words into registers, which go to K
// staging areas of the warp's shared buffer; so a warp waits for two memory
// round trips per K tiles instead of two per tile.  The re-code loop is not
// unrolled (one copy of the width dispatch).
template <int BMAX>
__global__ void __launch_bounds__(kThreads) k_repack(const uint32_t* __restrict__ slots,
                                                     uint32_t slot_words,
                                                     const uint8_t* __restrict__ tile_width,
                                                     ccm_header* out, uint32_t* words,
                                                     uint64_t capacity, uint64_t n, int b_spec) {
  constexpr int Q = (BMAX + 3) / 4;                        // uint4 per lane of a full slot
  constexpr int K = BMAX <= 8 ? 4 : (BMAX <= 16 ? 2 : 1);  // tiles in flight per warp
  constexpr int kArea = 33 * BMAX;                         // staged words of one tile
  static_assert(K * kArea <= kBufWords, "staging areas exceed the warp's buffer");
  __shared__ __align__(16) uint32_t s_buf[kWarps][kBufWords];
  ax::grid_dep_wait();  // (launched early: the local pass must have finished)
  int b, sgn;
  if (!resolve_output(out, words, capacity, n, b, sgn)) return;
  if (b_spec < 0 || (b_spec && b == b_spec)) return;  // k_pack_local wrote every tile at b
  const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  uint32_t* buf = s_buf[warp];
  const uint64_t dw = data_words(n, b);
  const uint32_t mask = b >= 32 ? 0xffffffffu : ((1u << b) - 1u);
  const uint64_t ntiles = (n + kTile - 1) / kTile;
  const uint64_t gwarps = (uint64_t)gridDim.x * kWarps;
  for (uint64_t t0 = (uint64_t)blockIdx.x * kWarps + warp; t0 < ntiles; t0 += K * gwarps) {
    int tw[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint64_t t = t0 + k * gwarps;
      tw[k] = t < ntiles ? (int)tile_width[t] : 0;
    }
    uint4 r[K][Q];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint64_t t = t0 + k * gwarps;
      const int bl = tw[k] & 0x7f;
      const uint4* src = reinterpret_cast<const uint4*>(slots + t * (uint64_t)slot_words);
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const int q = lane + 32 * j;
        // (a tile wider than BMAX, width byte 0xFF, is never read)
        r[k][j] = (t < ntiles && bl <= BMAX && q < 8 * bl) ? __ldg(src + q) : make_uint4(0, 0, 0, 0);
      }
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const uint64_t t = t0 + k * gwarps;
      const int bl = tw[k] & 0x7f;
      if (t >= ntiles || bl > BMAX) continue;
      if (bl == b && t * (uint64_t)(32 * b) + 32 * b <= dw) {
        // the tile is already at the matrix width: its bits are final (a value
        // that fits b bits has the same low b bits signed or unsigned)
        uint4* dst = reinterpret_cast<uint4*>(words + t * (uint64_t)(32 * b));
#pragma unroll
        for (int j = 0; j < Q; ++j)
          if (lane + 32 * j < 8 * b) dst[lane + 32 * j] = r[k][j];
        continue;
      }
      uint32_t* area = buf + k * kArea;
#pragma unroll
      for (int j = 0; j < Q; ++j) {
        const int q = lane + 32 * j;
        if (q < 8 * bl) {
          const int w = 4 * q;
          area[stage_pos(w, bl)] = r[k][j].x;
          area[stage_pos(w + 1, bl)] = r[k][j].y;
          area[stage_pos(w + 2, bl)] = r[k][j].z;
          area[stage_pos(w + 3, bl)] = r[k][j].w;
        }
      }
    }
    __syncwarp();
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      const uint64_t t = t0 + k * gwarps;
      const int twk = (int)tile_width[t < ntiles ? t : 0];  // (L1: read above)
      const int bl = twk & 0x7f, sl = twk >> 7;
      if (t >= ntiles || bl > BMAX) continue;
      if (bl == b && t * (uint64_t)(32 * b) + 32 * b <= dw) continue;  // copied above
      uint32_t* area = buf + k * kArea;
      uint32_t u[32];
      decode_dispatch<BMAX>(bl, sl, area, lane,
                            [&](int f, int64_t x) { u[f] = (uint32_t)x & mask; });
      __syncwarp();
      encode_dispatch<BMAX>(b, u, area, lane);
      __syncwarp();
      store_packed(area, words, t, b, dw, lane);
    }
    __syncwarp();
  }
}

// Workspace of the single-pass forms: one slot of 32*cls words per tile (cls
// the output's width class), then one width byte per tile.
inline size_t pack_ws_bytes(uint64_t n, int cls) {
  const uint64_t ntiles = (n + kTile - 1) / kTile;
  return ((ntiles * 32 * cls * 4 + 255) & ~(size_t)255) + ((ntiles + 255) & ~(size_t)255);
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
enum class EwKind {
  PackI64, PackI32, AddStats, AddSpec, AddPack, ScaleStats, ScaleSpec, ScalePack, UnpackI64,
  UnpackI32, LocalI64, LocalI32, Repack
};

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
  void* ws;               // Local* / Repack: workspace (slots, then tile widths)
  int slot_class;         // Local* / Repack: width class of the output (slot = 32*class words)
  int spec;               // AddPack / ScalePack: an AddSpec / ScaleSpec launch came first;
                          // LocalI64 / LocalI32 / Repack: the speculative width (0: none)
  int pdl;                // LocalI64 / LocalI32: launched with programmatic dependent launch
};

inline int ew_grid(uint64_t n, int per_sm) {
  uint64_t tiles = (n + kTile - 1) / kTile;
  uint64_t want = (tiles + kWarps - 1) / kWarps;
  return (int)umin(umax(want, 1), (uint64_t)num_sms() * per_sm);
}

// Launchers of one width class C, one per family of EwKind (each family is
// instantiated in a translation unit of its own so that they compile in
// parallel).  Each returns the number of kernels launched.  Grids are
// persistent-style: every warp keeps walking tiles (and prefetching).

// AddStats / AddSpec / AddPack
template <int C>
int launch_ew_add(const EwCall& c, cudaStream_t st) {
  int launched = 1;
  const uint64_t n = c.rows * c.cols;
  PackedIn a{c.ha, c.wa, 0, 0, 0}, b{c.hb, c.wb, 0, 0, 0};
  const int g = ew_grid(n, 8);
  const OpAdd op{a, b};
  if (c.kind == EwKind::AddStats)
    k_ew<OpAdd, C, kStats><<<g, kThreads, 0, st>>>(op, c.out, nullptr, 0, n, 0);
  else if (c.kind == EwKind::AddSpec) {
    launch_lanes_add(op, c.out, c.words, c.capacity, n, C, st);
    launched = 2;
    // the passes after the lane pass usually return at once: launched early
    // (programmatic dependent launch) so that their launch overlaps it
    ax::launch_pdl(k_ew<OpAdd, C, kSpec>, dim3(g), dim3(kThreads), 0, st, op, c.out, c.words,
                   c.capacity, n, 0);
  } else {
    ax::launch_pdl(k_ew<OpAdd, C, kPack>, dim3(g), dim3(kThreads), 0, st, op, c.out, c.words,
                   c.capacity, n, c.spec);
  }
  return launched;
}

// ScaleStats / ScaleSpec / ScalePack; SMALL: |s| < 2^15 (OpScale<SMALL>)
template <int C, bool SMALL>
int launch_ew_scale(const EwCall& c, cudaStream_t st) {
  int launched = 1;
  const uint64_t n = c.rows * c.cols;
  const OpScale<SMALL> op{PackedIn{c.ha, c.wa, 0, 0, 0}, c.s};
  const int g = ew_grid(n, 8);
  if (c.kind == EwKind::ScaleStats) {
    k_ew<OpScale<SMALL>, C, kStats><<<g, kThreads, 0, st>>>(op, c.out, nullptr, 0, n, 0);
  } else if (c.kind == EwKind::ScaleSpec) {
    if constexpr (SMALL) {
      if (c.s != 0 && c.s > -32 && c.s < 32) {  // (the lane pass needs 1 <= |s| < 2^5)
        launch_lanes_scale(op, c.out, c.words, c.capacity, n, C, st);
        launched = 2;
      }
    }
    ax::launch_pdl(k_ew<OpScale<SMALL>, C, kSpec>, dim3(g), dim3(kThreads), 0, st, op, c.out,
                   c.words, c.capacity, n, 0);
  } else {
    ax::launch_pdl(k_ew<OpScale<SMALL>, C, kPack>, dim3(g), dim3(kThreads), 0, st, op, c.out,
                   c.words, c.capacity, n, c.spec);
  }
  return launched;
}

// PackI64 / PackI32 / LocalI64 / LocalI32 / Repack / UnpackI64 / UnpackI32
template <int C>
int launch_ew_pack(const EwCall& c, cudaStream_t st) {
  const uint64_t n = c.rows * c.cols;
  switch (c.kind) {
    case EwKind::PackI64:
      k_pack_dense<int64_t, C><<<ew_grid(n, 12), kThreads, 0, st>>>(
          (const int64_t*)c.dense, c.out, c.words, c.capacity, n);
      break;
    case EwKind::PackI32:
      k_pack_dense<int32_t, C><<<ew_grid(n, 12), kThreads, 0, st>>>(
          (const int32_t*)c.dense, c.out, c.words, c.capacity, n);
      break;
    case EwKind::LocalI64:
    case EwKind::LocalI32:
    case EwKind::Repack: {
      const uint64_t ntiles = (n + kTile - 1) / kTile;
      const int sc = c.slot_class;
      const uint32_t slot_words = (uint32_t)(32 * sc);
      // (no workspace: the exact-width form, spec < 0, which needs neither)
      uint32_t* slots = (uint32_t*)c.ws;
      uint8_t* widths =
          c.ws ? (uint8_t*)c.ws + ((ntiles * 32 * sc * 4 + 255) & ~(size_t)255) : nullptr;
      const int gl = ew_grid(n, 12);
      if (c.kind == EwKind::LocalI64) {
        const size_t smem = (size_t)kWarps * 2 * 2 * kDensePad * sizeof(uint32_t);
        static bool attr = false;
        if (!attr) {
          cudaFuncSetAttribute(k_pack_local<int64_t, C>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
          attr = true;
        }
        if (c.pdl)
          ax::launch_pdl(k_pack_local<int64_t, C>, dim3(gl), dim3(kThreads), smem, st,
                         (const int64_t*)c.dense, c.out, slots, slot_words, widths, n, c.words,
                         c.spec);
        else
          k_pack_local<int64_t, C><<<gl, kThreads, smem, st>>>((const int64_t*)c.dense, c.out,
                                                               slots, slot_words, widths, n,
                                                               c.words, c.spec);
      } else if (c.kind == EwKind::LocalI32) {
        const size_t smem = (size_t)kWarps * 2 * kDensePad32 * sizeof(uint32_t);
        if (c.pdl)
          ax::launch_pdl(k_pack_local<int32_t, C>, dim3(gl), dim3(kThreads), smem, st,
                         (const int32_t*)c.dense, c.out, slots, slot_words, widths, n, c.words,
                         c.spec);
        else
          k_pack_local<int32_t, C><<<gl, kThreads, smem, st>>>((const int32_t*)c.dense, c.out,
                                                               slots, slot_words, widths, n,
                                                               c.words, c.spec);
      } else {
        ax::launch_pdl(k_repack<C>, dim3(gl), dim3(kThreads), 0, st, (const uint32_t*)slots,
                       slot_words, (const uint8_t*)widths, c.out, c.words, c.capacity, n,
                       c.spec);
      }
      break;
    }
    case EwKind::UnpackI64:
      k_unpack_ge<int64_t, C><<<ew_grid(n, 12), kThreads, 0, st>>>(
          c.out, c.words, c.rows, c.cols, c.capacity, (int64_t*)c.dense, c.err);
      break;
    case EwKind::UnpackI32:
      k_unpack_ge<int32_t, C><<<ew_grid(n, 12), kThreads, 0, st>>>(
          c.out, c.words, c.rows, c.cols, c.capacity, (int32_t*)c.dense, c.err);
      break;
    default:
      return 0;
  }
  return 1;
}

extern template int launch_ew_add<8>(const EwCall&, cudaStream_t);
extern template int launch_ew_add<16>(const EwCall&, cudaStream_t);
extern template int launch_ew_add<32>(const EwCall&, cudaStream_t);
extern template int launch_ew_scale<8, true>(const EwCall&, cudaStream_t);
extern template int launch_ew_scale<16, true>(const EwCall&, cudaStream_t);
extern template int launch_ew_scale<32, true>(const EwCall&, cudaStream_t);
extern template int launch_ew_scale<8, false>(const EwCall&, cudaStream_t);
extern template int launch_ew_scale<16, false>(const EwCall&, cudaStream_t);
extern template int launch_ew_scale<32, false>(const EwCall&, cudaStream_t);
extern template int launch_ew_pack<8>(const EwCall&, cudaStream_t);
extern template int launch_ew_pack<16>(const EwCall&, cudaStream_t);
extern template int launch_ew_pack<32>(const EwCall&, cudaStream_t);

template <int C>
inline int launch_ew_class(const EwCall& c, cudaStream_t st) {
  switch (c.kind) {
    case EwKind::AddStats:
    case EwKind::AddSpec:
    case EwKind::AddPack: return launch_ew_add<C>(c, st);
    case EwKind::ScaleStats:
    case EwKind::ScaleSpec:
    case EwKind::ScalePack:
      return c.s > -32768 && c.s < 32768 ? launch_ew_scale<C, true>(c, st)
                                         : launch_ew_scale<C, false>(c, st);
    default: return launch_ew_pack<C>(c, st);
  }
}

}  // namespace ge
}  // namespace ccm
