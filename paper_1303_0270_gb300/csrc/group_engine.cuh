// group_engine.cuh -- lane-per-group decode / encode of SM bit streams.
//
// 32 consecutive fields of a width-b stream occupy exactly b whole words and
// start on a word boundary (Methods, Method 1: fields laid end to end from
// the least significant bit).  A warp therefore works on a tile of 1024
// fields = 32 groups = 32*b words: the tile is staged through shared memory
// with coalesced loads, and lane t decodes (or encodes) group t -- its 32
// fields -- entirely in registers, with every shift fixed at compile time.
// The width is only known on the GPU (it lives in the matrix header), so the
// kernels dispatch on it at run time over template instances up to a width
// class BMAX that the host derives from the buffer capacities.
//
// Shared-memory staging layout of the words of a tile: word W at W for odd b
// (lane t then reads words t*b + k: distinct banks), W + W/32 for even b (one
// pad word per 32, which keeps those reads at most 2-way conflicted).
#pragma once

#include "ccm_device.cuh"

namespace ccm {
namespace ge {

constexpr int kWarps = 4;                    // warps per CTA
constexpr int kThreads = kWarps * kWarp;
constexpr int kTile = 1024;                  // fields per warp tile
constexpr int kBufWords = 2 * (kTile + 32);  // an int64 tile with a pad per 32 fields

__device__ __forceinline__ int stage_pos(int w, int b) { return (b & 1) ? w : w + (w >> 5); }

// Copies the words of tile `tile` of a packed stream (width b, `dw` data
// words in total) into `buf`; words past the end read as zero.
__device__ __forceinline__ void stage_packed(uint32_t* buf, const uint32_t* __restrict__ words,
                                             uint64_t tile, int b, uint64_t dw, int lane) {
  const uint64_t w0 = tile * (uint64_t)(32 * b);
  const int tw = 32 * b;
  const uint64_t avail = dw > w0 ? dw - w0 : 0;
  if (avail >= (uint64_t)tw && (w0 & 3) == 0) {
    // whole tile: 16-byte loads (the tile starts at byte 128*b*tile)
    const uint4* src = reinterpret_cast<const uint4*>(words + w0);
    // all of the lane's 16-byte loads (at most 8: b <= 32) before any store
    uint4 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int q = lane + 32 * j;
      if (q < tw / 4) v[j] = __ldg(src + q);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int q = lane + 32 * j;
      if (q < tw / 4) {
        const int w = 4 * q;
        buf[stage_pos(w, b)] = v[j].x;
        buf[stage_pos(w + 1, b)] = v[j].y;
        buf[stage_pos(w + 2, b)] = v[j].z;
        buf[stage_pos(w + 3, b)] = v[j].w;
      }
    }
  } else {
    for (int w = lane; w < tw; w += 32)
      buf[stage_pos(w, b)] = (uint64_t)w < avail ? __ldg(words + w0 + w) : 0u;
  }
}

// Stores `count` staged words of a tile (output width b) to global memory.
__device__ __forceinline__ void store_packed(const uint32_t* buf, uint32_t* __restrict__ words,
                                             uint64_t tile, int b, uint64_t dw, int lane) {
  const uint64_t w0 = tile * (uint64_t)(32 * b);
  const int tw = (int)umin((uint64_t)(32 * b), dw > w0 ? dw - w0 : 0);
  if (tw == 32 * b && (w0 & 3) == 0) {
    uint4* dst = reinterpret_cast<uint4*>(words + w0);
    for (int q = lane; q < tw / 4; q += 32) {
      int w = 4 * q;
      dst[q] = make_uint4(buf[stage_pos(w, b)], buf[stage_pos(w + 1, b)], buf[stage_pos(w + 2, b)],
                          buf[stage_pos(w + 3, b)]);
    }
  } else {
    for (int w = lane; w < tw; w += 32) words[w0 + w] = buf[stage_pos(w, b)];
  }
}

// Dense tiles: element f of the tile at f + f/32 (64-bit or 32-bit slots).
template <typename T>
__device__ __forceinline__ void stage_dense(T* buf, const T* __restrict__ src, uint64_t base,
                                            uint32_t nt, int lane) {
#pragma unroll 8
  for (int j = 0; j < 32; ++j) {
    uint32_t f = lane + 32 * j;
    buf[f + (f >> 5)] = f < nt ? __ldg(src + base + f) : (T)0;
  }
}

template <typename T>
__device__ __forceinline__ void store_dense(const T* buf, T* __restrict__ dst, uint64_t base,
                                            uint32_t nt, int lane) {
#pragma unroll 8
  for (int j = 0; j < 32; ++j) {
    uint32_t f = lane + 32 * j;
    if (f < nt) dst[base + f] = buf[f + (f >> 5)];
  }
}

// ---------------------------------------------------------------------------
// Compile-time width: decode the lane's group (32 fields of width B) and hand
// each value to fn(k, value) with k a compile-time index.
// ---------------------------------------------------------------------------
template <int B, bool SGN, class F>
__device__ __forceinline__ void decode_group(const uint32_t* buf, int lane, F&& fn) {
  uint32_t w[B + 1];
#pragma unroll
  for (int j = 0; j < B; ++j) w[j] = buf[stage_pos(lane * B + j, B)];
  w[B] = 0;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const int bit = k * B, wi = bit >> 5, s = bit & 31;
    uint32_t t = (s + B <= 32) ? (w[wi] >> s) : __funnelshift_r(w[wi], w[wi + 1], s);
    int64_t v;
    if constexpr (B == 32) {
      v = SGN ? (int64_t)(int32_t)t : (int64_t)t;
    } else if constexpr (SGN) {
      v = (int64_t)((int32_t)(t << (32 - B)) >> (32 - B));
    } else {
      v = (int64_t)(t & ((1u << B) - 1u));
    }
    fn(k, v);
  }
}

// Encode 32 values (already reduced to their low B bits) into the lane's
// B words of the staging buffer.
template <int B>
__device__ __forceinline__ void encode_group(const uint32_t (&u)[32], uint32_t* buf, int lane) {
  uint32_t w[B];
#pragma unroll
  for (int j = 0; j < B; ++j) w[j] = 0;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const int bit = k * B, wi = bit >> 5, s = bit & 31;
    w[wi] |= u[k] << s;
    if (s + B > 32) w[wi + 1] |= u[k] >> (32 - s);
  }
#pragma unroll
  for (int j = 0; j < B; ++j) buf[stage_pos(lane * B + j, B)] = w[j];
}

// Run-time dispatch over the instances up to BMAX: one switch (a jump table)
// on 2*b + sign.
#define CCM_GE_CASES_8(M) M(1) M(2) M(3) M(4) M(5) M(6) M(7) M(8)
#define CCM_GE_CASES_16(M) CCM_GE_CASES_8(M) M(9) M(10) M(11) M(12) M(13) M(14) M(15) M(16)
#define CCM_GE_CASES_32(M)                                                                     \
  CCM_GE_CASES_16(M) M(17) M(18) M(19) M(20) M(21) M(22) M(23) M(24) M(25) M(26) M(27) M(28) \
  M(29) M(30) M(31) M(32)

template <int BMAX, class F>
__device__ __forceinline__ void decode_dispatch(int b, int sgn, const uint32_t* buf, int lane,
                                                F&& fn) {
#define CCM_GE_DEC(B)                                            \
  case 2 * B:                                                    \
    if constexpr (B <= BMAX) decode_group<B, false>(buf, lane, fn); \
    break;                                                       \
  case 2 * B + 1:                                                \
    if constexpr (B <= BMAX) decode_group<B, true>(buf, lane, fn);  \
    break;
  switch (2 * b + sgn) {
    CCM_GE_CASES_32(CCM_GE_DEC)
    default: break;
  }
#undef CCM_GE_DEC
}

template <int BMAX>
__device__ __forceinline__ void encode_dispatch(int b, const uint32_t (&u)[32], uint32_t* buf,
                                                int lane) {
#define CCM_GE_ENC(B)                                     \
  case B:                                                 \
    if constexpr (B <= BMAX) encode_group<B>(u, buf, lane); \
    break;
  switch (b) {
    CCM_GE_CASES_32(CCM_GE_ENC)
    default: break;
  }
#undef CCM_GE_ENC
}

}  // namespace ge
}  // namespace ccm
