// matvec_stream.cuh -- y = A x for row-aligned A (cols a multiple of 128)
// whose fields have at most 8 bits: the streaming kernel of ccm_matvec.
//
// One call is three launches chained by programmatic dependent launch, so
// each starts while the previous one finishes:
//   k_mv_init   validates A and x, clears y's header and the int64 y sums,
//               and decodes x once into an image in the workspace;
//   k_mv        streams A: it issues its first copies of A before it waits
//               for k_mv_init (A does not depend on it);
//   k_mv_ypack  y's width statistics and y packed at that width, by one CTA
//               (y of up to kYSmallRows rows; larger y use the pack engine).
//
// k_mv: the packed A is cut into warp-stages of up to 32 consecutive
// 128-field chunks of one row (a chunk is 16*b contiguous bytes, 16-byte
// aligned since cols % 128 == 0).  Warp w of the W warps of the grid takes the
// contiguous range [T w / W, T (w + 1) / W) of the T warp-stages.  Each warp
// owns a ring of D slots in shared memory; a slot receives one warp-stage
// (512*b contiguous bytes) through one 1-D bulk copy of the asynchronous copy
// engine, whose completion is counted in bytes on the slot's mbarrier.  While
// the warp decodes one slot, the copies of the next D - 1 are in flight.
// Chunks sit 16*b bytes apart in the slot: for odd b the lanes' 16-byte
// shared loads are then conflict-free as they are; for b = 2, 4, 8 (fields
// that never straddle a byte) lane l reads its b vectors starting at vector
// (l*b/8) mod b, which spreads any eight consecutive lanes over all banks (the
// products are summed, so the order is free).  Lane l decodes chunk l against its x
// (dp4a on byte lanes when b <= 8 and b_x <= 8, signed fields in offset
// binary corrected by the chunk's sum of x; int32 multiply-adds otherwise),
// reading x from the image in global memory (L1-cached: a few KB per chunk
// row shared by every warp of the SM).
// A row's partial sums are reduced across the warp and added to y when the
// warp leaves the row (atomically: a row may be split between two warps).
// Every wait is bounded: a wait that gives up records CCM_E_TIMEOUT in y's
// header, and the warp drains its copies in flight before it exits.
#pragma once

#include "async_copy.cuh"
#include "ccm_device.cuh"
#include "matvec_fast.cuh"

namespace ccm {
namespace mvs {

using mvf::kKC;

constexpr int kChunks = 32;     // chunks of a warp-stage (one per lane)
constexpr int kWarps = 8;       // warps of a CTA
constexpr int kMaxSlots = 6;    // ring slots of a warp
constexpr uint64_t kYSmallRows = 16384;

// Shared bytes of one ring slot (one warp-stage, chunks back to back) for width b.
__host__ __device__ constexpr uint32_t slot_bytes(int b) { return kChunks * 16u * (uint32_t)b; }

constexpr int kXPitch8 = 144;   // x image: 128 bytes + 16 pad per chunk
constexpr int kXPitch32 = 528;  // or 128 int32 + 16 pad

// Bytes of the x image (x rows plus the per-chunk sums of x).
__host__ __device__ constexpr uint64_t x_image_bytes(uint64_t n, bool bytes) {
  return n / kKC * ((bytes ? kXPitch8 : kXPitch32) + 4);
}

struct Args {
  ccm_header* out;  // y header
  const ccm_header* ha;
  const uint32_t* wa;
  uint64_t a_cap;
  const ccm_header* hx;
  const uint32_t* wx;
  uint64_t x_cap;
  uint64_t m, n;
  int64_t* y;             // int64 sums (cleared by k_mv_init)
  uint8_t* ximg;          // x image (written by k_mv_init)
  uint32_t ring_bytes;    // shared bytes of each warp's ring
  int dp;                 // 1: byte-lane path (x image in bytes; the capacities bound b_x by 8)
};

// The width conditions of this kernel, read from the (valid) headers.
__device__ __forceinline__ bool stream_ok(int b, int bx, uint64_t n) {
  return b <= 8 && bx <= 31 && b + bx + bitlen64(n) <= 63;
}

__device__ __forceinline__ void flush_row(long long& acc, int64_t* y, uint64_t row, int lane) {
  for (int d = 16; d; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if (lane == 0 && acc != 0)
    atomicAdd(reinterpret_cast<unsigned long long*>(y + row), (unsigned long long)acc);
  acc = 0;
}


// Widths whose chunks are read in the rotated vector order.
__host__ __device__ constexpr bool rotated(int B) { return B == 2 || B == 4 || B == 8; }

// First vector a lane reads (B = 2, 4, 8): eight consecutive lanes then hit
// the eight 16-byte bank groups once each.
template <int B>
__device__ __forceinline__ int first_vector(int lane) {
  return ((lane * B) >> 3) & (B - 1);
}

// sum over the 128 fields of a chunk of u_j * x_j (u the unsigned or
// offset-binary field, x bytes in dp4a order), B in {2, 4, 8}: vector v (four
// words, 128/B fields) pairs with x int4 words [R v, R v + R), R = 8/B, the
// same pairing as mvf::dp4a_stage.
template <int B, bool SGN, bool XS>
__device__ __forceinline__ int dp4a_rot(const uint8_t* chunk, const int* __restrict__ xw,
                                        int lane) {
  constexpr int R = 8 / B;
  constexpr uint32_t m = mvf::low_bits(B) * 0x01010101u;
  constexpr uint32_t sign = mvf::low_bits(32) / mvf::low_bits(B) << (B - 1);  // top bit of each field
  const uint4* cv = reinterpret_cast<const uint4*>(chunk);
  const int4* xv = reinterpret_cast<const int4*>(xw);
  const int r = first_vector<B>(lane);
  int acc[4] = {0, 0, 0, 0};
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const int v = (i + r) & (B - 1);
    const uint4 q = cv[v];
    uint32_t w[4] = {q.x, q.y, q.z, q.w};
    if constexpr (SGN) {
#pragma unroll
      for (int j = 0; j < 4; ++j) w[j] ^= sign;
    }
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int4 xq = xv[R * v + t];
      const int xa[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = 4 * t + u, j = e / R, k = e % R;
        const uint32_t val = B == 8 ? w[j] : (w[j] >> (B * k)) & m;
        acc[u] = mvf::dp4a_u<XS>(val, xa[u], acc[u]);
      }
    }
  }
  return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// acc += sum over the 128 fields of a chunk of a_j * x_j with x int32, B in
// {2, 4, 8}, vectors in the rotated order (vector v holds fields
// [v 128/B, (v + 1) 128/B)).
template <int B, bool SGN>
__device__ __forceinline__ void mac_rot(const uint8_t* chunk, const int* __restrict__ xs,
                                        long long& acc, int lane) {
  constexpr int F = 128 / B;  // fields per vector
  const uint4* cv = reinterpret_cast<const uint4*>(chunk);
  const int4* xv = reinterpret_cast<const int4*>(xs);
  const int r = first_vector<B>(lane);
#pragma unroll
  for (int i = 0; i < B; ++i) {
    const int v = (i + r) & (B - 1);
    const uint4 q = cv[v];
    const uint32_t w[4] = {q.x, q.y, q.z, q.w};
    long long part = 0;
#pragma unroll
    for (int f4 = 0; f4 < F / 4; ++f4) {
      const int4 xq = xv[(F / 4) * v + f4];
      const int xa[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int f = 4 * f4 + u, bit = f * B, wi = bit >> 5, sh = bit & 31;
        const uint32_t t = w[wi] >> sh;
        int val;
        if constexpr (SGN)
          val = (int)(t << (32 - B)) >> (32 - B);
        else
          val = (int)(t & mvf::low_bits(B));
        part += (long long)val * xa[u];
      }
    }
    acc += part;
  }
}

template <int B, bool SGN, bool DP, bool XS, bool NARROW>
__device__ __forceinline__ void body(const Args& a, uint8_t* smem, uint64_t* bars) {
  constexpr uint32_t CB = 16 * B;        // bytes of one chunk
  constexpr uint32_t SB = kChunks * CB;  // bytes of one slot
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t D = umin(kMaxSlots, a.ring_bytes / SB);
  uint8_t* ring = smem + warp * a.ring_bytes;
  uint64_t* bar = bars + warp * kMaxSlots;
  const uint32_t nchunks = (uint32_t)(a.n / kKC);
  const uint8_t* xg = a.ximg;  // x image (global memory, L1-cached reads)
  const int* csum = reinterpret_cast<const int*>(xg + (uint64_t)nchunks * (DP ? kXPitch8 : kXPitch32));
  const uint32_t S = (nchunks + kChunks - 1) / kChunks;  // warp-stages per row
  const uint64_t T = a.m * S;
  const uint64_t GW = (uint64_t)gridDim.x * kWarps, gw = (uint64_t)blockIdx.x * kWarps + warp;
  const uint64_t t0 = T / GW * gw + umin(gw, T % GW);
  const uint64_t count = T / GW + (gw < T % GW ? 1 : 0);
  const uint64_t row_bytes = a.n / 8 * B;
  const uint8_t* A = reinterpret_cast<const uint8_t*>(a.wa);
  // row sums of the byte-lane path fit int32 when n <= 16384 (|u x| < 2^16)
  const bool sum32 = DP && a.n <= 16384;

  if (lane == 0) {
    for (uint32_t s = 0; s < D; ++s) ax::mbar_init(&bar[s], 1);
    ax::mbar_init_fence();
  }
  __syncwarp();

  // producer position (row, stage of the row) and slot of the next copy
  uint64_t prow = t0 / S;
  uint32_t pseg = (uint32_t)(t0 % S), pslot = 0;
  auto issue = [&]() {
    const uint32_t ch = umin(kChunks, nchunks - pseg * kChunks);
    if (lane == 0) {
      ax::mbar_expect_tx(&bar[pslot], ch * CB);
      ax::bulk_g2s(ring + pslot * SB, A + prow * row_bytes + (uint64_t)pseg * SB, ch * CB,
                   &bar[pslot]);
    }
    if (++pseg == S) pseg = 0, ++prow;
    if (++pslot == D) pslot = 0;
  };

  // the first stages of A in flight before waiting for k_mv_init (which
  // writes the x image and clears y)
  const uint64_t pre = umin(count, D);
  for (uint64_t k = 0; k < pre; ++k) issue();
  ax::grid_dep_wait();
  ax::grid_dep_launch();  // the y epilogue may launch now

  long long acc = 0;
  int acc32 = 0;
  uint64_t row = t0 / S;
  uint32_t seg = (uint32_t)(t0 % S), slot = 0, phase = 0;
  uint64_t k = 0;
  for (; k < count; ++k) {
    if (!ax::mbar_wait(&bar[slot], phase)) break;
    const uint32_t ch = umin(kChunks, nchunks - seg * kChunks);
    if ((uint32_t)lane < ch) {
      const uint32_t c = seg * kChunks + lane;
      const uint8_t* rp = ring + slot * SB + lane * CB;
      if constexpr (DP) {
        const int* xw = reinterpret_cast<const int*>(xg + c * kXPitch8);
        int part;
        if constexpr (rotated(B))
          part = dp4a_rot<B, SGN, XS>(rp, xw, lane);
        else
          part = mvf::dp4a_stage<B, SGN, XS>(rp, xw);
        if constexpr (SGN) part -= __ldg(csum + c) * (1 << (B - 1));
        if (sum32)
          acc32 += part;
        else
          acc += part;
      } else {
        const int* xi = reinterpret_cast<const int*>(xg + c * kXPitch32);
        if constexpr (rotated(B))
          mac_rot<B, SGN>(rp, xi, acc, lane);
        else
          mvf::decode_mac<B, SGN, NARROW>(rp, xi, acc);
      }
    }
    __syncwarp();
    if (k + D < count) {
      ax::fence_proxy_async_smem();  // this slot's reads before its refill
      issue();
    }
    if (++slot == D) slot = 0, phase ^= 1;
    if (++seg == S || k + 1 == count) {  // leaving the row (or the range)
      if (sum32) {
        const int r = __reduce_add_sync(0xffffffffu, acc32);
        if (lane == 0 && r != 0)
          atomicAdd(reinterpret_cast<unsigned long long*>(a.y + row),
                    (unsigned long long)(long long)r);
        acc32 = 0;
      } else {
        flush_row(acc, a.y, row, lane);
      }
      seg = 0;
      ++row;
    }
  }
  if (k < count) {
    // a wait gave up: let the copies still in flight land before the CTA's
    // shared memory goes away, and report the timeout
    const uint64_t issued = umin(count, k + D);
    for (uint64_t j = k; j < issued; ++j) {
      if (!ax::mbar_wait(&bar[slot], phase)) break;
      if (++slot == D) slot = 0, phase ^= 1;
    }
    if (lane == 0) set_status(a.out, CCM_E_TIMEOUT);
  }
}

template <bool NARROW, bool DP, bool XS, int B = 1>
__device__ __forceinline__ void dispatch(const Args& a, int b, int sgn, uint8_t* smem,
                                         uint64_t* bars) {
  if constexpr (B <= 8) {
    if (b == B) {
      if (sgn)
        body<B, true, DP, XS, NARROW>(a, smem, bars);
      else
        body<B, false, DP, XS, NARROW>(a, smem, bars);
      return;
    }
    dispatch<NARROW, DP, XS, B + 1>(a, b, sgn, smem, bars);
  }
}

// One kernel per path so that each gets its own register budget: DP = byte
// lanes (the x capacity bounds b_x by 8; the x image holds bytes), else int32
// x (any b_x <= 31, x image of int32).
template <bool DP, bool NARROW>
__global__ void __launch_bounds__(kWarps * 32, DP ? 3 : 2) k_mv(const __grid_constant__ Args a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bars[kWarps * kMaxSlots];
  // A and x are checked here as well (k_mv_init may not have run yet): no
  // word is read unless both headers describe buffers of the sizes given
  const HeaderView ha = load_header(a.ha), hx = load_header(a.hx);  // both loads in flight
  int st = check_header(ha, a.m, a.n, a.a_cap);
  if (st == CCM_OK) st = check_header(hx, a.n, 1, a.x_cap);
  const int b = ha.width, sgn = ha.is_signed;
  const int bx = hx.width, sx = hx.is_signed;
  if (st != CCM_OK || !stream_ok(b, bx, a.n) || (DP && bx > 8)) {
    ax::grid_dep_wait();  // k_mv_init reports input errors into y's header
    if (st == CCM_OK && threadIdx.x == 0 && blockIdx.x == 0) set_status(a.out, CCM_E_INPUT);
    return;
  }
  if constexpr (DP) {
    if (sx)
      dispatch<NARROW, true, true>(a, b, sgn, smem, bars);
    else
      dispatch<NARROW, true, false>(a, b, sgn, smem, bars);
  } else {
    dispatch<NARROW, false, true>(a, b, sgn, smem, bars);
  }
}

}  // namespace mvs
}  // namespace ccm
