// matvec_stream.cuh -- y = A x for row-aligned A (cols a multiple of 128)
// whose fields have at most 8 bits: the streaming kernel of ccm_matvec.
//
// One call is three launches chained by programmatic dependent launch, so
// each starts while the previous one finishes:
//   k_mv_init   validates A and x, clears y's header and the int64 y sums,
//               and decodes x once into the staging image in the workspace;
//   k_mv        streams A: before it waits for k_mv_init it has already
//               issued its first copies of A (A does not depend on it);
//   k_mv_ypack  y's width statistics and y packed at that width, by one CTA
//               (y of up to kYSmallRows rows; larger y use the pack engine).
//
// k_mv: the packed A is cut into warp-stages of up to 32 consecutive
// 128-field chunks of one row (a chunk is 16*b contiguous bytes, 16-byte
// aligned since cols % 128 == 0).  Warp w of the W warps of the grid takes the
// contiguous range [T w / W, T (w + 1) / W) of the T warp-stages.  Each warp
// owns a ring of D slots in shared memory; a slot receives one warp-stage
// through 1-D bulk copies of the asynchronous copy engine (one copy per
// chunk, landing at an odd multiple of 16 bytes per chunk so that the lanes'
// 16-byte shared loads are conflict-free), whose completion is counted in
// bytes on the slot's mbarrier.  While the warp decodes one slot, the copies
// of the next D - 1 are in flight.  Lane l decodes chunk l against its x
// (dp4a on byte lanes when b <= 8 and b_x <= 8, signed fields in offset
// binary corrected by the chunk's sum of x; int32 multiply-adds otherwise).
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
using mvf::pitch_bytes;

constexpr int kChunks = 32;     // chunks of a warp-stage (one per lane)
constexpr int kWarps = 8;       // warps of a CTA
constexpr int kMaxSlots = 6;    // ring slots of a warp
constexpr int kXPitch8 = 144;   // x image: 128 bytes + 16 pad per chunk
constexpr int kXPitch32 = 528;  // or 128 int32 + 16 pad
constexpr uint64_t kYSmallRows = 16384;

// Shared bytes of one ring slot for width b.
__host__ __device__ constexpr uint32_t slot_bytes(int b) { return kChunks * pitch_bytes(b); }

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
  const uint8_t* ximg;    // x image (written by k_mv_init)
  uint32_t ring_bytes;    // shared bytes of each warp's ring
  uint32_t x_offset;      // shared offset of the x image (after the rings)
  uint32_t x_bytes;       // its size, a multiple of 16
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

template <int B, bool SGN, bool DP, bool XS, bool NARROW>
__device__ __noinline__ void body(const Args& a, uint8_t* smem, uint64_t* bars) {
  constexpr int P = pitch_bytes(B);
  constexpr uint32_t SB = slot_bytes(B);
  constexpr uint32_t CB = 16 * B;  // bytes of one chunk
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t D = umin(kMaxSlots, a.ring_bytes / SB);
  uint8_t* ring = smem + warp * a.ring_bytes;
  uint64_t* bar = bars + warp * kMaxSlots;
  uint8_t* xb = smem + a.x_offset;
  const uint32_t nchunks = (uint32_t)(a.n / kKC);
  const int* csum = reinterpret_cast<const int*>(xb + (uint64_t)nchunks * (DP ? kXPitch8 : kXPitch32));
  const uint32_t S = (nchunks + kChunks - 1) / kChunks;  // warp-stages per row
  const uint64_t T = a.m * S;
  const uint64_t GW = (uint64_t)gridDim.x * kWarps, gw = (uint64_t)blockIdx.x * kWarps + warp;
  const uint64_t t0 = T / GW * gw + umin(gw, T % GW);
  const uint64_t count = T / GW + (gw < T % GW ? 1 : 0);
  const uint64_t row_bytes = a.n / 8 * B;
  const uint8_t* A = reinterpret_cast<const uint8_t*>(a.wa);

  if (lane == 0) {
    for (uint32_t s = 0; s < D; ++s) ax::mbar_init(&bar[s], 1);
    ax::mbar_init_fence();
  }
  __syncwarp();

  // producer position (row, stage of the row) of the next stage to copy
  uint64_t prow = t0 / S;
  uint32_t pseg = (uint32_t)(t0 % S);
  auto issue = [&](uint32_t slot) {
    const uint32_t ch = umin(kChunks, nchunks - pseg * kChunks);
    if (lane == 0) ax::mbar_expect_tx(&bar[slot], ch * CB);
    __syncwarp();
    if ((uint32_t)lane < ch)
      ax::bulk_g2s(ring + slot * SB + lane * P,
                   A + prow * row_bytes + (uint64_t)pseg * (kChunks * CB) + lane * CB, CB,
                   &bar[slot]);
    if (++pseg == S) pseg = 0, ++prow;
  };

  // the first stages of A in flight before anything else
  const uint64_t pre = umin(count, D);
  for (uint32_t k = 0; k < (uint32_t)pre; ++k) issue(k);

  // x image (written by k_mv_init): wait for that kernel, then copy it
  ax::grid_dep_wait();
  __shared__ uint64_t xbar;
  __shared__ int s_fail;
  if (threadIdx.x == 0) {
    s_fail = 0;
    ax::mbar_init(&xbar, 1);
    ax::mbar_init_fence();
    ax::mbar_expect_tx(&xbar, a.x_bytes);
    for (uint32_t o = 0; o < a.x_bytes; o += 32768)
      ax::bulk_g2s(xb + o, a.ximg + o, umin(32768, a.x_bytes - o), &xbar);
  }
  __syncthreads();
  if (!ax::mbar_wait(&xbar, 0)) s_fail = 1;
  __syncthreads();
  ax::grid_dep_launch();  // the y epilogue may launch now
  bool ok = s_fail == 0 && a.out->status == CCM_OK;

  long long acc = 0;
  uint64_t row = t0 / S;
  uint32_t seg = (uint32_t)(t0 % S);
  uint64_t k = 0;
  for (; ok && k < count; ++k) {
    const uint32_t slot = (uint32_t)(k % D);
    if (!ax::mbar_wait(&bar[slot], (uint32_t)((k / D) & 1))) {
      ok = false;
      break;
    }
    const uint32_t ch = umin(kChunks, nchunks - seg * kChunks);
    if ((uint32_t)lane < ch) {
      const uint32_t c = seg * kChunks + lane;
      const uint8_t* rp = ring + slot * SB + lane * P;
      if constexpr (DP) {
        acc += mvf::dp4a_stage<B, SGN, XS>(rp, reinterpret_cast<const int*>(xb + c * kXPitch8));
        if constexpr (SGN) acc -= (long long)csum[c] * (1ll << (B - 1));
      } else {
        mvf::decode_mac<B, SGN, NARROW>(rp, reinterpret_cast<const int*>(xb + c * kXPitch32), acc);
      }
    }
    __syncwarp();
    if (k + D < count) {
      ax::fence_proxy_async_smem();  // this slot's reads before its refill
      issue(slot);
    }
    if (++seg == S || k + 1 == count) {  // leaving the row (or the range)
      flush_row(acc, a.y, row, lane);
      seg = 0;
      ++row;
    }
  }
  if (k < count) {
    // stopped early (a failed wait or an error): let the copies still in
    // flight land before the CTA's shared memory goes away
    const uint64_t issued = umin(count, k + D);
    for (uint64_t j = k; j < issued; ++j)
      if (!ax::mbar_wait(&bar[j % D], (uint32_t)((j / D) & 1))) break;
    if (lane == 0 && a.out->status == CCM_OK) set_status(a.out, CCM_E_TIMEOUT);
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

template <bool NARROW>
__global__ void __launch_bounds__(kWarps * 32, 3) k_mv(Args a) {
  extern __shared__ __align__(128) uint8_t smem[];
  __shared__ uint64_t bars[kWarps * kMaxSlots];
  // A and x are checked here as well (k_mv_init may not have run yet): no
  // word is read unless both headers describe buffers of the sizes given
  int st = check_input(a.ha, a.m, a.n, a.a_cap);
  if (st == CCM_OK) st = check_input(a.hx, a.n, 1, a.x_cap);
  const int b = a.ha->width, sgn = a.ha->is_signed;
  const int bx = a.hx->width, sx = a.hx->is_signed;
  if (st != CCM_OK || !stream_ok(b, bx, a.n)) {
    ax::grid_dep_wait();  // k_mv_init reports input errors into y's header
    if (st == CCM_OK && threadIdx.x == 0 && blockIdx.x == 0) set_status(a.out, CCM_E_INPUT);
    return;
  }
  if (b <= 8 && bx <= 8) {
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
