// pack_engine.cuh -- width selection and SM packing of any stream of int64
// values produced on the fly (dense input, the sum of two packed inputs, a
// scaled packed input, a result held in scratch).
//
// Every result is packed in two launches on the same stream:
//   k_stats  -- one pass over the produced values: OR of folded values and
//               the any-negative flag, reduced per block and merged into the
//               output header with one atomicOr each (width rule, Eq. 1 with
//               the two's complement reading);
//   k_pack   -- reads the width from the header and writes the fields.  A warp
//               packs a tile of 1024 fields (32 groups of 32, i.e. 32*b whole
//               words): lanes produce fields with coalesced loads into a
//               padded shared-memory tile, then each lane assembles whole
//               output words from the fields that overlap them (funnel
//               shifts), so no word is written by more than one lane and
//               every store is a coalesced 32-bit store.
// A preceding k_init (one thread) validates inputs and clears the header.
#pragma once

#include "ccm_device.cuh"
#include "kernels.h"

namespace ccm {

constexpr int kStatsThreads = 256;
constexpr int kPackWarps = 4;
constexpr int kPackThreads = kPackWarps * kWarp;
constexpr int kTilePad = kTileFields + kTileFields / 32;  // one pad slot per 32 fields

// ---------------------------------------------------------------------------
// Producers: value of field i of the result.  `ovf` is or-ed with 1 when the
// exact value does not fit int64.  init() runs once per thread before use.
// ---------------------------------------------------------------------------
struct ProdDenseI64 {
  const int64_t* __restrict__ p;
  __device__ __forceinline__ void init() {}
  __device__ __forceinline__ int64_t operator()(uint64_t i, int&) const { return __ldg(p + i); }
};

struct ProdDenseI32 {
  const int32_t* __restrict__ p;
  __device__ __forceinline__ void init() {}
  __device__ __forceinline__ int64_t operator()(uint64_t i, int&) const {
    return (int64_t)__ldg(p + i);
  }
};

struct ProdPacked {
  const ccm_header* h;
  const uint32_t* __restrict__ w;
  int b, sgn;
  __device__ __forceinline__ void init() {
    b = h->width;
    sgn = h->is_signed;
  }
  __device__ __forceinline__ int64_t operator()(uint64_t i, int&) const {
    return decode_field(w, i, b, sgn);
  }
};

struct ProdAdd {
  ProdPacked a, b;
  __device__ __forceinline__ void init() {
    a.init();
    b.init();
  }
  __device__ __forceinline__ int64_t operator()(uint64_t i, int& ovf) const {
    return add_checked(a(i, ovf), b(i, ovf), ovf);
  }
};

struct ProdScale {
  ProdPacked a;
  int64_t s;
  __device__ __forceinline__ void init() { a.init(); }
  __device__ __forceinline__ int64_t operator()(uint64_t i, int& ovf) const {
    return mul_checked(a(i, ovf), s, ovf);
  }
};

// ---------------------------------------------------------------------------
// k_init: validate up to two input headers, clear the output header.
// ---------------------------------------------------------------------------
struct InitArgs {
  ccm_header* out;
  const ccm_header* in0;
  const ccm_header* in1;
  uint64_t in0_rows, in0_cols, in1_rows, in1_cols;
  uint64_t in0_capacity, in1_capacity;
  uint64_t out_rows, out_cols;
  int64_t* zero_ptr;  // optional int64 buffer cleared here
  uint64_t zero_count;
};

__global__ void k_init(InitArgs a);

// ---------------------------------------------------------------------------
// k_stats
// ---------------------------------------------------------------------------
// `after_lanes`: an add/scale whose lane pass may have run first (it marks
// the header, reserved1 = 1, and leaves the exact statistics there).
template <class P>
__global__ void __launch_bounds__(kStatsThreads) k_stats(P prod, ccm_header* out, uint64_t n,
                                                         int after_lanes) {
  if (out->status != CCM_OK) return;
  if (after_lanes && out->reserved1) return;
  prod.init();
  uint64_t orv = 0;
  uint32_t neg = 0;
  int ovf = 0;
  uint64_t stride = (uint64_t)gridDim.x * kStatsThreads;
  for (uint64_t i = (uint64_t)blockIdx.x * kStatsThreads + threadIdx.x; i < n; i += stride) {
    int64_t v = prod(i, ovf);
    orv |= fold(v);
    neg |= (uint32_t)(v < 0);
  }
  orv = warp_or64(orv);
  neg = __reduce_or_sync(0xffffffffu, neg);
  ovf = (int)__reduce_or_sync(0xffffffffu, (uint32_t)ovf);
  __shared__ uint64_t s_or[kStatsThreads / kWarp];
  __shared__ uint32_t s_neg[kStatsThreads / kWarp];
  __shared__ int s_ovf[kStatsThreads / kWarp];
  int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  if (lane == 0) {
    s_or[warp] = orv;
    s_neg[warp] = neg;
    s_ovf[warp] = ovf;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 1; k < kStatsThreads / kWarp; ++k) {
      orv |= s_or[k];
      neg |= s_neg[k];
      ovf |= s_ovf[k];
    }
    if (orv) atomicOr(reinterpret_cast<unsigned long long*>(&out->stat_or), (unsigned long long)orv);
    if (neg) atomicOr(&out->stat_neg, 1u);
    if (ovf) set_status(out, CCM_E_OVERFLOW);
  }
}

// ---------------------------------------------------------------------------
// k_pack
// ---------------------------------------------------------------------------
// Resolves the output width from the header statistics; returns false (and
// leaves the words alone) when an error is pending or the capacity is short.
// Block 0 publishes width, sign, word count and magic, and zeroes pad words.
__device__ __forceinline__ bool resolve_output(ccm_header* out, uint32_t* words, uint64_t capacity,
                                               uint64_t n, int& b, int& sgn) {
  if (out->status != CCM_OK) return false;
  uint64_t orv = out->stat_or;
  uint32_t neg = out->stat_neg;
  b = width_from_stats(orv, neg);
  sgn = neg ? 1 : 0;
  uint64_t nw = words_for(n, b);
  bool fits = nw <= capacity;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    out->width = b;
    out->is_signed = sgn;
    out->nwords = nw;
    out->magic = CCM_MAGIC;
    if (!fits) out->status = CCM_E_CAPACITY;
  }
  if (!fits) return false;
  uint64_t dw = data_words(n, b);
  if (blockIdx.x == 0 && threadIdx.x < nw - dw) words[dw + threadIdx.x] = 0u;
  return true;
}

template <class P>
__global__ void __launch_bounds__(kPackThreads) k_pack(P prod, ccm_header* out, uint32_t* words,
                                                       uint64_t capacity, uint64_t n,
                                                       int after_lanes) {
  __shared__ uint32_t s_lo[kPackWarps][kTilePad];
  __shared__ uint32_t s_hi[kPackWarps][kTilePad];
  int b, sgn;
  if (!resolve_output(out, words, capacity, n, b, sgn)) return;
  // the lane pass wrote every field at the exact width: nothing left to do
  if (after_lanes && out->reserved1 && b == (int)out->reserved0) return;
  prod.init();
  const int warp = threadIdx.x / kWarp, lane = threadIdx.x % kWarp;
  uint32_t* lo_t = s_lo[warp];
  uint32_t* hi_t = s_hi[warp];
  const uint64_t mask = field_mask(b);
  const bool wide = b > 32;
  const uint64_t ntiles = (n + kTileFields - 1) / kTileFields;
  const uint64_t gwarps = (uint64_t)gridDim.x * kPackWarps;
  for (uint64_t tile = (uint64_t)blockIdx.x * kPackWarps + warp; tile < ntiles; tile += gwarps) {
    const uint64_t base = tile * kTileFields;
    const uint32_t nt = (uint32_t)min((uint64_t)kTileFields, n - base);
    int ovf = 0;
    // 1. produce the tile's fields (coalesced) into the padded shared tile
#pragma unroll 4
    for (int s = 0; s < kTileFields / kWarp; ++s) {
      uint32_t f = (uint32_t)s * kWarp + lane;
      uint64_t pat = 0;
      if (f < nt) pat = (uint64_t)prod(base + f, ovf) & mask;
      lo_t[f + (f >> 5)] = (uint32_t)pat;
      if (wide) hi_t[f + (f >> 5)] = (uint32_t)(pat >> 32);
    }
    __syncwarp();
    // 2. assemble whole words; word W of the tile covers tile bits [32W, 32W+32)
    const uint32_t tw = (uint32_t)((nt * (uint64_t)b + 31) >> 5);
    uint32_t* wout = words + tile * (uint64_t)(kWarp * b);
    for (uint32_t W = lane; W < tw; W += kWarp) {
      const uint32_t bit0 = W * 32u;
      uint32_t f = bit0 / (uint32_t)b;
      uint32_t f_end = min((bit0 + 31u) / (uint32_t)b, nt - 1u);
      uint32_t acc = 0;
      for (; f <= f_end; ++f) {
        int o = (int)(f * (uint32_t)b) - (int)bit0;  // field start relative to the word
        uint32_t lo = lo_t[f + (f >> 5)];
        if (o >= 0) {
          acc |= lo << o;
        } else {
          uint32_t hi = wide ? hi_t[f + (f >> 5)] : 0u;
          uint64_t pat = ((uint64_t)hi << 32) | lo;
          acc |= (uint32_t)(pat >> (-o));
        }
      }
      wout[W] = acc;
    }
    __syncwarp();
  }
}

// Launch helpers (stream order: init, stats, pack).
int num_sms();
void note_launch(int count);
template <class P>
void launch_stats(const P& prod, ccm_header* out, uint64_t n, cudaStream_t st,
                  int after_lanes = 0) {
  uint64_t want = (n + kStatsThreads * 8 - 1) / (kStatsThreads * 8);
  int grid = (int)umin(umax(want, 1), (uint64_t)num_sms() * 8);
  k_stats<P><<<grid, kStatsThreads, 0, st>>>(prod, out, n, after_lanes);
  note_launch();
}

template <class P>
void launch_pack(const P& prod, ccm_header* out, uint32_t* words, uint64_t capacity, uint64_t n,
                 cudaStream_t st, int after_lanes = 0) {
  uint64_t tiles = (n + kTileFields - 1) / kTileFields;
  uint64_t want = (tiles + kPackWarps - 1) / kPackWarps;
  int grid = (int)umin(umax(want, 1), (uint64_t)num_sms() * 16);
  k_pack<P><<<grid, kPackThreads, 0, st>>>(prod, out, words, capacity, n, after_lanes);
  note_launch();
}

void launch_init(const InitArgs& a, cudaStream_t st);
void launch_check(const ccm_matrix& p, const ccm_matrix& q, ccm_header* out, cudaStream_t st);

}  // namespace ccm
