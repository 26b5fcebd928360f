// cta_pack.cuh -- a short vector of int64 values (up to 16,384) packed by a
// small grid in one launch: every CTA reads all the values for the width
// statistics (a few hundred KB of L2 reads at most), stages only its own
// groups of 32 fields in shared memory and packs them; CTA 0 writes the
// header and the pad words.  No CTA waits for another (k_mv_ypack's y,
// k_pack_small's small dense input).
#pragma once

#include "ccm_device.cuh"

namespace ccm {

constexpr uint32_t kVecGroupsPerCta = 16;  // 32-field groups a CTA packs
constexpr int kVecThreads = 512;

// CTAs for m values.
__host__ __device__ constexpr uint32_t vec_pack_ctas(uint64_t m) {
  return (uint32_t)(((m + 31) / 32 + kVecGroupsPerCta - 1) / kVecGroupsPerCta);
}

// Shared state of one CTA: its groups' fields (33 slots per group, so the 32
// lanes that fill a group hit 32 different banks) and the statistics.
struct VecPackSmem {
  uint64_t ys[kVecGroupsPerCta * 33];
  uint64_t s_or[kVecThreads / 32];
  uint32_t s_neg[kVecThreads / 32];
};

// Reads the mm values get(i) (int64) once: the CTA's statistics over all of
// them (OR of the folded values, any negative), reduced to every thread, and
// the fields of groups [g0, g0 + kVecGroupsPerCta) staged in sm.ys.
template <class Get>
__device__ __forceinline__ void vec_stats_stage(Get get, uint32_t mm, uint32_t g0,
                                                VecPackSmem& sm, uint64_t& orv, uint32_t& neg) {
  const uint32_t lo = g0 * 32, hi = umin(mm, (g0 + kVecGroupsPerCta) * 32);
  uint64_t o = 0;
  uint32_t ng = 0;
  for (uint32_t base = 0; base < mm; base += 8 * kVecThreads) {
    int64_t v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {  // all eight loads in flight together
      const uint32_t i = base + j * kVecThreads + threadIdx.x;
      v[j] = i < mm ? get(i) : 0;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const uint32_t i = base + j * kVecThreads + threadIdx.x;
      if (i >= lo && i < hi) sm.ys[((i - lo) >> 5) * 33 + (i & 31)] = (uint64_t)v[j];
      o |= fold(v[j]);
      ng |= (uint32_t)(v[j] < 0);
    }
  }
  o = warp_or64(o);
  ng = __reduce_or_sync(0xffffffffu, ng);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) {
    sm.s_or[warp] = o;
    sm.s_neg[warp] = ng;
  }
  __syncthreads();
  orv = 0;
  neg = 0;
  for (int w = 0; w < kVecThreads / 32; ++w) {
    orv |= sm.s_or[w];
    neg |= sm.s_neg[w];
  }
}

// Packs the staged groups [g0, g0 + kVecGroupsPerCta) of the mm fields at
// width b.  A group is b whole words; lane i of the warp that takes the group
// assembles its words i and i + 32 from the fields that overlap them (no
// word is written twice).  CTA 0 also zeroes the pad words from dw to nw.
__device__ __forceinline__ void vec_pack_groups(const VecPackSmem& sm, uint32_t mm, uint32_t g0,
                                                int b, uint32_t* words, uint64_t dw,
                                                uint64_t nw) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint64_t mask = field_mask(b);
  const uint32_t g1 = umin((mm + 31) / 32, g0 + kVecGroupsPerCta);
  int flo[2], fhi[2];  // fields overlapping word i (and i + 32) of a group
  for (int h = 0; h < 2; ++h) {
    const int wi = lane + 32 * h;
    flo[h] = wi * 32 / b;
    fhi[h] = (wi * 32 + 31) / b;
  }
  for (uint32_t g = g0 + warp; g < g1; g += kVecThreads / 32) {
    const uint32_t nf = umin(32, mm - g * 32);
    const uint32_t nwg = (uint32_t)((nf * (uint64_t)b + 31) / 32);  // words of this group
    const uint64_t* src = sm.ys + (g - g0) * 33;
    for (int h = 0; h < 2; ++h) {
      const uint32_t wi = lane + 32 * h;
      if (wi >= nwg) continue;
      uint32_t acc = 0;
      const int fe = fhi[h] < (int)nf - 1 ? fhi[h] : (int)nf - 1;
      for (int f = flo[h]; f <= fe; ++f) {
        const int o = f * b - (int)wi * 32;  // field start relative to the word
        const uint64_t pat = src[f] & mask;
        acc |= o >= 0 ? (uint32_t)(pat << o) : (uint32_t)(pat >> (-o));
      }
      words[(uint64_t)g * b + wi] = acc;
    }
  }
  if (blockIdx.x == 0)
    for (uint64_t W = dw + threadIdx.x; W < nw; W += kVecThreads) words[W] = 0;
}

}  // namespace ccm
