// cta_pack.cuh -- one CTA packs a short vector of int64 values, held in
// shared memory, at a width it already knows (the last step of the one-CTA
// pack kernels: k_mv_ypack's y, k_pack_small's small dense input).
#pragma once

#include "ccm_device.cuh"

namespace ccm {

// The fields f of group g (32 fields) sit at ys[g * 33 + f] (33 slots per
// group: the 32 lanes that fill a group hit 32 different banks).  A group is
// b whole words; lane i of the warp that takes the group assembles its words
// i and i + 32 from the fields that overlap them, so no word is written
// twice; then the zero pad words from dw to nw.  Every thread of the CTA
// calls it (after a __syncthreads that makes ys complete).
__device__ __forceinline__ void cta_pack_groups(const uint64_t* ys, uint32_t mm, int b,
                                                uint32_t* words, uint64_t dw, uint64_t nw) {
  const int nwarps = blockDim.x / 32, warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint64_t mask = field_mask(b);
  const uint32_t groups = (mm + 31) / 32;
  int flo[2], fhi[2];  // fields overlapping word i (and i + 32) of a group
  for (int h = 0; h < 2; ++h) {
    const int wi = lane + 32 * h;
    flo[h] = wi * 32 / b;
    fhi[h] = (wi * 32 + 31) / b;
  }
  for (uint32_t g = warp; g < groups; g += nwarps) {
    const uint32_t nf = umin(32, mm - g * 32);
    const uint32_t nwg = (uint32_t)((nf * (uint64_t)b + 31) / 32);  // words of this group
    const uint64_t* src = ys + g * 33;
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
  for (uint64_t W = dw + threadIdx.x; W < nw; W += blockDim.x) words[W] = 0;
}

}  // namespace ccm
