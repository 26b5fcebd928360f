// ew_lanes.cuh -- host launcher of the lane pass (k_ew_lanes, ew_kernels.cuh).
#pragma once
#include "ew_kernels.cuh"

namespace ccm {
namespace ge {

// One wave: the tiles are assigned to warps statically (grid stride), so a
// second wave of CTAs would only add a tail.  Shared memory per CTA from the
// width bound `bmax` (inputs up to bmax bits, results up to Op::kLaneGrow
// bits wider).
template <class Op>
static void launch_lanes(const Op& op, ccm_header* out, uint32_t* words, uint64_t capacity,
                         uint64_t n, int bmax, cudaStream_t st) {
  const uint32_t ww = lane_warp_words(bmax, Op::kTwoInputs ? 2 : 1, Op::kLaneGrow);
  const size_t smem = (size_t)kWarps * ww * sizeof(uint32_t);
  static int dev_done = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev_done != dev) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    cudaFuncGetAttributes(&fa, k_ew_lanes<Op>);  // (its static mbarriers count against optin)
    cudaFuncSetAttribute(k_ew_lanes<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         optin - (int)fa.sharedSizeBytes);
    dev_done = dev;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ew_lanes<Op>, kThreads, smem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  k_ew_lanes<Op><<<ew_grid(n, per_sm), kThreads, smem, st>>>(op, out, words, capacity, n, ww);
}

}  // namespace ge
}  // namespace ccm
