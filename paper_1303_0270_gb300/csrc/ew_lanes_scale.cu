// ew_lanes_scale.cu -- the lane pass of scale (see ew_kernels.cuh).
#include "ew_lanes.cuh"

namespace ccm {
namespace ge {

void launch_lanes_scale(const OpScale<true>& op, ccm_header* out, uint32_t* words,
                        uint64_t capacity, uint64_t n, int bmax, cudaStream_t st) {
  launch_lanes<OpScale<true>>(op, out, words, capacity, n, bmax, st);
}

}  // namespace ge
}  // namespace ccm
