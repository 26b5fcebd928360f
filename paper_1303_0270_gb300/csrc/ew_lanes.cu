// ew_lanes.cu -- the lane pass of add (see ew_kernels.cuh), instantiated
// once here rather than in every width-class unit; scale's lane pass is in
// ew_lanes_scale.cu.
#include "ew_lanes.cuh"

namespace ccm {
namespace ge {

void launch_lanes_add(const OpAdd& op, ccm_header* out, uint32_t* words, uint64_t capacity,
                      uint64_t n, int bmax, cudaStream_t st) {
  launch_lanes<OpAdd>(op, out, words, capacity, n, bmax, st);
}

}  // namespace ge
}  // namespace ccm
