// ew_lanes.cu -- the byte-lane pass of add and scale (see ew_kernels.cuh),
// instantiated once here rather than in every width-class unit.
#include "ew_kernels.cuh"

namespace ccm {
namespace ge {

void launch_lanes_add(const OpAdd& op, ccm_header* out, uint32_t* words, uint64_t capacity,
                      uint64_t n, cudaStream_t st) {
  k_ew_lanes<OpAdd><<<ew_grid(n, 12), kThreads, 0, st>>>(op, out, words, capacity, n);
}

void launch_lanes_scale(const OpScale<true>& op, ccm_header* out, uint32_t* words,
                        uint64_t capacity, uint64_t n, cudaStream_t st) {
  k_ew_lanes<OpScale<true>><<<ew_grid(n, 12), kThreads, 0, st>>>(op, out, words, capacity, n);
}

}  // namespace ge
}  // namespace ccm
