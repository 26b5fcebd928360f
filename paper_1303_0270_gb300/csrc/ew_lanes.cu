// ew_lanes.cu -- the byte-lane pass of add and scale (see ew_kernels.cuh),
// instantiated once here rather than in every width-class unit.
#include "ew_kernels.cuh"

namespace ccm {
namespace ge {

// One wave: the tiles are assigned to warps statically (grid stride), so a
// second wave of CTAs would only add a tail.
template <class Op>
static int lanes_grid(uint64_t n) {
  static int per_sm = 0;
  if (!per_sm) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ew_lanes<Op>, kThreads, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  return ew_grid(n, per_sm);
}

void launch_lanes_add(const OpAdd& op, ccm_header* out, uint32_t* words, uint64_t capacity,
                      uint64_t n, cudaStream_t st) {
  k_ew_lanes<OpAdd><<<lanes_grid<OpAdd>(n), kThreads, 0, st>>>(op, out, words, capacity, n);
}

void launch_lanes_scale(const OpScale<true>& op, ccm_header* out, uint32_t* words,
                        uint64_t capacity, uint64_t n, cudaStream_t st) {
  k_ew_lanes<OpScale<true>><<<lanes_grid<OpScale<true>>(n), kThreads, 0, st>>>(op, out, words,
                                                                             capacity, n);
}

}  // namespace ge
}  // namespace ccm
