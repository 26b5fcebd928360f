// matvec_fast32.cu -- the streaming matvec kernel for widths <= 32
// (see matvec_fast.cuh); a translation unit of its own so the width classes
// compile in parallel.
#include "matvec_fast.cuh"

namespace ccm {
namespace mvf {

void launch_matvec_fast32(const Args& a, dim3 grid, int threads, size_t smem, cudaStream_t st) {
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_matvec_fast<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr_done = true;
  }
  k_matvec_fast<32><<<grid, threads, smem, st>>>(a);
}

}  // namespace mvf
}  // namespace ccm
