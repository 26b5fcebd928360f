// matvec_fast16.cu -- the streaming matvec kernel for widths <= 16
// (see matvec_fast.cuh); a translation unit of its own so the width classes
// compile in parallel.
#include "matvec_fast.cuh"

namespace ccm {
namespace mvf {

template <bool NARROW>
static void launch(const Args& a, dim3 grid, int threads, size_t smem, cudaStream_t st) {
  static bool attr_done = false;
  if (!attr_done) {
    cudaFuncSetAttribute(k_matvec_fast<16, NARROW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         227 * 1024);
    attr_done = true;
  }
  k_matvec_fast<16, NARROW><<<grid, threads, smem, st>>>(a);
}

int resident_ctas_16(int threads, size_t smem) {
  int n = 0;
  cudaFuncSetAttribute(k_matvec_fast<16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       227 * 1024);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_matvec_fast<16, true>, threads, smem) !=
      cudaSuccess)
    return 1;
  return n;
}

void launch_matvec_fast16(const Args& a, bool narrow, dim3 grid, int threads, size_t smem,
                         cudaStream_t st) {
  if (narrow)
    launch<true>(a, grid, threads, smem, st);
  else
    launch<false>(a, grid, threads, smem, st);
}

}  // namespace mvf
}  // namespace ccm
