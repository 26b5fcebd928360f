// matvec_rows8.cu -- the row-streaming matvec kernel for widths <= 8
// (see matvec_fast.cuh); a translation unit of its own so the width classes
// compile in parallel.
#include "matvec_fast.cuh"

namespace ccm {
namespace mvf {
namespace rows {

template <bool NARROW>
static void set_smem_limit() {
  static int done_dev = -1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (done_dev != dev) {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncSetAttribute(k_matvec_rows<8, NARROW>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         optin);
    done_dev = dev;
  }
}

int resident_ctas_8(int threads, size_t smem) {
  set_smem_limit<true>();
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_matvec_rows<8, true>, threads, smem) !=
      cudaSuccess)
    return 0;
  return n;
}

void launch_8(const RowArgs& a, bool narrow, unsigned grid, int threads, size_t smem,
               cudaStream_t st) {
  if (narrow) {
    set_smem_limit<true>();
    k_matvec_rows<8, true><<<grid, threads, smem, st>>>(a);
  } else {
    set_smem_limit<false>();
    k_matvec_rows<8, false><<<grid, threads, smem, st>>>(a);
  }
}

}  // namespace rows
}  // namespace mvf
}  // namespace ccm
