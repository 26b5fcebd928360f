// ew32_scale_wide.cu -- scale by |s| >= 2^15 (statistics, speculative and
// pack passes) for widths <= 32 (see ew_kernels.cuh).
#include "ew_kernels.cuh"

namespace ccm {
namespace ge {

template int launch_ew_scale<32, false>(const EwCall& c, cudaStream_t st);

}  // namespace ge
}  // namespace ccm
