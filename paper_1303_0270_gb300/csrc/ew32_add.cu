// ew32_add.cu -- add (statistics, speculative and pack passes) for widths
// <= 32 (see ew_kernels.cuh).
#include "ew_kernels.cuh"

namespace ccm {
namespace ge {

template int launch_ew_add<32>(const EwCall& c, cudaStream_t st);

}  // namespace ge
}  // namespace ccm
