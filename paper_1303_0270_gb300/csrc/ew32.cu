// ew32.cu -- the group-engine elementwise kernels for widths <= 32 (see
// ew_kernels.cuh); one translation unit per width class.
#include "ew_kernels.cuh"

namespace ccm {
namespace ge {

template int launch_ew_class<32>(const EwCall& c, cudaStream_t st);

}  // namespace ge
}  // namespace ccm
