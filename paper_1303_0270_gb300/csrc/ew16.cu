// ew16.cu -- the group-engine elementwise kernels for widths <= 16 (see
// ew_kernels.cuh): every launcher family of the class.
#include "ew_kernels.cuh"

namespace ccm {
namespace ge {

template int launch_ew_add<16>(const EwCall& c, cudaStream_t st);
template int launch_ew_scale<16, true>(const EwCall& c, cudaStream_t st);
template int launch_ew_scale<16, false>(const EwCall& c, cudaStream_t st);
template int launch_ew_pack<16>(const EwCall& c, cudaStream_t st);

}  // namespace ge
}  // namespace ccm
