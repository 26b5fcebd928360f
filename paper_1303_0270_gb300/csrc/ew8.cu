// ew8.cu -- the group-engine elementwise kernels for widths <= 8 (see
// ew_kernels.cuh): every launcher family of the class.
#include "ew_kernels.cuh"

namespace ccm {
namespace ge {

template int launch_ew_add<8>(const EwCall& c, cudaStream_t st);
template int launch_ew_scale<8, true>(const EwCall& c, cudaStream_t st);
template int launch_ew_scale<8, false>(const EwCall& c, cudaStream_t st);
template int launch_ew_pack<8>(const EwCall& c, cudaStream_t st);

}  // namespace ge
}  // namespace ccm
