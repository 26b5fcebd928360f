// ew32.cu -- the group-engine pack/unpack kernels for widths <= 32 (see
// ew_kernels.cuh).  The add and scale families of this class are the
// largest instantiations and sit in ew32_add.cu / ew32_scale*.cu so that
// the units compile in parallel.
#include "ew_kernels.cuh"

namespace ccm {
namespace ge {

template int launch_ew_pack<32>(const EwCall& c, cudaStream_t st);

}  // namespace ge
}  // namespace ccm
