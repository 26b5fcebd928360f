// matvec_static.cu -- ccm_matvec for callers that must not allocate device
// memory.
//
// ccm_matvec needs a device workspace (x decoded to int64 and the int64
// partial sums of y) that the caller provides.  Some callers cannot provide
// one: a process whose device memory is entirely reserved up front by
// another component's allocator, or code on a latency-critical path where
// the device-wide synchronisation that cudaMalloc/cudaFree may cause is not
// acceptable.  ccm_matvec_static serves them from one fixed scratch array
// compiled into this library (CCM_STATIC_SCRATCH_BYTES per GPU that loads
// it, held until the process exits) and allocates nothing.
//
// The array is shared by every call on a device and keeps whatever the last
// call left in it; the matvec kernels clear what they need before use.  Two
// calls whose work overlaps on the GPU (different streams, no ordering
// between them) use the same array at the same time and race: order them.
#include <mutex>

#include "ccm.h"
#include "ccm_device.cuh"
#include "kernels.h"

namespace ccm {
namespace {

// The scratch itself.  In host code `g_static_scratch` only names a host-side
// stand-in of the symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_static_scratch[CCM_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached; nullptr on failure.
void* scratch_for_current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess) return nullptr;
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

}  // namespace
}  // namespace ccm

extern "C" ccm_status ccm_matvec_static(const ccm_matrix* a, const ccm_matrix* x,
                                        const ccm_matrix* y, ccm_stream_t stream) {
  // ccm_matvec's host checks apply unchanged (matvec_host_check below); the
  // size limit comes first so that no size arithmetic can wrap
  if (!a || !x || !y) return CCM_E_INVAL;
  if (x->rows != a->cols || x->cols != 1 || y->rows != a->rows || y->cols != 1)
    return CCM_E_SHAPE;
  if (a->rows > CCM_STATIC_SCRATCH_BYTES / 8 || a->cols > CCM_STATIC_SCRATCH_BYTES / 8)
    return CCM_E_CAPACITY;
  const size_t need = ccm::matvec_workspace(a->rows, a->cols);
  if (need > CCM_STATIC_SCRATCH_BYTES) return CCM_E_CAPACITY;  // too large for the fixed scratch
  // every other host check before the first CUDA call
  const ccm_status hc = ccm::matvec_host_check(a, x, y);
  if (hc != CCM_OK) return hc;
  void* ws = ccm::scratch_for_current_device();
  if (!ws) return CCM_E_CUDA;
  return ccm_matvec(a, x, y, ws, CCM_STATIC_SCRATCH_BYTES, stream);
}
