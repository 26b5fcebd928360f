// runtime.cu -- launch accounting and the per-call kernel timing hook.
#include <atomic>

#include "kernels.h"

namespace ccm {

namespace {
std::atomic<uint64_t> g_launches{0};
thread_local cudaEvent_t t_start = nullptr, t_stop = nullptr;
thread_local bool t_armed = false, t_open = false;
}  // namespace

void note_launch(int count) { g_launches.fetch_add((uint64_t)count, std::memory_order_relaxed); }

void profile_begin(cudaStream_t st) {
  if (t_armed && !t_open) {
    cudaEventRecord(t_start, st);
    t_open = true;
  }
}

bool profile_armed() { return t_armed && !t_open; }

void profile_end(cudaStream_t st) {
  if (t_armed && t_open) {
    cudaEventRecord(t_stop, st);
    t_open = false;
    t_armed = false;
  }
}

}  // namespace ccm

extern "C" {

uint64_t ccm_launch_count(void) { return ccm::g_launches.load(std::memory_order_relaxed); }

ccm_status ccm_profile_next(void* start_event, void* stop_event) {
  if ((start_event == nullptr) != (stop_event == nullptr)) return CCM_E_INVAL;
  ccm::t_start = reinterpret_cast<cudaEvent_t>(start_event);
  ccm::t_stop = reinterpret_cast<cudaEvent_t>(stop_event);
  ccm::t_armed = start_event != nullptr;
  ccm::t_open = false;
  return CCM_OK;
}

}  // extern "C"
