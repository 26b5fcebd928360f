// gen.cu -- synthetic workload inputs generated on the GPU.  Not part of the
// compression method: it draws the integer matrices the workloads are made
// of, with the counter-based SplitMix64 scheme (Steele, Lea and Flood 2014)
// that the host-side test-input generator uses, so large inputs need not
// cross PCIe and any entry can be regenerated on its own.
#include "ccm_device.cuh"
#include "kernels.h"

namespace ccm {

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_gen_uniform(int64_t* __restrict__ out, uint64_t count, uint64_t key,
                              uint64_t start, uint64_t lo, uint64_t range) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    uint64_t u = mix64(key + (start + i + 1) * kGamma);
    uint64_t off = range ? __umul64hi(u, range) : u;  // range 0 encodes 2^64
    out[i] = (int64_t)(lo + off);
  }
}

__global__ void k_gen_poisson(int64_t* __restrict__ out, uint64_t count, uint64_t key,
                              uint64_t start, const double* __restrict__ table, uint32_t len) {
  extern __shared__ double s_table[];
  for (uint32_t t = threadIdx.x; t < len; t += blockDim.x) s_table[t] = table[t];
  __syncthreads();
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    uint64_t u = mix64(key + (start + i + 1) * kGamma);
    double x = (double)(u >> 11) * 0x1.0p-53;
    // number of table entries <= x (the table is non-decreasing)
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
      uint32_t mid = (lo + hi) >> 1;
      if (s_table[mid] <= x)
        lo = mid + 1;
      else
        hi = mid;
    }
    out[i] = (int64_t)lo;
  }
}

int gen_grid(uint64_t count) {
  return (int)umin(umax((count + 255) / 256, 1), (uint64_t)num_sms() * 16);
}

}  // namespace

void run_gen_uniform(int64_t* out, uint64_t count, uint64_t seed, uint64_t stream_id,
                     uint64_t start, int64_t lo, int64_t hi, cudaStream_t st) {
  uint64_t key = mix64(seed + (stream_id + 1) * kGamma);
  uint64_t range = (uint64_t)hi - (uint64_t)lo + 1;
  k_gen_uniform<<<gen_grid(count), 256, 0, st>>>(out, count, key, start, (uint64_t)lo, range);
  note_launch();
}

void run_gen_poisson(int64_t* out, uint64_t count, uint64_t seed, uint64_t stream_id,
                     uint64_t start, const double* table, uint32_t table_len, cudaStream_t st) {
  uint64_t key = mix64(seed + (stream_id + 1) * kGamma);
  k_gen_poisson<<<gen_grid(count), 256, table_len * sizeof(double), st>>>(out, count, key, start,
                                                                         table, table_len);
  note_launch();
}

}  // namespace ccm
