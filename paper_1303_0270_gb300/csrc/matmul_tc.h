// matmul_tc.h -- exact integer matmul on the tcgen05 tensor cores (internal).
#pragma once

#include <cuda_runtime.h>

#include "ccm.h"

namespace ccm {

// True when both operand widths (bounded by their capacities) are at most
// 16 bits and the inner size keeps every digit-class sum below 2^24.
bool matmul_tc_supported(const ccm_matrix& a, const ccm_matrix& b);
size_t matmul_tc_workspace(const ccm_matrix& a, const ccm_matrix& b);
size_t matmul_tc_workspace_upper(uint64_t m, uint64_t k, uint64_t n);
// Writes the exact int64 product into `c_scratch` (m x n, row-major) and
// merges its width statistics into c's header.
int run_matmul_tc(const ccm_matrix& a, const ccm_matrix& b, const ccm_matrix& c,
                  int64_t* c_scratch, void* ws, cudaStream_t st);

}  // namespace ccm
