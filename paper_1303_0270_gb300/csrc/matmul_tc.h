// matmul_tc.h -- exact integer matmul on the tcgen05 tensor cores (internal).
#pragma once

#include <cuda_runtime.h>

#include "ccm.h"

namespace ccm {

bool matmul_tc_supported(uint64_t m, uint64_t k, uint64_t n);
size_t matmul_tc_workspace(uint64_t m, uint64_t k, uint64_t n);
// Writes the exact int64 product into `c_scratch` (m x n, row-major).
void run_matmul_tc(const ccm_matrix& a, const ccm_matrix& b, const ccm_matrix& c,
                   int64_t* c_scratch, void* ws, cudaStream_t st);

}  // namespace ccm
