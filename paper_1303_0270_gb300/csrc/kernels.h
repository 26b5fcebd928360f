// kernels.h -- host-side launchers behind the C ABI (internal to libccm).
#pragma once

#include <cuda_runtime.h>

#include "ccm.h"

namespace ccm {

int num_sms();
int max_smem_optin();  // shared memory a CTA may opt in to (bytes)

// Largest width whose words fit `capacity` words for n fields (64 for n = 0):
// a bound the host can compute although the width itself lives on the GPU.
int width_bound(uint64_t capacity, uint64_t n);
int bitlen_host(uint64_t v);

// Launch accounting and the per-call profiling hook (ccm_profile_next).
void note_launch(int count = 1);
void profile_begin(cudaStream_t st);
// True when the next profile_begin() will record (the calling thread armed
// ccm_profile_next); such a call launches without programmatic dependent
// launch, so no event record sits between two programmatically linked kernels.
bool profile_armed();
void profile_end(cudaStream_t st);

void run_measure(const void* dense, int dtype, uint64_t rows, uint64_t cols, ccm_header* hdr,
                 cudaStream_t st);
// Workspace of the single-pass pack (0 when the capacity gives no width class).
size_t pack_workspace(uint64_t rows, uint64_t cols, uint64_t capacity);
void run_pack(const void* dense, int dtype, uint64_t rows, uint64_t cols, const ccm_matrix& out,
              void* ws, size_t ws_bytes, cudaStream_t st);
void run_unpack(const ccm_matrix& a, void* dense, int dtype, int32_t* err, cudaStream_t st);
void run_get(const ccm_matrix& a, const uint64_t* idx, uint64_t count, int64_t* out, int32_t* err,
             cudaStream_t st);
void run_add(const ccm_matrix& a, const ccm_matrix& b, const ccm_matrix& c, void* ws,
             size_t ws_bytes, cudaStream_t st);
void run_scale(const ccm_matrix& a, int64_t s, const ccm_matrix& c, void* ws, size_t ws_bytes,
               cudaStream_t st);
// Packs an int64 result held in scratch; `stats_done` when the producing
// kernel has already merged the width statistics into out's header.
void run_pack_scratch(const int64_t* vals, const ccm_matrix& out, cudaStream_t st,
                      bool stats_done = false);
// The same from an int32 scratch whose width statistics the producing kernel
// has already merged into out's header.
void run_pack_scratch32(const int32_t* vals, const ccm_matrix& out, cudaStream_t st);
// The tensor matmul writes C as int32 when the output capacity bounds C's
// width by 31 bits (every result the output can hold fits int32).
bool matmul_c32(const ccm_matrix& c);

// Host checks of ccm_matvec that need no workspace (pointers, alignment,
// shapes, y's minimum capacity).
ccm_status matvec_host_check(const ccm_matrix* a, const ccm_matrix* x, const ccm_matrix* y);
size_t matvec_workspace(uint64_t m, uint64_t n);
// The streaming matvec (matvec_stream.cu): whether it takes an m x n product
// whose widths the capacities bound by bmax_a and bmax_x, and its launches.
namespace mvs {
bool stream_applies(uint64_t m, uint64_t n, int bmax_a, int bmax_x);
void run_stream(const ccm_matrix& a, const ccm_matrix& x, const ccm_matrix& y, void* ws,
                cudaStream_t st);
}  // namespace mvs
size_t matvec2_workspace(uint64_t m, uint64_t n1, uint64_t n2);
void run_matvec2(const ccm_matrix& a, const ccm_matrix& x, const ccm_matrix& b,
                 const ccm_matrix& z, const ccm_matrix& y, void* ws, cudaStream_t st);
void run_matvec(const ccm_matrix& a, const ccm_matrix& x, const ccm_matrix& y, void* ws,
                cudaStream_t st);

void run_repack(const ccm_matrix& in, int width, int is_signed, const ccm_matrix& out,
                uint64_t row_offset, cudaStream_t st);

size_t matmul_workspace(const ccm_matrix& a, const ccm_matrix& b);
// Shape-only bound on matmul_workspace (the widths are unknown): the tensor
// path at its widest (4 digits per field).
size_t matmul_workspace_upper(uint64_t m, uint64_t k, uint64_t n);
int run_matmul(const ccm_matrix& a, const ccm_matrix& b, const ccm_matrix& c, int path, void* ws,
               cudaStream_t st);

size_t vlb_workspace(uint64_t n);
size_t vlb_matvec_workspace(uint64_t rows);
void run_vlb_matvec(const ccm_header* hdr, const uint32_t* words, uint64_t capacity,
                    const uint64_t* index, uint64_t rows, uint64_t cols, const ccm_matrix& x,
                    const ccm_matrix& y, void* ws, cudaStream_t st);
void run_vlb_pack(const void* dense, int dtype, uint64_t rows, uint64_t cols, ccm_header* hdr,
                  uint32_t* words, uint64_t capacity, uint64_t* index, void* ws, cudaStream_t st);
void run_vlb_unpack(const ccm_header* hdr, const uint32_t* words, uint64_t capacity,
                    const uint64_t* index, uint64_t rows, uint64_t cols, void* dense, int dtype,
                    int32_t* err, cudaStream_t st);

void run_gen_uniform(int64_t* out, uint64_t count, uint64_t seed, uint64_t stream_id,
                     uint64_t start, int64_t lo, int64_t hi, cudaStream_t st);
void run_gen_poisson(int64_t* out, uint64_t count, uint64_t seed, uint64_t stream_id,
                     uint64_t start, const double* table, uint32_t table_len, cudaStream_t st);

}  // namespace ccm
