// api.cu -- the extern "C" entry points of libccm (declared in ccm.h): host
// checks that need no GPU, then the launchers in pack.cu, matvec.cu and
// matmul.cu.  Every entry point returns before launching anything when a
// host-side check fails.
#include <cuda_runtime.h>

#include "ccm.h"
#include "ccm_device.cuh"
#include "kernels.h"

namespace {

using ccm::words_for;

cudaStream_t to_cuda(ccm_stream_t s) { return reinterpret_cast<cudaStream_t>(s); }

bool valid_out(const ccm_matrix* m) {
  if (!m || !m->hdr || !ccm::shape_ok(m->rows, m->cols)) return false;
  if (m->capacity && !m->words) return false;
  if (reinterpret_cast<uintptr_t>(m->hdr) % 16 || reinterpret_cast<uintptr_t>(m->words) % 16)
    return false;
  return true;
}

bool valid_in(const ccm_matrix* m) {
  if (!m || !m->hdr || !ccm::shape_ok(m->rows, m->cols)) return false;
  if (m->rows * m->cols && !m->words) return false;
  return reinterpret_cast<uintptr_t>(m->hdr) % 16 == 0 &&
         reinterpret_cast<uintptr_t>(m->words) % 16 == 0;
}

ccm_status launched() {
  return cudaGetLastError() == cudaSuccess ? CCM_OK : CCM_E_CUDA;
}

// Words a result can never go below (width 1); a smaller capacity is a
// host-detectable error.
bool capacity_ok(const ccm_matrix* m) { return m->capacity >= words_for(m->rows * m->cols, 1); }

}  // namespace

namespace ccm {
ccm_status matvec_host_check(const ccm_matrix* a, const ccm_matrix* x, const ccm_matrix* y) {
  if (!valid_in(a) || !valid_in(x) || !valid_out(y)) return CCM_E_INVAL;
  if (x->rows != a->cols || x->cols != 1 || y->rows != a->rows || y->cols != 1)
    return CCM_E_SHAPE;
  if (!capacity_ok(y)) return CCM_E_CAPACITY;
  return CCM_OK;
}
}  // namespace ccm

extern "C" {

uint64_t ccm_words_for(uint64_t rows, uint64_t cols, int width) {
  return words_for(rows * cols, width);
}

const char* ccm_status_str(int status) {
  switch (status) {
    case CCM_OK: return "CCM_OK";
    case CCM_E_INVAL: return "CCM_E_INVAL";
    case CCM_E_SHAPE: return "CCM_E_SHAPE";
    case CCM_E_WIDTH: return "CCM_E_WIDTH";
    case CCM_E_OVERFLOW: return "CCM_E_OVERFLOW";
    case CCM_E_CAPACITY: return "CCM_E_CAPACITY";
    case CCM_E_RANGE: return "CCM_E_RANGE";
    case CCM_E_CUDA: return "CCM_E_CUDA";
    case CCM_E_TIMEOUT: return "CCM_E_TIMEOUT";
    case CCM_E_INPUT: return "CCM_E_INPUT";
    default: return "CCM_E_UNKNOWN";
  }
}

int ccm_version(void) { return 100; }

ccm_status ccm_measure(const void* dense, int dtype, uint64_t rows, uint64_t cols,
                       ccm_header* hdr, ccm_stream_t stream) {
  if (!hdr || !ccm::shape_ok(rows, cols) || (rows * cols && !dense)) return CCM_E_INVAL;
  if (dtype != CCM_I32 && dtype != CCM_I64) return CCM_E_INVAL;
  ccm::run_measure(dense, dtype, rows, cols, hdr, to_cuda(stream));
  return launched();
}

ccm_status ccm_pack(const void* dense, int dtype, uint64_t rows, uint64_t cols,
                    const ccm_matrix* out, void* ws, size_t ws_bytes, ccm_stream_t stream) {
  if (!valid_out(out) || !ccm::shape_ok(rows, cols) || (rows * cols && !dense)) return CCM_E_INVAL;
  if (dtype != CCM_I32 && dtype != CCM_I64) return CCM_E_INVAL;
  if (out->rows != rows || out->cols != cols) return CCM_E_SHAPE;
  if (!capacity_ok(out)) return CCM_E_CAPACITY;
  if (ws && reinterpret_cast<uintptr_t>(ws) % 256) return CCM_E_INVAL;
  ccm::run_pack(dense, dtype, rows, cols, *out, ws, ws_bytes, to_cuda(stream));
  return launched();
}

ccm_status ccm_unpack(const ccm_matrix* a, void* dense, int dtype, int32_t* err,
                      ccm_stream_t stream) {
  if (!valid_in(a) || (a->rows * a->cols && !dense)) return CCM_E_INVAL;
  if (dtype != CCM_I32 && dtype != CCM_I64) return CCM_E_INVAL;
  if (a->rows * a->cols == 0 && !err) return CCM_OK;
  ccm::run_unpack(*a, dense, dtype, err, to_cuda(stream));
  return launched();
}

ccm_status ccm_get(const ccm_matrix* a, const uint64_t* idx, uint64_t count, int64_t* out,
                   int32_t* err, ccm_stream_t stream) {
  if (!valid_in(a) || (count && (!idx || !out))) return CCM_E_INVAL;
  ccm::run_get(*a, idx, count, out, err, to_cuda(stream));
  return launched();
}

ccm_status ccm_add(const ccm_matrix* a, const ccm_matrix* b, const ccm_matrix* c, void* ws,
                   size_t ws_bytes, ccm_stream_t stream) {
  if (!valid_in(a) || !valid_in(b) || !valid_out(c)) return CCM_E_INVAL;
  if (a->rows != b->rows || a->cols != b->cols || c->rows != a->rows || c->cols != a->cols)
    return CCM_E_SHAPE;
  if (!capacity_ok(c)) return CCM_E_CAPACITY;
  if (ws && reinterpret_cast<uintptr_t>(ws) % 256) return CCM_E_INVAL;
  ccm::run_add(*a, *b, *c, ws, ws_bytes, to_cuda(stream));
  return launched();
}

ccm_status ccm_scale(const ccm_matrix* a, int64_t s, const ccm_matrix* c, void* ws,
                     size_t ws_bytes, ccm_stream_t stream) {
  if (!valid_in(a) || !valid_out(c)) return CCM_E_INVAL;
  if (c->rows != a->rows || c->cols != a->cols) return CCM_E_SHAPE;
  if (!capacity_ok(c)) return CCM_E_CAPACITY;
  if (ws && reinterpret_cast<uintptr_t>(ws) % 256) return CCM_E_INVAL;
  ccm::run_scale(*a, s, *c, ws, ws_bytes, to_cuda(stream));
  return launched();
}

size_t ccm_workspace_bytes(int op, uint64_t m, uint64_t k, uint64_t n) {
  // shapes whose sizes would wrap: saturated, never a small wrapped value
  using ccm::shape_ok;
  if (op == CCM_OP_MATMUL && !(shape_ok(m, k) && shape_ok(k, n) && shape_ok(m, n)))
    return SIZE_MAX;
  if ((op == CCM_OP_PACK || op == CCM_OP_VLB) && !shape_ok(m, k)) return SIZE_MAX;
  if (op == CCM_OP_VLB_MATVEC && m > ccm::kMaxFields) return SIZE_MAX;
  switch (op) {
    case CCM_OP_MATVEC: return ccm::matvec_workspace(m, k);
    case CCM_OP_PACK: return ccm::pack_workspace(m, k, n);
    case CCM_OP_VLB: return ccm::vlb_workspace(m * k);
    case CCM_OP_VLB_MATVEC: return ccm::vlb_matvec_workspace(m);
    case CCM_OP_MATMUL: return ccm::matmul_workspace_upper(m, k, n);
    default: return 0;
  }
}

ccm_status ccm_matvec(const ccm_matrix* a, const ccm_matrix* x, const ccm_matrix* y, void* ws,
                      size_t ws_bytes, ccm_stream_t stream) {
  const ccm_status hc = ccm::matvec_host_check(a, x, y);
  if (hc != CCM_OK) return hc;
  if (!ws || reinterpret_cast<uintptr_t>(ws) % 256) return CCM_E_INVAL;
  if (ws_bytes < ccm::matvec_workspace(a->rows, a->cols)) return CCM_E_CAPACITY;
  ccm::run_matvec(*a, *x, *y, ws, to_cuda(stream));
  return launched();
}

ccm_status ccm_matvec2(const ccm_matrix* a, const ccm_matrix* x, const ccm_matrix* b,
                       const ccm_matrix* z, const ccm_matrix* y, void* ws, size_t ws_bytes,
                       ccm_stream_t stream) {
  if (!valid_in(a) || !valid_in(x) || !valid_in(b) || !valid_in(z) || !valid_out(y) || !ws)
    return CCM_E_INVAL;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return CCM_E_INVAL;
  if (x->rows != a->cols || x->cols != 1 || z->rows != b->cols || z->cols != 1 ||
      b->rows != a->rows || y->rows != a->rows || y->cols != 1)
    return CCM_E_SHAPE;
  if (!capacity_ok(y)) return CCM_E_CAPACITY;
  if (ws_bytes < ccm::matvec2_workspace(a->rows, a->cols, b->cols)) return CCM_E_CAPACITY;
  ccm::run_matvec2(*a, *x, *b, *z, *y, ws, to_cuda(stream));
  return launched();
}

ccm_status ccm_matmul(const ccm_matrix* a, const ccm_matrix* b, const ccm_matrix* c, int path,
                      void* ws, size_t ws_bytes, ccm_stream_t stream) {
  if (!valid_in(a) || !valid_in(b) || !valid_out(c) || !ws) return CCM_E_INVAL;
  if (path != CCM_MATMUL_AUTO && path != CCM_MATMUL_TENSOR && path != CCM_MATMUL_CUDACORE)
    return CCM_E_INVAL;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return CCM_E_INVAL;
  if (b->rows != a->cols || c->rows != a->rows || c->cols != b->cols) return CCM_E_SHAPE;
  if (!capacity_ok(c)) return CCM_E_CAPACITY;
  if (ws_bytes < ccm::matmul_workspace(*a, *b)) return CCM_E_CAPACITY;  // <= the shape bound
  int st = ccm::run_matmul(*a, *b, *c, path, ws, to_cuda(stream));
  if (st != CCM_OK) return (ccm_status)st;
  return launched();
}

ccm_status ccm_repack(const ccm_matrix* in, int width, int is_signed, const ccm_matrix* out,
                      uint64_t row_offset, ccm_stream_t stream) {
  if (!valid_in(in) || !valid_out(out)) return CCM_E_INVAL;
  if (width < 1 || width > 64 || (is_signed != 0 && is_signed != 1)) return CCM_E_WIDTH;
  if (out->cols != in->cols || row_offset > out->rows || in->rows > out->rows - row_offset)
    return CCM_E_SHAPE;
  // a non-empty block must start on a word boundary of the output stream
  if (in->rows && (row_offset * in->cols * (uint64_t)width) % 32) return CCM_E_SHAPE;
  if (out->capacity < words_for(out->rows * out->cols, width)) return CCM_E_CAPACITY;
  ccm::run_repack(*in, width, is_signed, *out, row_offset, to_cuda(stream));
  return launched();
}

uint64_t ccm_vlb_index_entries(uint64_t rows, uint64_t cols) {
  return (rows * cols + CCM_VLB_INDEX_STRIDE - 1) / CCM_VLB_INDEX_STRIDE + 1;
}

ccm_status ccm_vlb_pack(const void* dense, int dtype, uint64_t rows, uint64_t cols,
                        ccm_header* hdr, uint32_t* words, uint64_t capacity, uint64_t* index,
                        void* ws, size_t ws_bytes, ccm_stream_t stream) {
  if (!hdr || !ws || !ccm::shape_ok(rows, cols) || (rows * cols && !dense)) return CCM_E_INVAL;
  if (dtype != CCM_I32 && dtype != CCM_I64) return CCM_E_INVAL;
  if (words && !index) return CCM_E_INVAL;
  if (reinterpret_cast<uintptr_t>(hdr) % 16 || reinterpret_cast<uintptr_t>(ws) % 256)
    return CCM_E_INVAL;
  if (ws_bytes < ccm::vlb_workspace(rows * cols)) return CCM_E_CAPACITY;
  ccm::run_vlb_pack(dense, dtype, rows, cols, hdr, words, capacity, index, ws, to_cuda(stream));
  return launched();
}

ccm_status ccm_vlb_unpack(const ccm_header* hdr, const uint32_t* words, uint64_t capacity,
                          const uint64_t* index, uint64_t rows, uint64_t cols, void* dense,
                          int dtype, int32_t* err, ccm_stream_t stream) {
  if (!hdr || !ccm::shape_ok(rows, cols) || (rows * cols && (!words || !index || !dense)))
    return CCM_E_INVAL;
  if (dtype != CCM_I32 && dtype != CCM_I64) return CCM_E_INVAL;
  if (rows * cols == 0) return CCM_OK;
  ccm::run_vlb_unpack(hdr, words, capacity, index, rows, cols, dense, dtype, err,
                      to_cuda(stream));
  return launched();
}

ccm_status ccm_vlb_matvec(const ccm_header* hdr, const uint32_t* words, uint64_t capacity,
                          const uint64_t* index, uint64_t rows, uint64_t cols,
                          const ccm_matrix* x, const ccm_matrix* y, void* ws, size_t ws_bytes,
                          ccm_stream_t stream) {
  if (!hdr || !ws || !valid_in(x) || !valid_out(y) || !ccm::shape_ok(rows, cols))
    return CCM_E_INVAL;
  if (rows * cols && (!words || !index)) return CCM_E_INVAL;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return CCM_E_INVAL;
  if (x->rows != cols || x->cols != 1 || y->rows != rows || y->cols != 1) return CCM_E_SHAPE;
  if (!capacity_ok(y)) return CCM_E_CAPACITY;
  if (ws_bytes < ccm::vlb_matvec_workspace(rows)) return CCM_E_CAPACITY;
  ccm::run_vlb_matvec(hdr, words, capacity, index, rows, cols, *x, *y, ws, to_cuda(stream));
  return launched();
}

ccm_status ccm_header_read(const ccm_header* dev, ccm_header* host, ccm_stream_t stream) {
  if (!dev || !host) return CCM_E_INVAL;
  cudaStream_t s = to_cuda(stream);
  if (cudaMemcpyAsync(host, dev, sizeof(ccm_header), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CCM_E_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CCM_E_CUDA;
  return CCM_OK;
}

ccm_status ccm_gen_uniform(int64_t* out, uint64_t count, uint64_t seed, uint64_t stream_id,
                           uint64_t start, int64_t lo, int64_t hi, ccm_stream_t stream) {
  if (count && !out) return CCM_E_INVAL;
  if (hi < lo) return CCM_E_INVAL;
  if (!count) return CCM_OK;
  ccm::run_gen_uniform(out, count, seed, stream_id, start, lo, hi, to_cuda(stream));
  return launched();
}

ccm_status ccm_gen_poisson(int64_t* out, uint64_t count, uint64_t seed, uint64_t stream_id,
                           uint64_t start, const double* table, uint32_t table_len,
                           ccm_stream_t stream) {
  if ((count && !out) || !table || table_len == 0 || table_len > 4096) return CCM_E_INVAL;
  if (!count) return CCM_OK;
  ccm::run_gen_poisson(out, count, seed, stream_id, start, table, table_len, to_cuda(stream));
  return launched();
}

}  // extern "C"
