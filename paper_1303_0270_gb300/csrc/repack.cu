// repack.cu -- re-pack a packed matrix at a given width and sign mode, at a
// row offset of a larger output (the assembly step of a matvec whose rows are
// split across devices: each device re-packs its block of y at the width all
// blocks agree on, and the disjoint word ranges are then combined).
#include "ccm_device.cuh"
#include "kernels.h"

namespace ccm {
namespace {

constexpr int kThreads = 256;

// Output word W of `out` (nw words): inside the block (words [w0, w0 + bw))
// it is assembled from the fields that overlap it, re-encoded at `width`;
// every other word (the other rows, the bits above the block's last field,
// the pad) is zero.
__global__ void __launch_bounds__(kThreads) k_repack_into(
    const ccm_header* hin, const uint32_t* __restrict__ win, uint64_t in_rows, uint64_t cols,
    uint64_t in_cap, ccm_header* hout, uint32_t* __restrict__ wout, uint64_t out_rows,
    uint64_t row_offset, int width, int is_signed) {
  const HeaderView h = load_header(hin);
  int st = check_header(h, in_rows, cols, in_cap);
  // every value of a b-bit input fits the target when its range does
  if (st == CCM_OK) {
    const bool fits = is_signed ? (h.is_signed ? h.width <= width : h.width < width)
                                : (!h.is_signed && h.width <= width);
    if (!fits) st = CCM_E_WIDTH;
  }
  const uint64_t n_out = out_rows * cols, n_in = in_rows * cols;
  const uint64_t nw = words_for(n_out, width);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    hout->magic = CCM_MAGIC;
    hout->width = width;
    hout->is_signed = is_signed;
    hout->status = st;
    hout->rows = out_rows;
    hout->cols = cols;
    hout->nwords = nw;
    hout->stat_or = 0;
    hout->stat_neg = 0;
    hout->reserved0 = 0;
    hout->reserved1 = 0;
  }
  if (st != CCM_OK) return;
  const uint64_t w0 = row_offset * cols * (uint64_t)width / 32;  // whole words (host-checked)
  const uint64_t bw = data_words(n_in, width);
  const uint64_t mask = field_mask(width);
  const uint64_t stride = (uint64_t)gridDim.x * kThreads;
  for (uint64_t W = (uint64_t)blockIdx.x * kThreads + threadIdx.x; W < nw; W += stride) {
    uint32_t acc = 0;
    if (W >= w0 && W < w0 + bw && n_in) {
      const uint64_t bit0 = (W - w0) * 32;
      uint64_t f = bit0 / (uint64_t)width;
      const uint64_t f_end = umin((bit0 + 31) / (uint64_t)width, n_in - 1);
      for (; f <= f_end; ++f) {
        const int64_t o = (int64_t)(f * (uint64_t)width) - (int64_t)bit0;
        const uint64_t pat = (uint64_t)decode_field(win, f, h.width, h.is_signed) & mask;
        acc |= o >= 0 ? (uint32_t)(pat << o) : (uint32_t)(pat >> (-o));
      }
    }
    wout[W] = acc;
  }
}

}  // namespace

void run_repack(const ccm_matrix& in, int width, int is_signed, const ccm_matrix& out,
                uint64_t row_offset, cudaStream_t st) {
  const uint64_t nw = words_for(out.rows * out.cols, width);
  const int grid = (int)umax(1, umin((nw + kThreads - 1) / kThreads, (uint64_t)num_sms() * 8));
  k_repack_into<<<grid, kThreads, 0, st>>>(in.hdr, in.words, in.rows, in.cols, in.capacity,
                                           out.hdr, out.words, out.rows, row_offset, width,
                                           is_signed);
  note_launch();
}

}  // namespace ccm
