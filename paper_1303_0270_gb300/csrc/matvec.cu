// matvec.cu -- y = A x on the compressed form.  The exact product
// y_i = sum_j a_ij x_j (the same integers as on the uncompressed matrix,
// Introduction) is accumulated in int64 when the operand widths bound every
// partial sum below 2^63, in 128-bit integers otherwise; y is then re-packed
// at its own width by the pack engine.
//
// Launch sequence on the stream:
//   k_init          validate A (m x n) and x (n x 1), clear y's header and
//                   the int64 y scratch
//   k_matvec_fast   when cols % 128 == 0 and the buffers bound both widths
//                   by 31/32 bits (see matvec_fast.cuh); otherwise
//     k_decode_vec  x -> int64 scratch, and
//     k_matvec_rows one warp per row, fields decoded from A's words
//   k_stats, k_pack y scratch -> packed y
//
// The host cannot see the widths (they live in device headers), but a
// buffer of `capacity` words can only hold a matrix of width
// <= 32*capacity/(rows*cols); that bound picks the kernel and sizes its
// shared memory.
#include "pack_engine.cuh"
#include "kernels.h"
#include "matvec_fast.cuh"

namespace ccm {

namespace {

constexpr int kMvThreads = 256;

// Every partial sum of n products of a b_a-bit and a b_x-bit integer stays
// below 2^(b_a + b_x + bitlen(n)) in magnitude.
__device__ __forceinline__ bool needs_wide(int ba, int bx, uint64_t n) {
  return ba + bx + bitlen64(n) > 63;
}

__global__ void __launch_bounds__(256) k_decode_vec(const ccm_header* out, const ccm_header* hx,
                                                    const uint32_t* __restrict__ wx, uint64_t n,
                                                    int64_t* __restrict__ xs) {
  if (out->status != CCM_OK) return;
  const int b = hx->width, sgn = hx->is_signed;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += stride)
    xs[j] = decode_field(wx, j, b, sgn);
}

__device__ __forceinline__ bool fits64(__int128 v) {
  return v >= -((__int128)1 << 63) && v < ((__int128)1 << 63);
}

__device__ __forceinline__ __int128 shfl_down_i128(__int128 v, int d) {
  uint64_t lo = (uint64_t)v, hi = (uint64_t)(v >> 64);
  lo = __shfl_down_sync(0xffffffffu, lo, d);
  hi = __shfl_down_sync(0xffffffffu, hi, d);
  return (__int128)(((unsigned __int128)hi << 64) | lo);
}

__global__ void __launch_bounds__(kMvThreads) k_matvec_rows(ccm_header* out, const ccm_header* ha,
                                                            const uint32_t* __restrict__ wa,
                                                            const ccm_header* hx,
                                                            const int64_t* __restrict__ xs,
                                                            uint64_t m, uint64_t n,
                                                            int64_t* __restrict__ y) {
  if (out->status != CCM_OK) return;
  const int ba = ha->width, sa = ha->is_signed;
  const bool wide = needs_wide(ba, hx->width, n);
  const int lane = threadIdx.x % kWarp;
  const uint64_t warps = (uint64_t)gridDim.x * (kMvThreads / kWarp);
  int ovf = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * (kMvThreads / kWarp) + threadIdx.x / kWarp; i < m;
       i += warps) {
    const uint64_t row0 = i * n;
    if (!wide) {
      int64_t acc = 0;
      for (uint64_t j = lane; j < n; j += kWarp) acc += decode_field(wa, row0 + j, ba, sa) * xs[j];
      for (int d = 16; d; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
      if (lane == 0) y[i] = acc;
    } else {
      __int128 acc = 0;
      for (uint64_t j = lane; j < n; j += kWarp)
        acc += (__int128)decode_field(wa, row0 + j, ba, sa) * (__int128)xs[j];
      for (int d = 16; d; d >>= 1) acc += shfl_down_i128(acc, d);
      if (lane == 0) {
        if (!fits64(acc)) ovf = 1;
        y[i] = (int64_t)acc;
      }
    }
  }
  if (ovf) set_status(out, CCM_E_OVERFLOW);
}

}  // namespace

namespace mvf {
int resident_ctas_8(int threads, size_t smem);
int resident_ctas_16(int threads, size_t smem);
int resident_ctas_32(int threads, size_t smem);
int resident_ctas(int bmax, int threads, size_t smem) {
  return bmax <= 8 ? resident_ctas_8(threads, smem)
                   : bmax <= 16 ? resident_ctas_16(threads, smem) : resident_ctas_32(threads, smem);
}
}  // namespace mvf

size_t matvec_workspace(uint64_t m, uint64_t n) {
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  return up(n * sizeof(int64_t)) + up(m * sizeof(int64_t)) + 256;
}

void run_matvec(const ccm_matrix& a, const ccm_matrix& x, const ccm_matrix& y, void* ws,
                cudaStream_t st) {
  const uint64_t m = a.rows, n = a.cols;
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  int64_t* xs = (int64_t*)ws;
  int64_t* yv = (int64_t*)((char*)ws + up(n * sizeof(int64_t)));
  InitArgs ia{};
  ia.out = y.hdr;
  ia.in0 = a.hdr;
  ia.in0_rows = a.rows;
  ia.in0_cols = a.cols;
  ia.in0_capacity = a.capacity;
  ia.in1 = x.hdr;
  ia.in1_rows = x.rows;
  ia.in1_cols = x.cols;
  ia.in1_capacity = x.capacity;
  ia.out_rows = y.rows;
  ia.out_cols = y.cols;
  if (n == 0) {  // an empty inner dimension gives y = 0
    ia.zero_ptr = yv;
    ia.zero_count = m;
  }
  const int bmax_a = width_bound(a.capacity, m * n), bmax_x = width_bound(x.capacity, n);
  const bool fast = m && n && n % mvf::kKC == 0 && bmax_a <= 32 && bmax_x <= 31 &&
                    bmax_a + bmax_x + bitlen_host(n) <= 63;
  if (fast) ia.zero_ptr = yv, ia.zero_count = m;
  launch_init(ia, st);
  if (fast) {
    const int warps = bmax_a <= 12 ? 8 : 4;
    const uint64_t row_blocks = (m + 32 * warps - 1) / (32 * warps);
    const uint64_t groups = n / mvf::kKC;  // 128-column groups
    const size_t stage_region = (size_t)warps * mvf::kStages * 32 * mvf::pitch_bytes(bmax_a);
    // one wave: as many CTAs as stay resident; column slabs split the work
    // when there are fewer row blocks than that, CTAs loop over row blocks
    // when there are more
    const int per_sm0 = mvf::resident_ctas(bmax_a, warps * 32,
                                           stage_region + umin(n, 1024) * sizeof(int));
    const uint64_t resident0 = (uint64_t)num_sms() * (uint64_t)(per_sm0 > 0 ? per_sm0 : 1);
    uint64_t splits = umin(umax(resident0 / umax(row_blocks, 1), 1), groups);
    splits = umin(splits, 65535);
    const uint64_t per = (groups + splits - 1) / splits;
    splits = (groups + per - 1) / per;
    const int per_sm = mvf::resident_ctas(bmax_a, warps * 32,
                                          stage_region + per * mvf::kKC * sizeof(int));
    const uint64_t resident = (uint64_t)num_sms() * (uint64_t)(per_sm > 0 ? per_sm : 1);
    const uint64_t grid_x = umin(row_blocks, umax(resident / splits, 1));
    mvf::Args args{y.hdr, a.hdr, a.words, x.hdr, x.words, m, n,
                   (uint32_t)(per * mvf::kKC), 0u, yv};
    args.stage_region = (uint32_t)stage_region;
    const size_t smem = args.stage_region + per * mvf::kKC * sizeof(int);
    dim3 grid((unsigned)grid_x, (unsigned)splits);
    profile_begin(st);
    const bool narrow = bmax_a + bmax_x + 7 <= 31;
    if (bmax_a <= 8)
      mvf::launch_matvec_fast8(args, narrow, grid, warps * 32, smem, st);
    else if (bmax_a <= 16)
      mvf::launch_matvec_fast16(args, narrow, grid, warps * 32, smem, st);
    else
      mvf::launch_matvec_fast32(args, narrow, grid, warps * 32, smem, st);
    profile_end(st);
    note_launch();
    run_pack_scratch(yv, y, st);
    return;
  }
  if (n) {
    int g = (int)umin((n + 255) / 256, (uint64_t)num_sms() * 4);
    k_decode_vec<<<g, 256, 0, st>>>(y.hdr, x.hdr, x.words, n, xs);
    note_launch();
  }
  if (m && n) {
    int g = (int)umin((m + 7) / 8, (uint64_t)num_sms() * 8);
    profile_begin(st);
    k_matvec_rows<<<g, kMvThreads, 0, st>>>(y.hdr, a.hdr, a.words, x.hdr, xs, m, n, yv);
    profile_end(st);
    note_launch();
  }
  run_pack_scratch(yv, y, st);
}

}  // namespace ccm
