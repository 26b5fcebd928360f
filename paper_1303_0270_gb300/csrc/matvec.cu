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
    // (added to y: a second product term may already be there)
    if (!wide) {
      int64_t acc = 0;
      for (uint64_t j = lane; j < n; j += kWarp) acc += decode_field(wa, row0 + j, ba, sa) * xs[j];
      for (int d = 16; d; d >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, d);
      if (lane == 0) {
        const __int128 t = (__int128)y[i] + acc;
        if (!fits64(t)) ovf = 1;
        y[i] = (int64_t)t;
      }
    } else {
      __int128 acc = 0;
      for (uint64_t j = lane; j < n; j += kWarp)
        acc += (__int128)decode_field(wa, row0 + j, ba, sa) * (__int128)xs[j];
      for (int d = 16; d; d >>= 1) acc += shfl_down_i128(acc, d);
      if (lane == 0) {
        if (!fits64(acc)) ovf = 1;
        const __int128 t = (__int128)y[i] + (int64_t)acc;
        if (!fits64(t)) ovf = 1;
        y[i] = (int64_t)t;
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
namespace rows {
// The x staging image, built once per call: for every 128-column chunk c,
// x in dp4a byte order (144-byte rows) when b <= 8 and b_x <= 8, else int32
// (528-byte rows); then one int per chunk, the sum of its x (the offset-binary
// correction).  One CTA of 128 threads per chunk, grid-stride.
__global__ void __launch_bounds__(128) k_xprep(const ccm_header* out, const ccm_header* ha,
                                               const ccm_header* hx, const uint32_t* __restrict__ wx,
                                               uint64_t n, uint8_t* __restrict__ img) {
  __shared__ int s_part[4];
  if (out->status != CCM_OK) return;
  const int b = ha->width, bx = hx->width, sx = hx->is_signed;
  const bool dp = b <= 8 && bx <= 8;
  const uint32_t nchunks = (uint32_t)(n / kKC);
  int* csum = reinterpret_cast<int*>(img + (uint64_t)nchunks * (dp ? kXPitch8 : kXPitch32));
  const uint32_t f = threadIdx.x;
  for (uint32_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
    const int v = (int)decode_field(wx, (uint64_t)c * kKC + f, bx, sx);
    if (dp)
      img[(uint64_t)c * kXPitch8 + x8_pos_rt(f, b)] = (uint8_t)v;
    else
      reinterpret_cast<int*>(img + (uint64_t)c * kXPitch32)[f] = v;
    int sum = v;
    for (int d = 16; d; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
    if (f % 32 == 0) s_part[f / 32] = sum;
    __syncthreads();
    if (f == 0) csum[c] = s_part[0] + s_part[1] + s_part[2] + s_part[3];
    __syncthreads();
  }
}

int resident_ctas_8(int threads, size_t smem);
int resident_ctas_16(int threads, size_t smem);
int resident_ctas_32(int threads, size_t smem);
void launch_8(const RowArgs& a, bool narrow, unsigned grid, int threads, size_t smem,
              cudaStream_t st);
void launch_16(const RowArgs& a, bool narrow, unsigned grid, int threads, size_t smem,
               cudaStream_t st);
void launch_32(const RowArgs& a, bool narrow, unsigned grid, int threads, size_t smem,
               cudaStream_t st);
int resident_ctas(int bmax, int threads, size_t smem) {
  return bmax <= 8 ? resident_ctas_8(threads, smem)
                   : bmax <= 16 ? resident_ctas_16(threads, smem) : resident_ctas_32(threads, smem);
}
void launch(int bmax, const RowArgs& a, bool narrow, unsigned grid, int threads, size_t smem,
            cudaStream_t st) {
  if (bmax <= 8)
    launch_8(a, narrow, grid, threads, smem, st);
  else if (bmax <= 16)
    launch_16(a, narrow, grid, threads, smem, st);
  else
    launch_32(a, narrow, grid, threads, smem, st);
}
}  // namespace rows
}  // namespace mvf

size_t matvec_workspace(uint64_t m, uint64_t n) {
  // saturates instead of wrapping: a shape this large can never be served
  if (m > kMaxFields || n > kMaxFields) return SIZE_MAX;
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  return up(n * sizeof(int64_t)) + up(m * sizeof(int64_t)) + 256;
}

namespace {

// Launches the kernels of one product term A x, adding it to the int64 y
// scratch `yv` (zeroed by the caller).  `budget`: the bit bound every partial
// sum of this term must stay under for the int64 streaming kernels (63 for
// one term, 62 when two terms are summed).  `xs`: the x region of the
// workspace (8n bytes).
void matvec_term(const ccm_matrix& a, const ccm_matrix& x, const ccm_matrix& y, int64_t* xs,
                 int64_t* yv, int budget, cudaStream_t st) {
  const uint64_t m = a.rows, n = a.cols;
  if (!m || !n) return;  // an empty inner dimension adds 0
  const int bmax_a = width_bound(a.capacity, m * n), bmax_x = width_bound(x.capacity, n);
  // Streaming kernels: row-aligned A (cols % 128 == 0), fields of at most 32
  // bits, x of at most 31, and every partial sum inside the budget.
  const bool aligned = n % mvf::kKC == 0 && bmax_a <= 32 && bmax_x <= 31 &&
                       bmax_a + bmax_x + bitlen_host(n) <= budget;
  const bool narrow = bmax_a + bmax_x + 7 <= 31;
  // Row-streaming kernel when all of x fits in shared memory beside the
  // rings: CTAs of 8 or 4 warps, whichever keeps more warps resident.
  struct RowPlan {
    int warps = 0;
    unsigned grid = 0;
    size_t smem = 0;
    uint64_t resident_warps = 0;
  } rplan;
  if (aligned) {
    const bool bytes = bmax_a <= 8 && bmax_x <= 8;
    const uint64_t xr = (mvf::rows::x_region_bytes(n, bytes) + 15) & ~(uint64_t)15;
    const uint32_t wr = mvf::warp_region_bytes(bmax_a);
    const uint64_t nchunks = n / mvf::kKC;
    const uint64_t T = m * ((nchunks + mvf::rows::kChunksPerStage - 1) /
                            mvf::rows::kChunksPerStage);
    for (int w : {8, 4}) {
      const uint64_t smem = (uint64_t)w * wr + xr;
      if (smem > (uint64_t)max_smem_optin()) continue;
      const int per_sm = mvf::rows::resident_ctas(bmax_a, w * 32, (size_t)smem);
      if (per_sm <= 0) continue;
      const uint64_t need = (T + w - 1) / w;
      const uint64_t grid = umin((uint64_t)num_sms() * per_sm, need);
      const uint64_t rw = grid * w;
      if (rw > rplan.resident_warps) {
        rplan.warps = w;
        rplan.grid = (unsigned)grid;
        rplan.smem = (size_t)smem;
        rplan.resident_warps = rw;
      }
    }
  }
  if (rplan.warps > 0) {
    uint8_t* img = reinterpret_cast<uint8_t*>(xs);  // n * 8 bytes >= the image
    const unsigned gx = (unsigned)umin(n / mvf::kKC, (uint64_t)num_sms() * 8);
    mvf::rows::k_xprep<<<gx, mvf::kKC, 0, st>>>(y.hdr, a.hdr, x.hdr, x.words, n, img);
    note_launch();
    mvf::rows::RowArgs ra{y.hdr, a.hdr, a.words, x.hdr, x.words, m, n, 0u, 0u, yv, img};
    ra.warp_region = mvf::warp_region_bytes(bmax_a);
    ra.x_offset = (uint32_t)((size_t)rplan.warps * ra.warp_region);
    profile_begin(st);
    mvf::rows::launch(bmax_a, ra, narrow, rplan.grid, rplan.warps * 32, rplan.smem, st);
    profile_end(st);
    note_launch();
    return;
  }
  // Column-slab kernel (the slab kernel addresses a warp's 32 rows with
  // 32-bit offsets).  Launch plan for CTAs of `warps` warps: one wave of as
  // many CTAs as stay resident; column slabs split the work when there are
  // fewer row blocks than that, CTAs loop over row blocks when there are
  // more.  A slab's x (int32) must fit in shared memory beside the rings.
  struct Plan {
    int warps;
    uint64_t grid_x, splits, per, resident_warps;
    size_t smem;
  };
  const uint32_t warp_region = mvf::warp_region_bytes(bmax_a);
  const uint64_t groups = n / mvf::kKC;  // 128-column groups
  auto make_plan = [&](int warps) {
    Plan p{warps, 0, 0, 0, 0, 0};
    const size_t stage_region = (size_t)warps * warp_region;
    const size_t cap = (size_t)max_smem_optin();
    if (stage_region + mvf::kKC * sizeof(int) > cap) return p;
    const uint64_t per_cap = (cap - stage_region) / (mvf::kKC * sizeof(int));
    const uint64_t row_blocks = (m + 32 * warps - 1) / (32 * warps);
    const int per_sm0 = mvf::resident_ctas(bmax_a, warps * 32,
                                           stage_region + umin(n, 1024) * sizeof(int));
    const uint64_t resident0 = (uint64_t)num_sms() * (uint64_t)(per_sm0 > 0 ? per_sm0 : 1);
    uint64_t splits = umin(umax(resident0 / umax(row_blocks, 1), 1), groups);
    splits = umin(splits, 65535);
    p.per = umin((groups + splits - 1) / splits, per_cap);
    p.splits = (groups + p.per - 1) / p.per;
    p.smem = stage_region + p.per * mvf::kKC * sizeof(int);
    const int per_sm = mvf::resident_ctas(bmax_a, warps * 32, p.smem);
    const uint64_t resident = (uint64_t)num_sms() * (uint64_t)(per_sm > 0 ? per_sm : 1);
    p.grid_x = umin(row_blocks, umax(resident / p.splits, 1));
    p.resident_warps = umin(p.grid_x * p.splits, resident) * warps;
    return p;
  };
  if (aligned && n * (uint64_t)bmax_a < (1ull << 30)) {
    Plan plan = make_plan(8);
    const Plan p4 = make_plan(4);
    if (p4.resident_warps > plan.resident_warps) plan = p4;
    if (plan.per > 0) {
      const int warps = plan.warps;
      mvf::Args args{y.hdr, a.hdr, a.words, x.hdr, x.words, m, n,
                     (uint32_t)(plan.per * mvf::kKC), 0u, 0u, yv};
      args.stage_region = (uint32_t)((size_t)warps * warp_region);
      args.warp_region = warp_region;
      dim3 grid((unsigned)plan.grid_x, (unsigned)plan.splits);
      profile_begin(st);
      if (bmax_a <= 8)
        mvf::launch_matvec_fast8(args, narrow, grid, warps * 32, plan.smem, st);
      else if (bmax_a <= 16)
        mvf::launch_matvec_fast16(args, narrow, grid, warps * 32, plan.smem, st);
      else
        mvf::launch_matvec_fast32(args, narrow, grid, warps * 32, plan.smem, st);
      profile_end(st);
      note_launch();
      return;
    }
  }
  // generic: x decoded to int64, one warp per row, 128-bit sums when needed
  int g = (int)umin((n + 255) / 256, (uint64_t)num_sms() * 4);
  k_decode_vec<<<g, 256, 0, st>>>(y.hdr, x.hdr, x.words, n, xs);
  note_launch();
  g = (int)umin((m + 7) / 8, (uint64_t)num_sms() * 8);
  profile_begin(st);
  k_matvec_rows<<<g, kMvThreads, 0, st>>>(y.hdr, a.hdr, a.words, x.hdr, xs, m, n, yv);
  profile_end(st);
  note_launch();
}

InitArgs matvec_init(const ccm_matrix& a, const ccm_matrix& x, const ccm_matrix& y, int64_t* yv) {
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
  ia.zero_ptr = yv;
  ia.zero_count = y.rows;
  return ia;
}

}  // namespace

void run_matvec(const ccm_matrix& a, const ccm_matrix& x, const ccm_matrix& y, void* ws,
                cudaStream_t st) {
  const uint64_t n_a = a.rows * a.cols;
  if (mvs::stream_applies(a.rows, a.cols, width_bound(a.capacity, n_a),
                          width_bound(x.capacity, a.cols))) {
    mvs::run_stream(a, x, y, ws, st);
    return;
  }
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  int64_t* xs = (int64_t*)ws;
  int64_t* yv = (int64_t*)((char*)ws + up(a.cols * sizeof(int64_t)));
  launch_init(matvec_init(a, x, y, yv), st);
  matvec_term(a, x, y, xs, yv, 63, st);
  run_pack_scratch(yv, y, st);
}

size_t matvec2_workspace(uint64_t m, uint64_t n1, uint64_t n2) {
  return matvec_workspace(m, umax(n1, n2));
}

void run_matvec2(const ccm_matrix& a, const ccm_matrix& x, const ccm_matrix& b,
                 const ccm_matrix& z, const ccm_matrix& y, void* ws, cudaStream_t st) {
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  int64_t* xs = (int64_t*)ws;
  int64_t* yv = (int64_t*)((char*)ws + up(umax(a.cols, b.cols) * sizeof(int64_t)));
  launch_init(matvec_init(a, x, y, yv), st);
  launch_check(b, z, y.hdr, st);
  // both products summed into one int64 scratch, each kept below 2^62
  matvec_term(a, x, y, xs, yv, 62, st);
  matvec_term(b, z, y, xs, yv, 62, st);
  run_pack_scratch(yv, y, st);
}

}  // namespace ccm
