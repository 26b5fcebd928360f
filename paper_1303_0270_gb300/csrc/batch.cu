// batch.cu -- y_i = A_i x_i for thousands of packed matrices of uneven
// shapes and widths in one persistent launch.
//
// Work unit: a run of consecutive 32-field row segments of one matrix.  Row i
// of an m x n matrix is cut into ceil(n / 32) segments of up to 32 fields; a
// lane owns one segment.  A warp takes 32 consecutive segments at a time (a
// chunk: one contiguous word range) and streams its chunks through a ring of
// K = 2 or 4 cp.async slots in shared memory, so the words of the next K - 1
// chunks are in flight while the current one is decoded.  A segment starts at an
// arbitrary bit, so the lane reads the b + 1 words that cover it,
// funnel-shifts them once to the segment's start and then decodes its fields
// with shifts fixed at compile time (the width is dispatched per unit on the
// GPU).  Every x is decoded once, by the initialisation kernel, into an int32
// image in workspace with the [f/4][segment][f%4] layout (zero past the row's
// end), so the four x values a lane needs next are one 16-byte load
// (L1-resident while a matrix's units run).  Lanes of a
// warp hold consecutive segments; a segmented shuffle reduction keyed by row
// leaves each row's partial sum in its first lane, which adds it to the int64
// y scratch with one atomic.
//
// Persistent CTAs take units from an atomic ticket.  The CTA that finishes
// the last unit of a matrix (per-matrix completion counter) re-packs that
// matrix's y at its exact width (width rule of Eq. 1 with the two's
// complement reading) and writes y's header -- so the whole batch is one
// launch after a small initialisation kernel, and both can be captured in a
// CUDA graph.
#include <cstring>
#include <vector>

#include "ccm_device.cuh"
#include "kernels.h"

namespace ccm {
namespace bt {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxCols = 8192;      // x of at most 8192 entries per matrix (32 KB of shared)

// Shared words of one ring slot for A widths up to bmax: a chunk covers at
// most 32 * 32 fields, i.e. 32 bmax + 2 words (the lanes read one word past
// their segment), plus one padding word per 32 (stage_pos).
__host__ __device__ constexpr uint32_t slot_words(int bmax) {
  return (uint32_t)((33 * bmax + 4 + 3) & ~3);
}

struct Mat {
  const ccm_header* ha;
  const uint32_t* wa;
  const ccm_header* hx;
  const uint32_t* wx;
  ccm_header* hy;
  uint32_t* wy;
  uint64_t a_cap, x_cap, y_cap;
  uint32_t m, n;
  uint64_t y_off;      // offset of this matrix's rows in the int64 y scratch
  uint32_t units;      // work units of this matrix
  uint64_t x_off;      // offset of this matrix's x image (ints; a multiple of 32)
  uint32_t nseg_row;   // segments per row, ceil(n / 32)
  uint32_t dm, ds1, ds2;  // v / nseg_row as a multiply and shifts (DivSeg)
  uint32_t pad;
};

// Unsigned 32-bit division by a run-time invariant d >= 1 with one high
// multiply, after Granlund and Montgomery, "Division by invariant integers
// using multiplication" (1994), Fig. 4.1: with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, q = (t + ((v - t) >> min(l, 1))) >>
// max(l - 1, 0) where t = mulhi(m, v), for every 32-bit v.
struct DivSeg {
  uint32_t m, s1, s2;
  static DivSeg make(uint32_t d) {
    int l = 0;
    while (l < 32 && (1ull << l) < d) ++l;
    const uint64_t m = (((1ull << l) - d) << 32) / d + 1;
    return {(uint32_t)m, (uint32_t)(l < 1 ? l : 1), (uint32_t)(l > 1 ? l - 1 : 0)};
  }
};

__device__ __forceinline__ uint32_t div_seg(const Mat& M, uint32_t v) {
  const uint32_t t = __umulhi(v, M.dm);
  return (t + ((v - t) >> M.ds1)) >> M.ds2;
}

struct Unit {
  uint32_t mat;
  uint32_t seg0;   // first segment (row-major numbering within the matrix)
  uint32_t nseg;   // number of segments
  uint32_t pad;
};

struct Args {
  const Mat* mats;
  const Unit* units;
  uint32_t nmats, nunits;
  int64_t* yscratch;
  uint32_t* ticket;     // unit dispenser
  uint32_t* done;       // per-matrix completed units
  int* ximage;          // decoded x of every matrix (Mat::x_off)
  uint32_t slot;        // shared words of one ring slot (slot_words(bmax))
  uint32_t bmax;        // widest A the slots hold
  uint32_t slots;       // ring slots per warp: 2 or 4
};

__device__ __forceinline__ int stage_pos(int w, int b) { return (b & 1) ? w : w + (w >> 5); }

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The word range of the warp's chunk starting at segment `base` of unit u.
struct Chunk {
  uint64_t w_first;  // first word (holds the first segment's first bit)
  uint32_t nwords;   // words through the one after the last segment's last bit
};

template <int B>
__device__ __forceinline__ Chunk chunk_of(const Mat& M, const Unit& u, uint32_t base) {
  const uint32_t n = M.n, nsr = M.nseg_row;
  const uint32_t first_id = u.seg0 + base;
  const uint32_t frow = div_seg(M, first_id), fs = first_id - frow * nsr;
  const uint64_t w_first = (((uint64_t)frow * n + 32 * fs) * B) >> 5;
  const uint32_t last = min(base + 32, u.nseg) - 1 + u.seg0;
  const uint32_t lrow = div_seg(M, last), ls = last - lrow * nsr;
  const uint64_t end_bit = ((uint64_t)lrow * n + min(n, 32 * ls + 32)) * B;
  return {w_first, (uint32_t)(((end_bit + 31) >> 5) - w_first) + 1};
}

// cp.async of a chunk's words into a slot: the words inside the matrix's
// data are copied, the rest of the chunk (past the data, at the matrix's
// end) is zero-filled.  Word w goes to stage_pos(w), so from one lane's
// word to its next (32 on) the destination steps by 32 or 33 words.
template <int B>
__device__ __forceinline__ void issue_chunk(const uint32_t* __restrict__ wa, uint64_t dw, Chunk c,
                                            uint32_t* slot, int lane) {
  const uint32_t nin =
      (uint32_t)min((uint64_t)c.nwords, dw > c.w_first ? dw - c.w_first : (uint64_t)0);
  constexpr unsigned kStep = 4 * ((B & 1) ? 32 : 33);
  unsigned dst = (unsigned)__cvta_generic_to_shared(slot) + 4 * lane;  // stage_pos(lane) = lane
  const uint32_t* src = wa + c.w_first + lane;
  uint32_t w = lane;
  for (; w < nin; w += 32, src += 32, dst += kStep)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst), "l"(src) : "memory");
  for (; w < c.nwords; w += 32, dst += kStep)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, 0;\n" ::"r"(dst), "l"(wa) : "memory");
}

// ---------------------------------------------------------------------------
// Initialisation: validate inputs, write y headers, clear counters and the
// y scratch.
// ---------------------------------------------------------------------------
__global__ void k_batch_init(Args a) {
  __shared__ int s_st;
  const uint32_t i = blockIdx.x;  // one block per matrix
  const Mat& M = a.mats[i];
  if (threadIdx.x == 0) {
    int st = check_input(M.ha, M.m, M.n, M.a_cap);
    if (st == CCM_OK) st = check_input(M.hx, M.n, 1, M.x_cap);
    // widths the kernel handles, and sums that provably fit int64
    if (st == CCM_OK && (M.ha->width > (int)a.bmax || M.hx->width > 31 ||
                         M.ha->width + M.hx->width + bitlen64(M.n) > 63))
      st = CCM_E_WIDTH;
    ccm_header* y = M.hy;
    y->magic = CCM_MAGIC;
    y->width = 0;
    y->is_signed = 0;
    y->status = st;
    y->rows = M.m;
    y->cols = 1;
    y->nwords = 0;
    y->stat_or = 0;
    y->stat_neg = 0;
    a.done[i] = 0;
    if (i == 0) *a.ticket = 0;
    s_st = st;
  }
  for (uint32_t r = threadIdx.x; r < M.m; r += blockDim.x) a.yscratch[M.y_off + r] = 0;
  __syncthreads();
  if (s_st != CCM_OK) return;
  // x -> image, layout [f/4][segment][f%4], zero past n
  const int bx = M.hx->width, sx = M.hx->is_signed;
  const uint32_t nsr = M.nseg_row;
  int* xi = a.ximage + M.x_off;
  for (uint32_t j = threadIdx.x; j < nsr * 32; j += blockDim.x) {
    const uint32_t seg = j / 32, f = j % 32;
    xi[((f / 4) * nsr + seg) * 4 + (f % 4)] = j < M.n ? (int)decode_field(M.wx, j, bx, sx) : 0;
  }
}

// ---------------------------------------------------------------------------
// One unit at compile-time width B.
// ---------------------------------------------------------------------------
template <int B, bool SGN, int K>
__device__ __noinline__ void run_unit(const Mat& M, const Unit& u, const int4* __restrict__ x4,
                                      uint32_t* stage, uint32_t slot_w, int64_t* ys) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t n = M.n, nsr = M.nseg_row;
  const uint64_t dw = data_words((uint64_t)M.m * n, B);
  constexpr uint32_t kStep = kWarps * 32;  // segments between a warp's chunks
  uint32_t base = warp * 32;
  // the first K - 1 chunks in flight (one commit group each, empty or not)
#pragma unroll
  for (int p = 0; p < K - 1; ++p) {
    const uint32_t bp = base + p * kStep;
    if (bp < u.nseg) issue_chunk<B>(M.wa, dw, chunk_of<B>(M, u, bp), stage + p * slot_w, lane);
    cp_async_commit();
  }
  for (uint32_t k = 0; base < u.nseg; base += kStep, ++k) {
    // K - 1 chunks in flight while this one is decoded
    const uint32_t nb = base + (K - 1) * kStep;
    if (nb < u.nseg)
      issue_chunk<B>(M.wa, dw, chunk_of<B>(M, u, nb), stage + ((k + K - 1) % K) * slot_w, lane);
    cp_async_commit();
    cp_async_wait<K - 1>();  // chunk k has landed (groups complete in order)
    __syncwarp();
    const uint64_t w_first = chunk_of<B>(M, u, base).w_first;
    const uint32_t* sg = stage + (k % K) * slot_w;
    // the warp's 32 consecutive segments; lane -> (row, segment in the row)
    const uint32_t id = u.seg0 + base + lane;
    const bool live = base + lane < u.nseg;
    const uint32_t q = div_seg(M, id);
    const uint32_t row = live ? q : 0xffffffffu;
    const uint32_t s = live ? id - q * nsr : 0;
    const uint64_t bit = ((uint64_t)q * n + 32 * s) * B;
    long long acc = 0;
    if (live) {
      const int wo = (int)((bit >> 5) - w_first), s0 = (int)(bit & 31);
      uint32_t w[B + 1];
#pragma unroll
      for (int j = 0; j <= B; ++j) w[j] = sg[stage_pos(wo + j, B)];
#pragma unroll
      for (int j = 0; j < B; ++j) w[j] = __funnelshift_r(w[j], w[j + 1], s0);
      const int4* xv = x4 + s;  // [f/4][segment] of int4 (the matrix's image)
      // Fields past the row's end meet x = 0 (x is zero-padded to whole
      // segments), so no per-field bound is needed.
#pragma unroll
      for (int f4 = 0; f4 < 8; ++f4) {
        const int4 xq = __ldg(xv + f4 * nsr);
        const int xa[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
          const int f = 4 * f4 + qq;
          const int b0 = f * B, wi = b0 >> 5, sh = b0 & 31;
          const uint32_t t =
              (sh + B <= 32) ? (w[wi] >> sh) : __funnelshift_r(w[wi], w[wi + 1], sh);
          if constexpr (B == 32 && !SGN) {
            acc += (long long)t * xa[qq];
          } else {
            int v;  // the field as a 32-bit integer
            if constexpr (B == 32)
              v = (int)t;
            else if constexpr (SGN)
              v = (int)(t << (32 - B)) >> (32 - B);
            else
              v = (int)(t & ((1u << B) - 1u));
            acc += (long long)v * (long long)xa[qq];  // 32 x 32 -> 64 multiply-add
          }
        }
      }
    }
    __syncwarp();  // slot k % K is refilled by the issue of chunk k + K
    // segmented reduction by row: the first lane of each row gets the total
    uint32_t r = row;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const long long o = __shfl_down_sync(0xffffffffu, acc, d);
      const uint32_t ro = __shfl_down_sync(0xffffffffu, r, d);
      if (lane + d < 32 && ro == r) acc += o;
    }
    const uint32_t rprev = __shfl_up_sync(0xffffffffu, r, 1);
    if (live && (lane == 0 || rprev != r))
      atomicAdd(reinterpret_cast<unsigned long long*>(ys + row), (unsigned long long)acc);
  }
  cp_async_wait<0>();
}

// Re-pack y of one matrix (m <= 2^31 values in scratch) at its exact width;
// the whole CTA takes part.
__device__ void pack_y(const Mat& M, const int64_t* __restrict__ ys, uint64_t* s_or,
                       uint32_t* s_neg) {
  const uint32_t m = M.m;
  uint64_t orv = 0;
  uint32_t neg = 0;
  for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
    const int64_t v = __ldcg(ys + i);
    orv |= fold(v);
    neg |= (uint32_t)(v < 0);
  }
  orv = warp_or64(orv);
  neg = __reduce_or_sync(0xffffffffu, neg);
  if (threadIdx.x % 32 == 0) {
    s_or[threadIdx.x / 32] = orv;
    s_neg[threadIdx.x / 32] = neg;
  }
  __syncthreads();
  orv = 0;
  neg = 0;
  for (int k = 0; k < kWarps; ++k) {
    orv |= s_or[k];
    neg |= s_neg[k];
  }
  const int b = width_from_stats(orv, neg);
  const uint64_t nw = words_for(m, b), dw = data_words(m, b);
  const bool fits = nw <= M.y_cap;
  if (threadIdx.x == 0) {
    ccm_header* h = M.hy;
    h->stat_or = orv;
    h->stat_neg = neg;
    h->width = b;
    h->is_signed = neg ? 1 : 0;
    h->nwords = nw;
    if (!fits) h->status = CCM_E_CAPACITY;
  }
  if (!fits) return;
  const uint64_t mask = field_mask(b);
  for (uint64_t w = threadIdx.x; w < nw; w += blockDim.x) {
    uint32_t acc = 0;
    if (w < dw) {
      const uint64_t bit0 = w * 32;
      uint64_t f = bit0 / b;
      const uint64_t f_end = min((bit0 + 31) / b, (uint64_t)m - 1);
      for (; f <= f_end; ++f) {
        const uint64_t pat = (uint64_t)__ldcg(ys + f) & mask;
        const int64_t o = (int64_t)(f * b) - (int64_t)bit0;
        acc |= o >= 0 ? (uint32_t)(pat << o) : (uint32_t)(pat >> (-o));
      }
    }
    M.wy[w] = acc;
  }
}

// Dynamic shared memory: each warp's two ring slots.
__global__ void __launch_bounds__(kThreads) k_batch_mv(Args a) {
  extern __shared__ __align__(16) uint32_t s_slots[];
  __shared__ uint32_t s_unit;
  __shared__ int s_last;
  __shared__ uint64_t s_or[kWarps];
  __shared__ uint32_t s_neg[kWarps];
  for (;;) {
    if (threadIdx.x == 0) s_unit = atomicAdd(a.ticket, 1u);
    __syncthreads();
    const uint32_t ui = s_unit;
    if (ui >= a.nunits) break;
    const Unit u = a.units[ui];
    const Mat& M = a.mats[u.mat];
    const bool ok = M.hy->status == CCM_OK;  // validated by k_batch_init
    if (ok) {
      const int b = M.ha->width, sgn = M.ha->is_signed;
      int64_t* ys = a.yscratch + M.y_off;
      uint32_t* stage = s_slots + (threadIdx.x / 32) * a.slots * a.slot;
      const int4* x4 = reinterpret_cast<const int4*>(a.ximage + M.x_off);
      switch (4 * b + 2 * sgn + (a.slots == 4 ? 1 : 0)) {
#define CCM_BT_CASE(B)                                                                    \
  case 4 * B: run_unit<B, false, 2>(M, u, x4, stage, a.slot, ys); break;      \
  case 4 * B + 1: run_unit<B, false, 4>(M, u, x4, stage, a.slot, ys); break;  \
  case 4 * B + 2: run_unit<B, true, 2>(M, u, x4, stage, a.slot, ys); break;   \
  case 4 * B + 3: run_unit<B, true, 4>(M, u, x4, stage, a.slot, ys); break;
        CCM_BT_CASE(1) CCM_BT_CASE(2) CCM_BT_CASE(3) CCM_BT_CASE(4) CCM_BT_CASE(5)
        CCM_BT_CASE(6) CCM_BT_CASE(7) CCM_BT_CASE(8) CCM_BT_CASE(9) CCM_BT_CASE(10)
        CCM_BT_CASE(11) CCM_BT_CASE(12) CCM_BT_CASE(13) CCM_BT_CASE(14) CCM_BT_CASE(15)
        CCM_BT_CASE(16) CCM_BT_CASE(17) CCM_BT_CASE(18) CCM_BT_CASE(19) CCM_BT_CASE(20)
        CCM_BT_CASE(21) CCM_BT_CASE(22) CCM_BT_CASE(23) CCM_BT_CASE(24) CCM_BT_CASE(25)
        CCM_BT_CASE(26) CCM_BT_CASE(27) CCM_BT_CASE(28) CCM_BT_CASE(29) CCM_BT_CASE(30)
        CCM_BT_CASE(31) CCM_BT_CASE(32)
#undef CCM_BT_CASE
        default: break;
      }
    }
    // completion of the unit; the CTA that completes a matrix packs its y
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = atomicAdd(a.done + u.mat, 1u) + 1 == M.units;
    __syncthreads();
    if (s_last && ok) {
      __threadfence();
      pack_y(M, a.yscratch + M.y_off, s_or, s_neg);
    }
    __syncthreads();
  }
}

}  // namespace bt
}  // namespace ccm

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace ccm {
namespace bt {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// x image of an n-column matrix: whole 32-field segments.
uint64_t x_image_ints(uint64_t cols) { return (cols + 31) / 32 * 32; }

// Workspace: int64 y scratch, per-matrix done counters, the ticket, x images.
size_t ws_done(uint64_t yrows) { return align256(yrows * 8); }
size_t ws_ticket(uint64_t yrows, uint32_t count) {
  return ws_done(yrows) + align256((size_t)count * 4);
}
size_t ws_ximage(uint64_t yrows, uint32_t count) { return ws_ticket(yrows, count) + 256; }
size_t ws_bytes(uint64_t yrows, uint32_t count, uint64_t xints) {
  return ws_ximage(yrows, count) + align256(xints * 4);
}

struct Layout {
  uint32_t nmats = 0, nunits = 0;
  uint64_t yrows = 0;
  size_t mats_off = 0, units_off = 0, bytes = 0;
};

uint64_t segments_of(const ccm_batch_entry& e) { return e.a.rows * ((e.a.cols + 31) / 32); }

int validate(const ccm_batch_entry& e) {
  const ccm_matrix &a = e.a, &x = e.x, &y = e.y;
  if (!a.hdr || !x.hdr || !y.hdr) return CCM_E_INVAL;
  if (x.rows != a.cols || x.cols != 1 || y.rows != a.rows || y.cols != 1) return CCM_E_SHAPE;
  if (a.cols > (uint64_t)kMaxCols || a.rows >= (1ull << 31)) return CCM_E_SHAPE;
  const uint64_t n = a.rows * a.cols;
  if (y.capacity < words_for(y.rows, 1)) return CCM_E_CAPACITY;
  auto al = [](const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; };
  if (!al(a.hdr) || !al(x.hdr) || !al(y.hdr) || !al(a.words) || !al(x.words) || !al(y.words))
    return CCM_E_INVAL;
  if ((n && !a.words) || (a.cols && !x.words) || (y.capacity && !y.words)) return CCM_E_INVAL;
  return CCM_OK;
}

Layout layout(const ccm_batch_entry* e, int count, uint32_t unit_segs) {
  Layout L;
  L.nmats = (uint32_t)count;
  uint64_t units = 0;
  for (int i = 0; i < count; ++i) {
    const uint64_t s = segments_of(e[i]);
    units += s ? (s + unit_segs - 1) / unit_segs : 1;
    L.yrows += e[i].a.rows;
  }
  L.nunits = (uint32_t)units;
  L.mats_off = align256(sizeof(ccm_batch_info));
  L.units_off = L.mats_off + align256(sizeof(Mat) * (size_t)count);
  L.bytes = L.units_off + align256(sizeof(Unit) * (size_t)units);
  return L;
}

}  // namespace bt
}  // namespace ccm

extern "C" {

size_t ccm_batch_plan_bytes(const ccm_batch_entry* entries, int count, uint32_t unit_segments) {
  if (!entries || count <= 0 || unit_segments == 0) return 0;
  return ccm::bt::layout(entries, count, unit_segments).bytes;
}

size_t ccm_batch_workspace_bytes(const ccm_batch_entry* entries, int count) {
  if (!entries || count <= 0) return 0;
  uint64_t yrows = 0, xints = 0;
  for (int i = 0; i < count; ++i) {
    yrows += entries[i].a.rows;
    xints += ccm::bt::x_image_ints(entries[i].a.cols);
  }
  return ccm::bt::ws_bytes(yrows, (uint32_t)count, xints);
}

ccm_status ccm_batch_plan(const ccm_batch_entry* entries, int count, uint32_t unit_segments,
                          void* plan, size_t plan_bytes, ccm_batch_info* info) {
  using namespace ccm::bt;
  if (!entries || count <= 0 || !plan || !info || unit_segments == 0) return CCM_E_INVAL;
  if (unit_segments % 32) return CCM_E_INVAL;
  for (int i = 0; i < count; ++i) {
    int st = validate(entries[i]);
    if (st != CCM_OK) return (ccm_status)st;
  }
  Layout L = layout(entries, count, unit_segments);
  if (plan_bytes < L.bytes || reinterpret_cast<uintptr_t>(plan) % 256) return CCM_E_CAPACITY;
  std::vector<uint8_t> host(L.bytes, 0);
  Mat* mats = reinterpret_cast<Mat*>(host.data() + L.mats_off);
  Unit* units = reinterpret_cast<Unit*>(host.data() + L.units_off);
  uint64_t yoff = 0, xoff = 0, u = 0;
  for (int i = 0; i < count; ++i) {
    const ccm_batch_entry& e = entries[i];
    Mat& M = mats[i];
    M.ha = e.a.hdr;
    M.wa = e.a.words;
    M.hx = e.x.hdr;
    M.wx = e.x.words;
    M.hy = e.y.hdr;
    M.wy = e.y.words;
    M.a_cap = e.a.capacity;
    M.x_cap = e.x.capacity;
    M.y_cap = e.y.capacity;
    M.m = (uint32_t)e.a.rows;
    M.n = (uint32_t)e.a.cols;
    M.nseg_row = (uint32_t)((e.a.cols + 31) / 32);
    const DivSeg dv = DivSeg::make(M.nseg_row ? M.nseg_row : 1);
    M.dm = dv.m;
    M.ds1 = dv.s1;
    M.ds2 = dv.s2;
    M.y_off = yoff;
    yoff += e.a.rows;
    M.x_off = xoff;
    xoff += x_image_ints(e.a.cols);
    const uint64_t s = segments_of(e);
    const uint64_t nu = s ? (s + unit_segments - 1) / unit_segments : 1;
    M.units = (uint32_t)nu;
    for (uint64_t k = 0; k < nu; ++k, ++u) {
      units[u].mat = (uint32_t)i;
      units[u].seg0 = (uint32_t)(k * unit_segments);
      units[u].nseg = (uint32_t)(s ? ccm::umin(unit_segments, s - k * unit_segments) : 0);
    }
  }
  uint64_t maxcols = 0, maxw = 1;
  for (int i = 0; i < count; ++i) {
    maxcols = ccm::umax(maxcols, entries[i].a.cols);
    // the widest A the capacity admits (a valid header's width is at most this)
    const uint64_t n = entries[i].a.rows * entries[i].a.cols;
    if (n) maxw = ccm::umax(maxw, ccm::umin(entries[i].a.capacity * 32 / n, 32));
  }
  info->count = (uint32_t)count;
  info->max_cols = (uint32_t)maxcols;
  info->max_width = (uint32_t)maxw;
  info->slots = 2;
  info->x_ints = xoff;
  info->units = L.nunits;
  info->y_rows = L.yrows;
  info->unit_segments = unit_segments;
  info->plan_bytes = L.bytes;
  std::memcpy(host.data(), info, sizeof(ccm_batch_info));
  if (cudaMemcpy(plan, host.data(), L.bytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return CCM_E_CUDA;
  return CCM_OK;
}

ccm_status ccm_batch_matvec(const void* plan, const ccm_batch_info* info, void* ws,
                            size_t ws_bytes, int grid, ccm_stream_t stream) {
  using namespace ccm::bt;
  if (!plan || !info || !ws || info->count == 0) return CCM_E_INVAL;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return CCM_E_INVAL;
  if (ws_bytes < ccm::bt::ws_bytes(info->y_rows, info->count, info->x_ints))
    return CCM_E_CAPACITY;
  Layout L;
  L.mats_off = align256(sizeof(ccm_batch_info));
  L.units_off = L.mats_off + align256(sizeof(Mat) * (size_t)info->count);
  Args a;
  a.mats = reinterpret_cast<const Mat*>((const uint8_t*)plan + L.mats_off);
  a.units = reinterpret_cast<const Unit*>((const uint8_t*)plan + L.units_off);
  a.nmats = info->count;
  a.nunits = info->units;
  a.yscratch = (int64_t*)ws;
  a.done = (uint32_t*)((uint8_t*)ws + ws_done(info->y_rows));
  a.ticket = (uint32_t*)((uint8_t*)ws + ws_ticket(info->y_rows, info->count));
  a.ximage = (int*)((uint8_t*)ws + ws_ximage(info->y_rows, info->count));
  // the warps' ring slots, sized for the widest A
  if (info->max_width < 1 || info->max_width > 32 || info->max_cols > (uint32_t)kMaxCols)
    return CCM_E_INVAL;
  a.slot = slot_words((int)info->max_width);
  a.bmax = info->max_width;
  if (info->slots != 0 && info->slots != 2 && info->slots != 4) return CCM_E_INVAL;
  a.slots = info->slots == 4 ? 4 : 2;
  const size_t smem = (size_t)kWarps * a.slots * a.slot * sizeof(uint32_t);
  if (smem > (size_t)ccm::max_smem_optin()) return CCM_E_INVAL;
  if (grid <= 0) grid = ccm::num_sms() * 3;
  static size_t attr = 0;
  if (smem > attr) {
    if (cudaFuncSetAttribute(k_batch_mv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return CCM_E_CUDA;
    attr = smem;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_batch_init<<<info->count, 256, 0, st>>>(a);
  ccm::profile_begin(st);
  k_batch_mv<<<grid, kThreads, smem, st>>>(a);
  ccm::profile_end(st);
  ccm::note_launch(2);
  return cudaGetLastError() == cudaSuccess ? CCM_OK : CCM_E_CUDA;
}

}  // extern "C"
