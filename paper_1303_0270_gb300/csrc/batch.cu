// batch.cu -- y_i = A_i x_i for thousands of packed matrices of uneven
// shapes and widths in one persistent launch.
//
// Row i of an m x n matrix is cut into ceil(n / 32) segments of up to 32
// fields; segments are numbered row-major within a matrix, and a work unit is
// a run of consecutive segments of one matrix (the plan's unit list).  Every
// warp of the persistent kernel takes units from an atomic ticket of its own
// (no CTA barrier: the warps of a CTA are independent) and streams them
// through a ring of D slots in shared memory.  A stage is 32 P consecutive
// segments of one unit (P segments per lane, about `stage_bytes` bytes of A
// whatever the width); its word range is brought in by one 1-D
// cp.async.bulk completing on the slot's mbarrier, so D - 1 stages are in
// flight while one is decoded.  The warp fetches its next unit's ticket one
// unit ahead, so the ring runs on across unit and matrix boundaries.
//
// Lane l of a stage's sub-step p decodes segment 32 p + l: it reads the b + 1
// words that cover the segment from the slot and funnel-shifts them once to
// the segment's first bit (a segment starts at an arbitrary bit).  Fast
// path (b <= 24 and x of at most 8 signed bits, or 7 unsigned): x is decoded
// once into bytes and the segment's dot product runs on the integer dot
// units -- four fields spread into the bytes of a register per dp4a
// (b <= 8), two into the halves per dp2a (b <= 16), signed fields in offset
// binary corrected by 2^(b-1) times the segment's sum of x; b = 17..24 takes
// one 32 x 32 -> 64 multiply-add per field.  Other entries take the general
// path (int32 x image, one 64-bit multiply-add per field).  Lanes hold
// consecutive segments, so the rows of a sub-step are runs of lanes: one row
// is summed with two redux.sync, several with a segmented shuffle reduction;
// each row's partial sum is added to the int64 y scratch with one atomic.
//
// The tickets hand out the units in the order of their matrices' codes
// (width, sign, path): a one-CTA kernel after the initialisation sorts them
// by counting.  So at any time the warps of an SM decode one or two widths,
// and the code of one width-specialised decode stays in the instruction
// cache (with units in plan order, the warps of an SM ran up to 24 different
// decode bodies at once and mostly waited for instruction fetch).
//
// The warp that completes the last unit of a matrix (per-matrix counter)
// re-packs that matrix's y at its exact width (width rule of Eq. 1 with the
// two's complement reading) and writes y's header.  The whole batch is one
// launch after a small initialisation kernel, and both can be captured in a
// CUDA graph.
#include <cstring>
#include <vector>

#include "async_copy.cuh"
#include "ccm_device.cuh"
#include "kernels.h"

namespace ccm {
namespace bt {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxCols = 8192;       // x of at most 8192 entries per matrix
constexpr int kMaxSlots = 4;         // ring depth limit
constexpr int kMaxLaneSegs = 8;      // segments per lane in one stage
constexpr uint32_t kDefaultStageBytes = 3072;
constexpr int kFastMaxWidth = 24;    // widest A on the byte-dot path

// Segments per lane of one stage at width b: about stage_bytes of A per
// warp stage (a sub-step of 32 segments holds 128 b bytes).
__host__ __device__ inline uint32_t lane_segments(uint32_t stage_bytes, int b) {
  const uint32_t p = stage_bytes / (128u * (uint32_t)b);
  return p < 1 ? 1u : (p > (uint32_t)kMaxLaneSegs ? (uint32_t)kMaxLaneSegs : p);
}

// Bytes of one ring slot: the largest stage at any width up to bmax (at most
// 128 P b bytes of fields) plus what the reads around it need.  The copy
// starts up to 12 bytes before the stage's first bit (16-byte rounding) and
// a lane reads b + 1 words from its segment's first word, also when the
// segment is the short last one of a row: the highest word read is at most
// 32 P b + 4 + b words into the slot.
__host__ __device__ inline uint32_t slot_bytes(uint32_t stage_bytes, int bmax) {
  uint32_t m = 0;
  for (int b = 1; b <= bmax; ++b) {
    const uint32_t v = lane_segments(stage_bytes, b) * 128u * (uint32_t)b + 4u * (uint32_t)b;
    m = v > m ? v : m;
  }
  return (m + 64u + 127u) & ~127u;
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
  uint32_t unit0;      // index of the matrix's first unit in the unit list
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

__device__ __forceinline__ uint32_t div_seg(uint32_t v, uint32_t dm, uint32_t ds1, uint32_t ds2) {
  const uint32_t t = __umulhi(v, dm);
  return (t + ((v - t) >> ds1)) >> ds2;
}

struct Unit {
  uint32_t mat;
  uint32_t seg0;   // first segment (row-major numbering within the matrix)
  uint32_t nseg;   // number of segments
  uint32_t pad;
};

// Per-matrix run-time code, written by k_batch_init from the headers: 0 for
// an entry that is skipped (its y header holds the error), else
// width | sign << 7 | fast path << 8 | segments per lane << 9.
constexpr uint32_t kCodeSign = 1u << 7, kCodeFast = 1u << 8;
__device__ __forceinline__ int code_width(uint32_t c) { return (int)(c & 127u); }
__device__ __forceinline__ uint32_t code_lane_segs(uint32_t c) { return (c >> 9) & 15u; }

struct Args {
  const Mat* mats;
  const Unit* units;
  uint32_t nmats, nunits;
  int64_t* yscratch;
  uint32_t* ticket;     // unit dispenser
  uint32_t* done;       // per-matrix completed units
  uint32_t* codes;      // per-matrix run-time code
  uint32_t* order;      // unit indices in code order; order[nunits] = their count
  int* ximage;          // decoded x of every matrix (Mat::x_off)
  uint32_t slot_bytes;  // bytes of one ring slot
  uint32_t stage_bytes; // target bytes of A per stage
  uint32_t slots;       // ring depth D (2..4)
  uint32_t bmax;        // widest A the slots hold
};

// Position of field f of a segment in its 32-byte x image on the fast path:
// the order in which the width-b decode pairs fields with x bytes (natural,
// except for b = 1, 2, 4, where byte p of the k-th shifted copy of word i
// holds field i (32/b) + p (8/b) + k).
__device__ __forceinline__ uint32_t xbyte_pos(uint32_t f, int b) {
  if (b == 1 || b == 2 || b == 4) {
    const uint32_t per = 32u / b, r = 8u / b;
    const uint32_t i = f / per, q = f % per;
    return 4u * (i * r + q % r) + q / r;
  }
  return f;
}

// ---------------------------------------------------------------------------
// Initialisation: validate inputs, write y headers and codes, clear counters
// and the y scratch, decode x into its image.
// ---------------------------------------------------------------------------
__global__ void k_batch_init(Args a) {
  __shared__ int s_st;
  __shared__ uint32_t s_code;
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
    uint32_t code = 0;
    if (st == CCM_OK) {
      const int b = M.ha->width, bx = M.hx->width, sx = M.hx->is_signed;
      const bool fast = b <= kFastMaxWidth && (sx ? bx <= 8 : bx <= 7);
      code = (uint32_t)b | (M.ha->is_signed ? kCodeSign : 0u) | (fast ? kCodeFast : 0u) |
             (lane_segments(a.stage_bytes, b) << 9);
    }
    a.codes[i] = code;
    s_st = st;
    s_code = code;
  }
  for (uint32_t r = threadIdx.x; r < M.m; r += blockDim.x) a.yscratch[M.y_off + r] = 0;
  __syncthreads();
  if (s_st != CCM_OK) return;
  const int bx = M.hx->width, sx = M.hx->is_signed;
  const uint32_t nsr = M.nseg_row;
  int* xi = a.ximage + M.x_off;
  if (s_code & kCodeFast) {
    // bytes: [half][segment][16], half h holding image bytes 16 h .. 16 h + 15;
    // then the per-segment sums of x (int).  A warp covers whole segments.
    const int b = code_width(s_code);
    int8_t* xb = reinterpret_cast<int8_t*>(xi);
    int* xsum = xi + 8 * nsr;
    for (uint32_t j = threadIdx.x; j < nsr * 32; j += blockDim.x) {
      const uint32_t seg = j / 32, f = j % 32;
      const int v = j < M.n ? (int)decode_field(M.wx, j, bx, sx) : 0;
      const uint32_t pos = xbyte_pos(f, b);
      xb[(pos / 16) * 16 * nsr + 16 * seg + pos % 16] = (int8_t)v;
      const int s = __reduce_add_sync(0xffffffffu, v);
      if (f == 0) xsum[seg] = s;
    }
  } else {
    // int32, layout [f/4][segment][f%4], zero past n
    for (uint32_t j = threadIdx.x; j < nsr * 32; j += blockDim.x) {
      const uint32_t seg = j / 32, f = j % 32;
      xi[((f / 4) * nsr + seg) * 4 + (f % 4)] = j < M.n ? (int)decode_field(M.wx, j, bx, sx) : 0;
    }
  }
}

// ---------------------------------------------------------------------------
// Unit order: a counting sort of the valid entries' units by code, one CTA.
// ---------------------------------------------------------------------------
constexpr int kOrderThreads = 1024;
constexpr int kCodes = 512;  // codes & 0x1ff

__global__ void __launch_bounds__(kOrderThreads) k_batch_order(Args a) {
  __shared__ uint32_t s_cnt[kCodes];
  for (int c = threadIdx.x; c < kCodes; c += blockDim.x) s_cnt[c] = 0;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < a.nmats; i += blockDim.x) {
    const uint32_t code = a.codes[i];
    if (code) atomicAdd(&s_cnt[code & (kCodes - 1)], a.mats[i].units);
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // exclusive scan of the 512 counts by one warp, 16 per lane
    const int lane = threadIdx.x;
    uint32_t v[kCodes / 32], sum = 0;
#pragma unroll
    for (int k = 0; k < kCodes / 32; ++k) {
      v[k] = s_cnt[lane * (kCodes / 32) + k];
      sum += v[k];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
      if (lane >= d) incl += o;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int k = 0; k < kCodes / 32; ++k) {
      s_cnt[lane * (kCodes / 32) + k] = run;
      run += v[k];
    }
    if (lane == 31) a.order[a.nunits] = incl;  // units to hand out
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < a.nmats; i += blockDim.x) {
    const uint32_t code = a.codes[i];
    if (!code) continue;
    const Mat& M = a.mats[i];
    const uint32_t at = atomicAdd(&s_cnt[code & (kCodes - 1)], M.units);
    for (uint32_t k = 0; k < M.units; ++k) a.order[at + k] = M.unit0 + k;
  }
}

// ---------------------------------------------------------------------------
// Dot products of one segment (32 fields in f[0..B-1], f[B] spare)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int dp4a_us(uint32_t a, int b, int c) {
  int d;
  asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ int dp2a_lo_us(uint32_t a, int b, int c) {
  int d;
  asm("dp2a.lo.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
__device__ __forceinline__ int dp2a_hi_us(uint32_t a, int b, int c) {
  int d;
  asm("dp2a.hi.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}
// Byte k of w sign-extended to 32 bits (prmt with the sign-replicate bit
// set in the selectors of bytes 1..3).
__device__ __forceinline__ int sbyte(uint32_t w, int k) {
  const uint32_t sel = (uint32_t)k | ((uint32_t)(k | 8) * 0x1110u);
  int d;
  asm("prmt.b32 %0, %1, 0, %2;" : "=r"(d) : "r"(w), "r"(sel));
  return d;
}

__host__ __device__ constexpr uint32_t low_bits(int b) { return b >= 32 ? 0xffffffffu : ((1u << b) - 1u); }


// Fast path: sum over the segment's fields of a_f x_f with x bytes xw[0..7]
// in the order of xbyte_pos; `xs` is the segment's sum of x (offset binary).
template <int B, bool SGN>
__device__ __forceinline__ int64_t seg_dot_fast(uint32_t (&f)[B + 1], const int (&xw)[8], int xs) {
  if constexpr (B <= 16) {
    if constexpr (SGN) {
#pragma unroll
      for (int i = 0; i < B; ++i) f[i] ^= group_sign_bits(B, i);
    }
    int acc0 = 0, acc1 = 0;
    if constexpr (B == 1 || B == 2 || B == 4) {
      constexpr int R = 8 / B;
      constexpr uint32_t m = low_bits(B) * 0x01010101u;
#pragma unroll
      for (int i = 0; i < B; ++i)
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const uint32_t v = (f[i] >> (B * k)) & m;
          if ((i * R + k) & 1)
            acc1 = dp4a_us(v, xw[i * R + k], acc1);
          else
            acc0 = dp4a_us(v, xw[i * R + k], acc0);
        }
    } else if constexpr (B == 8) {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        if (i & 1)
          acc1 = dp4a_us(f[i], xw[i], acc1);
        else
          acc0 = dp4a_us(f[i], xw[i], acc0);
      }
    } else if constexpr (B < 8) {
      // four fields (4B bits) -> two 16-bit halves of two fields -> four bytes
      constexpr uint32_t m2 = low_bits(2 * B), m1 = low_bits(B) * 0x00010001u;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        constexpr int kB4 = 4 * B;
        const int bit = kB4 * c, wi = bit >> 5, sh = bit & 31;
        const uint32_t x4 = (sh + kB4 <= 32) ? (f[wi] >> sh) : __funnelshift_r(f[wi], f[wi + 1], sh);
        const uint32_t u = (x4 & m2) | ((x4 << (16 - 2 * B)) & (m2 << 16));
        const uint32_t v = (u & m1) | ((u << (8 - B)) & (m1 << 8));
        if (c & 1)
          acc1 = dp4a_us(v, xw[c], acc1);
        else
          acc0 = dp4a_us(v, xw[c], acc0);
      }
    } else if constexpr (B == 16) {
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        if (c & 1)
          acc1 = dp2a_hi_us(f[c], xw[c >> 1], acc1);
        else
          acc0 = dp2a_lo_us(f[c], xw[c >> 1], acc0);
      }
    } else {
      // two fields (2B bits) -> two 16-bit halves
      constexpr uint32_t mb = low_bits(B);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        constexpr int kB2 = 2 * B;
        const int bit = kB2 * c, wi = bit >> 5, sh = bit & 31;
        const uint32_t x2 = (sh + kB2 <= 32) ? (f[wi] >> sh) : __funnelshift_r(f[wi], f[wi + 1], sh);
        const uint32_t v = (x2 & mb) | ((x2 << (16 - B)) & (mb << 16));
        if (c & 1)
          acc1 = dp2a_hi_us(v, xw[c >> 1], acc1);
        else
          acc0 = dp2a_lo_us(v, xw[c >> 1], acc0);
      }
    }
    int acc = acc0 + acc1;
    if constexpr (SGN) acc -= xs * (1 << (B - 1));
    return acc;
  } else {
    // B = 17..24: a field is its low 16 bits plus 2^16 times its high B - 16
    // bits.  Per four fields: the low halves of two fields in one register
    // (prmt) against two x bytes (dp2a), the high parts of all four in the
    // bytes of one register (prmt, masked; signed fields: the sign bit
    // flipped, offset binary) against the four x bytes (dp4a).
    constexpr uint32_t mh = low_bits(B - 16) * 0x01010101u;
    constexpr uint32_t sflip = SGN ? (1u << (B - 17)) * 0x01010101u : 0u;
    int lo0 = 0, lo1 = 0, hi = 0;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      uint32_t t[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int bit = B * (4 * c + k), wi = bit >> 5, sh = bit & 31;
        t[k] = (sh + B <= 32) ? (f[wi] >> sh) : __funnelshift_r(f[wi], f[wi + 1], sh);
      }
      const uint32_t l01 = __byte_perm(t[0], t[1], 0x5410), l23 = __byte_perm(t[2], t[3], 0x5410);
      const uint32_t h01 = __byte_perm(t[0], t[1], 0x0062), h23 = __byte_perm(t[2], t[3], 0x0062);
      const uint32_t h = (__byte_perm(h01, h23, 0x5410) & mh) ^ sflip;
      lo0 = dp2a_lo_us(l01, xw[c], lo0);
      lo1 = dp2a_hi_us(l23, xw[c], lo1);
      hi = dp4a_us(h, xw[c], hi);
    }
    int64_t acc = (int64_t)(lo0 + lo1) + (int64_t)hi * 65536;
    if constexpr (SGN) acc -= (int64_t)xs * (1ll << (B - 1));
    return acc;
  }
}

// General path: x int32 in the [f/4][segment][f%4] image (xv = image + s).
template <int B, bool SGN>
__device__ __forceinline__ int64_t seg_dot_gen(const uint32_t (&f)[B + 1], const int4* __restrict__ xv,
                                               uint32_t nsr) {
  long long acc = 0;
#pragma unroll
  for (int f4 = 0; f4 < 8; ++f4) {
    const int4 xq = __ldg(xv + f4 * nsr);
    const int xa[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
    for (int qq = 0; qq < 4; ++qq) {
      const int e = 4 * f4 + qq;
      const int b0 = e * B, wi = b0 >> 5, sh = b0 & 31;
      const uint32_t t = (sh + B <= 32) ? (f[wi] >> sh) : __funnelshift_r(f[wi], f[wi + 1], sh);
      if constexpr (B == 32 && !SGN) {
        acc += (long long)t * xa[qq];
      } else {
        int v;
        if constexpr (B == 32)
          v = (int)t;
        else if constexpr (SGN)
          v = (int)(t << (32 - B)) >> (32 - B);
        else
          v = (int)(t & low_bits(B));
        acc += (long long)v * (long long)xa[qq];
      }
    }
  }
  return acc;
}

// General path: adds each lane's segment sum to its row of y.  The rows of a
// sub-step are runs of consecutive lanes, each at most nsr long (a row has
// nsr segments): a segmented shuffle reduction with as many steps as the
// longest run needs leaves each row's sum in its first lane.
__device__ __forceinline__ void row_add(int64_t acc, uint32_t row, uint32_t nsr, int64_t* ys,
                                        int lane) {
  const uint32_t span = nsr < 32 ? nsr : 32;
  long long s = acc;
  for (uint32_t d = 1; d < span; d <<= 1) {
    const long long o = __shfl_down_sync(0xffffffffu, s, d);
    const uint32_t ro = __shfl_down_sync(0xffffffffu, row, d);
    if (lane + d < 32 && ro == row) s += o;
  }
  const uint32_t rprev = __shfl_up_sync(0xffffffffu, row, 1);
  if (row != 0xffffffffu && (lane == 0 || rprev != row) && s)
    atomicAdd(reinterpret_cast<unsigned long long*>(ys + row), (unsigned long long)s);
}

// The staged words of a segment: b + 1 words from word `wo` of the slot
// (a generic pointer into shared memory: the loads take immediate offsets).
template <int B>
__device__ __forceinline__ void load_segment(uint32_t sp, uint32_t wo, uint32_t sh,
                                             uint32_t (&f)[B + 1]) {
  const uint32_t* w = reinterpret_cast<const uint32_t*>(__cvta_shared_to_generic(sp)) + wo;
#pragma unroll
  for (int j = 0; j <= B; ++j) f[j] = w[j];
#pragma unroll
  for (int j = 0; j < B; ++j) f[j] = __funnelshift_r(f[j], f[j + 1], sh);
}

// One stage of a matrix at compile-time width B: segments [g0, g1) whose
// words start at word w_lo of A, staged at shared address `sp`; n columns,
// nsr segments per row (divided by dm, ds & 255, ds >> 8).
template <int B, bool SGN, bool FAST>
__device__ __noinline__ void run_stage(uint32_t sp, uint64_t w_lo, uint32_t g0, uint32_t g1,
                                       uint32_t n, uint32_t nsr, uint32_t dm, uint32_t ds,
                                       const int* ximg, int64_t* ys) {
  const int lane = threadIdx.x % 32;
  const uint32_t ds1 = ds & 255u, ds2 = ds >> 8;
  // Fast path: each lane keeps a running sum for its current row and adds it
  // to y (one atomic, no warp-wide step) when its next segment starts another
  // row and at the end of the stage.  General path: rows reduced per sub-step.
  int64_t racc = 0;
  uint32_t rrow = 0xffffffffu;
  for (uint32_t base = g0; base < g1; base += 32) {
    const uint32_t g = base + lane;
    const bool live = g < g1;
    const uint32_t gg = live ? g : base;  // a dead lane decodes a live segment, then drops it
    const uint32_t q = div_seg(gg, dm, ds1, ds2);
    const uint32_t s = gg - q * nsr;
    const uint64_t bit = ((uint64_t)q * n + 32u * s) * (uint64_t)B;
    const uint32_t wo = (uint32_t)((bit >> 5) - w_lo), sh = (uint32_t)bit & 31u;
    if constexpr (FAST) {
      const int4* xb = reinterpret_cast<const int4*>(ximg);
      const int4 x0 = __ldg(xb + s), x1 = __ldg(xb + nsr + s);
      const int xs = SGN ? __ldg(ximg + 8 * nsr + s) : 0;
      uint32_t f[B + 1];
      load_segment<B>(sp, wo, sh, f);
      const int xw[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
      const int64_t acc = seg_dot_fast<B, SGN>(f, xw, xs);
      if (live) {
        if (q != rrow) {
          if (racc) atomicAdd(reinterpret_cast<unsigned long long*>(ys + rrow), (unsigned long long)racc);
          rrow = q;
          racc = acc;
        } else {
          racc += acc;
        }
      }
    } else {
      uint32_t f[B + 1];
      load_segment<B>(sp, wo, sh, f);
      int64_t acc = seg_dot_gen<B, SGN>(f, reinterpret_cast<const int4*>(ximg) + s, nsr);
      if (!live) acc = 0;
      row_add(acc, live ? q : 0xffffffffu, nsr, ys, lane);
    }
  }
  if (FAST && racc) atomicAdd(reinterpret_cast<unsigned long long*>(ys + rrow), (unsigned long long)racc);
}

// Re-pack y of one matrix at its exact width; the whole warp takes part
// (lane l assembles the b words of the 32-field groups l, l + 32, ...).
__device__ void pack_y_warp(const Mat& M, const int64_t* __restrict__ ys, int lane) {
  const uint32_t m = M.m;
  uint64_t orv = 0;
  uint32_t neg = 0;
  for (uint32_t i = lane; i < m; i += 32) {
    const int64_t v = __ldcg(ys + i);
    orv |= fold(v);
    neg |= (uint32_t)(v < 0);
  }
  orv = warp_or64(orv);
  neg = __reduce_or_sync(0xffffffffu, neg);
  const int b = width_from_stats(orv, neg);
  const uint64_t nw = words_for(m, b);
  const bool fits = nw <= M.y_cap;
  if (lane == 0) {
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
  const uint32_t groups = (m + 31) / 32;
  for (uint32_t g = lane; g < groups; g += 32) {
    uint64_t w = (uint64_t)g * b;  // first word of the group
    unsigned __int128 buf = 0;     // bits not yet written
    int fill = 0;
    for (int e = 0; e < 32; ++e) {
      const uint64_t i = (uint64_t)g * 32 + e;
      const uint64_t pat = i < m ? ((uint64_t)__ldcg(ys + i) & mask) : 0;
      buf |= (unsigned __int128)pat << fill;
      fill += b;
      while (fill >= 32) {
        if (w < nw) M.wy[w] = (uint32_t)buf;
        ++w;
        buf >>= 32;
        fill -= 32;
      }
    }
  }
  // words past the last group's (the 16-byte padding)
  for (uint64_t w = (uint64_t)groups * b + lane; w < nw; w += 32) M.wy[w] = 0;
}

// ---------------------------------------------------------------------------
// The persistent kernel
// ---------------------------------------------------------------------------
// A staged stage, written by lane 0 when it issues the copy: everything the
// decode needs, so that the consumer reads no descriptor from global memory.
__device__ __forceinline__ uint32_t lo32(const void* p) { return (uint32_t)(uintptr_t)p; }
__device__ __forceinline__ uint32_t hi32(const void* p) { return (uint32_t)((uintptr_t)p >> 32); }
template <typename T>
__device__ __forceinline__ T* ptr_of(uint32_t lo, uint32_t hi) {
  return reinterpret_cast<T*>(((uint64_t)hi << 32) | lo);
}

// A staged stage (64 bytes in shared memory, written by lane 0 with four
// 16-byte stores when it issues the copy, read back the same way): all the
// decode needs, so that the consumer reads nothing else.
//   q[0]: w_lo (first word of the slot's copy), x image
//   q[1]: y scratch rows, g0, g1 (segments)
//   q[2]: n, nsr, dm, ds (ds1 | ds2 << 8)
//   q[3]: code, matrix, last stage of its unit, 0
struct alignas(16) Desc {
  uint4 q[4];
};

// The unit a warp is issuing (64 bytes in shared memory, written by lane 0
// when the warp takes the unit, read by the producer per stage).
//   q[0]: A's words, x image     q[1]: y scratch rows, n, nsr
//   q[2]: dm, ds, code, matrix   q[3]: seg0, nseg, 0, 0
struct alignas(16) URec {
  uint4 q[4];
};

// The stage producer of one warp: every lane holds the same state; lane 0
// takes the tickets, fills the unit record and issues the copies.
struct Producer {
  uint32_t unit;   // unit being issued (>= nunits: none left)
  uint32_t pos;    // its segments already issued
  uint32_t nseg;   // its segments
  uint32_t tk;     // lane 0: the ticket taken one unit ahead
  uint32_t count;  // units to hand out (the valid entries')

  __device__ __forceinline__ void take(const Args& a, URec* rec, int lane) {
    const uint32_t t = __shfl_sync(0xffffffffu, tk, 0);
    pos = 0;
    unit = a.nunits;
    if (t < count) {
      if (lane == 0) {
        tk = atomicAdd(a.ticket, 1u);  // (its latency hides behind the loads below)
        const uint32_t ui = a.order[t];
        const Unit u = a.units[ui];
        const Mat& M = a.mats[u.mat];
        const uint32_t code = a.codes[u.mat];
        const int* ximg = a.ximage + M.x_off;
        int64_t* ys = a.yscratch + M.y_off;
        rec->q[0] = make_uint4(lo32(M.wa), hi32(M.wa), lo32(ximg), hi32(ximg));
        rec->q[1] = make_uint4(lo32(ys), hi32(ys), M.n, M.nseg_row);
        rec->q[2] = make_uint4(M.dm, M.ds1 | (M.ds2 << 8), code, u.mat);
        rec->q[3] = make_uint4(u.seg0, u.nseg, ui, 0);
      }
      __syncwarp();
      const uint4 r3 = rec->q[3];
      unit = r3.z;
      nseg = r3.y;
    }
  }

  // Issues the next stage into slot memory `dst` (false: no stage left).
  __device__ __forceinline__ bool issue(const Args& a, uint8_t* dst, uint64_t* bar, Desc* d,
                                        URec* rec, int lane) {
    if (unit >= a.nunits) return false;
    const uint4 r0 = rec->q[0], r1 = rec->q[1], r2 = rec->q[2], r3 = rec->q[3];
    const uint32_t n = r1.z, nsr = r1.w, dm = r2.x, ds = r2.y, code = r2.z;
    const int b = code_width(code);
    const uint32_t cnt = umin(nseg - pos, 32u * code_lane_segs(code));
    const uint32_t g0 = r3.x + pos, g1 = g0 + cnt;
    uint64_t w_lo = 0;
    uint32_t bytes = 0;
    if (cnt) {
      const uint32_t ds1 = ds & 255u, ds2 = ds >> 8;
      const uint32_t q0 = div_seg(g0, dm, ds1, ds2), s0 = g0 - q0 * nsr;
      const uint32_t ql = div_seg(g1 - 1, dm, ds1, ds2), sl = g1 - 1 - ql * nsr;
      const uint64_t fb = ((uint64_t)q0 * n + 32u * s0) * (uint64_t)b;
      const uint64_t eb = ((uint64_t)ql * n + umin(n, 32u * sl + 32u)) * (uint64_t)b;
      w_lo = (fb >> 5) & ~3ull;
      const uint64_t w_hi = (((eb + 31) >> 5) + 3) & ~3ull;
      bytes = (uint32_t)((w_hi - w_lo) * 4);
    }
    pos += cnt;
    const bool last = pos >= nseg;
    if (lane == 0) {
      d->q[0] = make_uint4((uint32_t)w_lo, (uint32_t)(w_lo >> 32), r0.z, r0.w);
      d->q[1] = make_uint4(r1.x, r1.y, g0, g1);
      d->q[2] = make_uint4(n, nsr, dm, ds);
      d->q[3] = make_uint4(code, r2.w, last ? 1u : 0u, 0u);
      ax::mbar_expect_tx(bar, bytes);
      if (bytes) ax::bulk_g2s(dst, ptr_of<const uint32_t>(r0.x, r0.y) + w_lo, bytes, bar);
    }
    if (last) take(a, rec, lane);
    return true;
  }
};

__device__ __forceinline__ void stage_dispatch(uint32_t sp, const uint4 (&d)[4]) {
  const uint64_t w_lo = ((uint64_t)d[0].y << 32) | d[0].x;
  const int* ximg = ptr_of<const int>(d[0].z, d[0].w);
  int64_t* ys = ptr_of<int64_t>(d[1].x, d[1].y);
  const uint32_t g0 = d[1].z, g1 = d[1].w, n = d[2].x, nsr = d[2].y, dm = d[2].z, ds = d[2].w;
  switch (d[3].x & 0x1ffu) {
#define CCM_BT_GEN(B)                                                          \
  case (B): run_stage<B, false, false>(sp, w_lo, g0, g1, n, nsr, dm, ds, ximg, ys); break; \
  case (B) | 128: run_stage<B, true, false>(sp, w_lo, g0, g1, n, nsr, dm, ds, ximg, ys); break;
#define CCM_BT_FAST(B)                                                         \
  case (B) | 256: run_stage<B, false, true>(sp, w_lo, g0, g1, n, nsr, dm, ds, ximg, ys); break; \
  case (B) | 384: run_stage<B, true, true>(sp, w_lo, g0, g1, n, nsr, dm, ds, ximg, ys); break;
#define CCM_BT_BOTH(B) CCM_BT_GEN(B) CCM_BT_FAST(B)
    CCM_BT_BOTH(1) CCM_BT_BOTH(2) CCM_BT_BOTH(3) CCM_BT_BOTH(4) CCM_BT_BOTH(5) CCM_BT_BOTH(6)
    CCM_BT_BOTH(7) CCM_BT_BOTH(8) CCM_BT_BOTH(9) CCM_BT_BOTH(10) CCM_BT_BOTH(11) CCM_BT_BOTH(12)
    CCM_BT_BOTH(13) CCM_BT_BOTH(14) CCM_BT_BOTH(15) CCM_BT_BOTH(16) CCM_BT_BOTH(17) CCM_BT_BOTH(18)
    CCM_BT_BOTH(19) CCM_BT_BOTH(20) CCM_BT_BOTH(21) CCM_BT_BOTH(22) CCM_BT_BOTH(23) CCM_BT_BOTH(24)
    CCM_BT_GEN(25) CCM_BT_GEN(26) CCM_BT_GEN(27) CCM_BT_GEN(28) CCM_BT_GEN(29) CCM_BT_GEN(30)
    CCM_BT_GEN(31) CCM_BT_GEN(32)
#undef CCM_BT_BOTH
#undef CCM_BT_FAST
#undef CCM_BT_GEN
    default: break;
  }
}

// Dynamic shared memory: each warp's D ring slots.
__global__ void __launch_bounds__(kThreads, 3) k_batch_mv(const __grid_constant__ Args a) {
  extern __shared__ __align__(128) uint8_t s_ring[];
  __shared__ __align__(8) uint64_t s_bar[kWarps][kMaxSlots];
  __shared__ Desc s_desc[kWarps][kMaxSlots];
  __shared__ URec s_rec[kWarps];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t D = a.slots, SB = a.slot_bytes;
  uint8_t* ring = s_ring + (size_t)warp * D * SB;
  uint64_t* bar = s_bar[warp];
  Desc* desc = s_desc[warp];
  URec* rec = &s_rec[warp];
  if (lane == 0) {
    for (uint32_t s = 0; s < D; ++s) ax::mbar_init(&bar[s], 1);
    ax::mbar_init_fence();
  }
  __syncwarp();
  Producer pr;
  pr.count = a.order[a.nunits];
  if (lane == 0) pr.tk = atomicAdd(a.ticket, 1u);
  pr.take(a, rec, lane);
  uint32_t issued = 0;
  while (issued < D && pr.issue(a, ring + issued * SB, &bar[issued], &desc[issued], rec, lane))
    ++issued;
  uint32_t consumed = 0, slot = 0, phase = 0;
  bool ok = true;
  while (consumed < issued) {
    if (!ax::mbar_wait(&bar[slot], phase)) {
      ok = false;
      break;
    }
    const uint4 d1 = desc[slot].q[1], d3 = desc[slot].q[3];  // (kept past the decode)
    if (d1.w > d1.z) {
      const uint4 d[4] = {desc[slot].q[0], d1, desc[slot].q[2], d3};
      stage_dispatch(ax::smem_u32(ring + slot * SB), d);
    }
    __syncwarp();
    ++consumed;
    ax::fence_proxy_async_smem();  // this slot's reads before its refill
    if (pr.issue(a, ring + slot * SB, &bar[slot], &desc[slot], rec, lane)) ++issued;
    if (d3.z) {
      // the unit is complete; the warp completing a matrix packs its y
      const uint32_t dmat = d3.y;
      __threadfence();
      __syncwarp();
      const Mat& M = a.mats[dmat];
      uint32_t fin = 0;
      if (lane == 0) fin = atomicAdd(a.done + dmat, 1u) + 1 == M.units;
      fin = __shfl_sync(0xffffffffu, fin, 0);
      if (fin) {
        __threadfence();
        pack_y_warp(M, ptr_of<int64_t>(d1.x, d1.y), lane);
      }
    }
    if (++slot == D) slot = 0, phase ^= 1;
  }
  if (!ok) {
    // a wait gave up: mark the entries this warp holds units of, and let the
    // copies still in flight land before the CTA's shared memory goes away
    for (uint32_t j = consumed; j < issued; ++j) {
      if (lane == 0) set_status(a.mats[desc[slot].q[3].y].hy, CCM_E_TIMEOUT);
      if (!ax::mbar_wait(&bar[slot], phase)) {
        // (a copy that never lands: report and leave it)
      }
      if (++slot == D) slot = 0, phase ^= 1;
    }
    if (lane == 0 && pr.unit < a.nunits) set_status(a.mats[rec->q[2].w].hy, CCM_E_TIMEOUT);
    const uint32_t t = __shfl_sync(0xffffffffu, pr.tk, 0);
    if (lane == 0 && t < pr.count) set_status(a.mats[a.units[a.order[t]].mat].hy, CCM_E_TIMEOUT);
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

// Workspace: int64 y scratch, per-matrix done counters, per-matrix codes,
// the ticket, x images.
size_t ws_done(uint64_t yrows) { return align256(yrows * 8); }
size_t ws_codes(uint64_t yrows, uint32_t count) {
  return ws_done(yrows) + align256((size_t)count * 4);
}
size_t ws_ticket(uint64_t yrows, uint32_t count) {
  return ws_codes(yrows, count) + align256((size_t)count * 4);
}
size_t ws_order(uint64_t yrows, uint32_t count) { return ws_ticket(yrows, count) + 256; }
size_t ws_ximage(uint64_t yrows, uint32_t count, uint64_t units) {
  return ws_order(yrows, count) + align256((units + 1) * 4);
}
size_t ws_bytes(uint64_t yrows, uint32_t count, uint64_t xints, uint64_t units) {
  return ws_ximage(yrows, count, units) + align256(xints * 4);
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
  uint64_t yrows = 0, xints = 0, units = 0;
  for (int i = 0; i < count; ++i) {
    yrows += entries[i].a.rows;
    xints += ccm::bt::x_image_ints(entries[i].a.cols);
    // the most units any plan cuts this entry into (unit_segments >= 32)
    units += ccm::umax(1, (ccm::bt::segments_of(entries[i]) + 31) / 32);
  }
  return ccm::bt::ws_bytes(yrows, (uint32_t)count, xints, units);
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
    M.unit0 = (uint32_t)u;
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
  info->slots = 0;
  info->stage_bytes = 0;
  info->reserved = 0;
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
  if (ws_bytes < ccm::bt::ws_bytes(info->y_rows, info->count, info->x_ints, info->units))
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
  a.codes = (uint32_t*)((uint8_t*)ws + ws_codes(info->y_rows, info->count));
  a.ticket = (uint32_t*)((uint8_t*)ws + ws_ticket(info->y_rows, info->count));
  a.order = (uint32_t*)((uint8_t*)ws + ws_order(info->y_rows, info->count));
  a.ximage = (int*)((uint8_t*)ws + ws_ximage(info->y_rows, info->count, info->units));
  // the warps' ring slots, sized for the widest A
  if (info->max_width < 1 || info->max_width > 32 || info->max_cols > (uint32_t)kMaxCols)
    return CCM_E_INVAL;
  a.bmax = info->max_width;
  if (info->slots != 0 && (info->slots < 2 || info->slots > (uint32_t)kMaxSlots))
    return CCM_E_INVAL;
  a.slots = info->slots ? info->slots : 3;
  if (info->stage_bytes != 0 && (info->stage_bytes < 128 || info->stage_bytes > 16384))
    return CCM_E_INVAL;
  a.stage_bytes = info->stage_bytes ? info->stage_bytes : kDefaultStageBytes;
  a.slot_bytes = slot_bytes(a.stage_bytes, (int)a.bmax);
  // warps per CTA: 8, or 4 when that keeps more warps resident per SM (the
  // rings are per warp, so a smaller CTA packs the shared memory tighter)
  static size_t attr = 0;
  const size_t smem_max = (size_t)kWarps * a.slots * a.slot_bytes;
  if (smem_max > (size_t)ccm::max_smem_optin()) return CCM_E_INVAL;
  if (smem_max > attr) {
    if (cudaFuncSetAttribute(k_batch_mv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_max) != cudaSuccess)
      return CCM_E_CUDA;
    attr = smem_max;
  }
  static uint64_t occ_key = 0;  // (slots, slot bytes) of the cached choice
  static int occ_warps = kWarps, occ_per = 1;
  const uint64_t key = ((uint64_t)a.slots << 32) | a.slot_bytes;
  if (key != occ_key) {
    int best = 0;
    occ_warps = kWarps;
    occ_per = 1;
    for (int w = kWarps; w >= 4; w /= 2) {
      int p = 0;
      const size_t sm = (size_t)w * a.slots * a.slot_bytes;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p, k_batch_mv, 32 * w, sm) !=
          cudaSuccess)
        p = 0;
      if (p * w > best) best = p * w, occ_warps = w, occ_per = p;
    }
    if (best == 0) occ_per = 1;
    occ_key = key;
  }
  const int warps = occ_warps, per = occ_per;
  const size_t smem = (size_t)warps * a.slots * a.slot_bytes;
  if (grid <= 0) grid = ccm::num_sms() * per;  // one resident wave
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_batch_init<<<info->count, 256, 0, st>>>(a);
  k_batch_order<<<1, kOrderThreads, 0, st>>>(a);
  ccm::profile_begin(st);
  k_batch_mv<<<grid, 32 * warps, smem, st>>>(a);
  ccm::profile_end(st);
  ccm::note_launch(3);
  return cudaGetLastError() == cudaSuccess ? CCM_OK : CCM_E_CUDA;
}

}  // extern "C"
