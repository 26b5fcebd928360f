// matvec_fast.cuh -- y = A x for row-aligned A (cols a multiple of 128) with
// fields of at most 32 bits: the streaming kernel whose roofline is the
// packed bytes of A.
//
// Mapping: a warp owns 32 consecutive rows, one row per lane, and walks a
// slab of K columns in stages of 128 columns.  128 fields of one row are
// exactly 4*b words = b 16-byte vectors, 16-byte aligned because every row
// starts at bit i*cols*b with cols % 128 == 0.  Each stage is copied
// global -> shared with 16-byte cp.async (coalesced runs of 16*b bytes per
// row, double-buffered), rows padded to a pitch that is an odd multiple of 16
// bytes so the per-lane 16-byte shared loads are bank-conflict free.  Lanes
// then decode their 128 fields in registers with shifts fixed at compile time
// (the width b is read from the header on the GPU and dispatched through a
// switch over the 64 (b, sign) instances), multiply by x_j -- held as int32 in
// shared memory and read as broadcasts, since every lane of the warp is at
// the same column -- and accumulate in int64.  Partial sums of a column slab
// go to y with one 64-bit atomicAdd per row and slab.
//
// Byte-lane path (b <= 8 and x representable in int8, chosen on the GPU from
// the headers): four fields at a time are spread into the four bytes of a
// register and multiplied with four int8 x values by one dp4a.  Signed fields
// are first turned into offset binary (u = a + 2^(b-1), one XOR per word with
// the fixed positions of the sign bits), so
//   sum_j a_j x_j = sum_j u_j x_j - 2^(b-1) sum_j x_j,
// and the second term is one per-slab constant.  x is staged as int8 in the
// byte order the spread produces.
#pragma once

#include "ccm_device.cuh"

namespace ccm {
namespace mvf {

constexpr int kKC = 128;   // columns per stage

__host__ __device__ constexpr int pitch_bytes(int b) { return (b & 1) ? 16 * b : 16 * (b + 1); }

// Stages of a warp's cp.async ring: four (three in flight while one is
// decoded) for the narrow widths, whose stages are small and decode fast;
// two for the wide ones, whose stages are large.
__host__ __device__ constexpr int ring_depth(int b) { return b <= 8 ? 4 : 2; }

// Shared memory of one warp's ring when the field width is at most bmax.
__host__ __device__ constexpr uint32_t warp_region_bytes(int bmax) {
  uint32_t m = 0;
  for (int b = 1; b <= bmax; ++b) {
    const uint32_t v = (uint32_t)ring_depth(b) * 32u * (uint32_t)pitch_bytes(b);
    if (v > m) m = v;
  }
  return m;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct Args {
  ccm_header* out;             // y header (status checked, errors reported)
  const ccm_header* ha;
  const uint32_t* wa;
  const ccm_header* hx;
  const uint32_t* wx;
  uint64_t m, n;
  uint32_t kslab;              // columns per CTA slab (multiple of 128)
  uint32_t stage_region;       // bytes of shared memory holding the stage buffers
  uint32_t warp_region;        // bytes of it per warp (warp_region_bytes of the width bound)
  int64_t* y;                  // int64 partial sums, zeroed before launch
};

// The cp.async copies of one warp's stages (32 rows x 16*B bytes each):
// chunk c = lane + 32 j of a stage is piece c % B of row c / B.  For B <= 8
// the offsets are computed once per row block, relative to the warp's first
// row (32-bit: the host keeps 32 rows of A below 4 GiB on this path), and a
// stage s adds s * 16 * B bytes.  Wider fields recompute the addresses per
// stage (issue_stage) rather than hold 2*B more registers.
template <int B>
struct Issuer {
  const uint8_t* base;
  uint32_t rows_left;
  uint32_t goff[B];
  uint32_t soff[B];
  __device__ __forceinline__ void init(const Args& a, uint64_t row0, uint64_t col0, int lane) {
    const uint32_t row_bytes = (uint32_t)(a.n / 8 * B);  // n * B / 8, a multiple of 16
    base = reinterpret_cast<const uint8_t*>(a.wa) + row0 * (uint64_t)row_bytes + col0 / 8 * B;
    rows_left = (uint32_t)umin(a.m - row0, 32);
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int c = lane + 32 * j;
      const int r = c / B, piece = c % B;
      goff[j] = (uint32_t)r * row_bytes + 16 * piece;
      soff[j] = (uint32_t)(r * pitch_bytes(B) + 16 * piece) | ((uint32_t)r << 24);
    }
  }
  __device__ __forceinline__ void issue(uint8_t* buf, uint32_t s) const {
    const unsigned sb = (unsigned)__cvta_generic_to_shared(buf);
    const uint8_t* g = base + (uint64_t)s * (16 * B);
#pragma unroll
    for (int j = 0; j < B; ++j)
      if ((soff[j] >> 24) < rows_left)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sb + (soff[j] & 0xffffffu)),
                     "l"(g + goff[j])
                     : "memory");
  }
};

template <int B>
__device__ __forceinline__ void issue_stage(const Args& a, uint8_t* buf, uint64_t row0,
                                            uint64_t col0, int lane) {
  const uint64_t row_bytes = a.n / 8 * B;  // n * B / 8, a multiple of 16
  const uint8_t* base = reinterpret_cast<const uint8_t*>(a.wa) + col0 / 8 * B;
#pragma unroll
  for (int j = 0; j < B; ++j) {
    const int c = lane + 32 * j;  // chunk within the warp's stage
    const int r = c / B, piece = c % B;
    if (row0 + r < a.m)
      cp_async16(buf + r * pitch_bytes(B) + 16 * piece, base + (row0 + r) * row_bytes + 16 * piece);
  }
}

// Decode 128 fields of width B from the lane's row chunk and accumulate the
// products with x (int32, 128 entries, broadcast reads).
template <int B, bool SGN, bool NARROW>
__device__ __forceinline__ void decode_mac(const uint8_t* row, const int* __restrict__ xs,
                                           long long& acc) {
  int acc32 = 0;  // NARROW: 128 products of |a| < 2^ba, |x| < 2^bx with ba + bx + 7 <= 31
  const uint4* rv = reinterpret_cast<const uint4*>(row);
  uint32_t w[4 * B + 1];
#pragma unroll
  for (int v = 0; v < B; ++v) {
    uint4 q = rv[v];
    w[4 * v] = q.x;
    w[4 * v + 1] = q.y;
    w[4 * v + 2] = q.z;
    w[4 * v + 3] = q.w;
  }
  w[4 * B] = 0;
  const int4* xv = reinterpret_cast<const int4*>(xs);
#pragma unroll
  for (int f4 = 0; f4 < kKC / 4; ++f4) {
    const int4 xq = xv[f4];
    const int xa[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int f = f4 * 4 + q;
      const int bit = f * B, wi = bit >> 5, s = bit & 31;
      if constexpr (!SGN && B == 32) {
        acc += (long long)w[wi] * (long long)xa[q];
      } else if constexpr (NARROW) {
        uint32_t t;
        if (s + B <= 32)
          t = w[wi] >> s;
        else
          t = __funnelshift_r(w[wi], w[wi + 1], s);
        int v;
        if constexpr (SGN)
          v = (int)(t << (32 - B)) >> (32 - B);
        else
          v = (int)(t & (0xffffffffu >> (32 - B)));
        acc32 += v * xa[q];
      } else {
        uint32_t t;
        if (s + B <= 32)
          t = w[wi] >> s;
        else
          t = __funnelshift_r(w[wi], w[wi + 1], s);
        int v;
        if constexpr (SGN)
          v = (int)(t << (32 - B)) >> (32 - B);
        else
          v = (int)(t & (0xffffffffu >> (32 - B)));
        acc += (long long)v * xa[q];
      }
    }
  }
  if constexpr (NARROW) acc += acc32;
}

__host__ __device__ constexpr uint32_t low_bits(int n) { return n >= 32 ? ~0u : (1u << n) - 1u; }

// Widths whose fields never straddle a byte: a word splits into 8/b
// registers of four byte-lane fields each with one shift and one mask.
__host__ __device__ constexpr bool byte_sliced(int B) { return B == 1 || B == 2 || B == 4 || B == 8; }

// Byte position of x_j (j counted from the start of a 128-aligned slab) in
// the int8 staging, matching the order in which dp4a_stage pairs fields with
// x bytes: natural order, except for the sliced widths, where register k of
// word i holds the fields q = p * (8/b) + k (p = byte 0..3) of that word.
template <int B>
__device__ __forceinline__ uint32_t x8_pos(uint32_t j) {
  if constexpr (B == 1 || B == 2 || B == 4) {
    constexpr uint32_t per = 32u / B, r = 8u / B;
    const uint32_t i = j / per, q = j % per;
    return i * per + (q % r) * 4 + q / r;
  } else {
    return j;
  }
}

// dp4a with unsigned bytes in a and signed (XS) or unsigned bytes in b.
template <bool XS>
__device__ __forceinline__ int dp4a_u(uint32_t a, int b, int c) {
  int d;
  if constexpr (XS)
    asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  else
    asm("dp4a.u32.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// sum over 128 fields of u_j * x_j (u the unsigned or offset-binary field,
// x int8 (XS) or uint8), |sum| <= 128 * 255 * 255 < 2^31.  `xw`: the 32 words
// of x bytes of these 128 columns.
template <int B, bool SGN, bool XS = true>
__device__ __forceinline__ int dp4a_stage(const uint8_t* row, const int* __restrict__ xw) {
  const uint4* rv = reinterpret_cast<const uint4*>(row);
  uint32_t w[4 * B + 1];
#pragma unroll
  for (int v = 0; v < B; ++v) {
    const uint4 q = rv[v];
    w[4 * v] = q.x;
    w[4 * v + 1] = q.y;
    w[4 * v + 2] = q.z;
    w[4 * v + 3] = q.w;
  }
  w[4 * B] = 0;
  if constexpr (SGN) {
#pragma unroll
    for (int i = 0; i < 4 * B; ++i) w[i] ^= group_sign_bits(B, i % B);
  }
  const int4* xv = reinterpret_cast<const int4*>(xw);
  int acc[4] = {0, 0, 0, 0};  // four independent dp4a chains
  if constexpr (byte_sliced(B)) {
    constexpr int R = 8 / B;
    constexpr uint32_t m = low_bits(B) * 0x01010101u;
#pragma unroll
    for (int g = 0; g < 8; ++g) {  // x words 4g..4g+3
      const int4 xq = xv[g];
      const int xa[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int xi = 4 * g + t, i = xi / R, k = xi % R;
        const uint32_t v = B == 8 ? w[i] : (w[i] >> (B * k)) & m;
        acc[t] = dp4a_u<XS>(v, xa[t], acc[t]);
      }
    }
  } else {
    // four fields (4b bits) -> two 16-bit halves of two fields -> four bytes
    constexpr uint32_t m2 = low_bits(2 * B), m1 = low_bits(B) * 0x00010001u;
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int4 xq = xv[g];
      const int xa[4] = {xq.x, xq.y, xq.z, xq.w};
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int c = 4 * g + t;
        const int bit = 4 * B * c, wi = bit >> 5, sh = bit & 31;
        uint32_t x4;
        if (sh + 4 * B <= 32)
          x4 = w[wi] >> sh;
        else
          x4 = __funnelshift_r(w[wi], w[wi + 1], sh);
        const uint32_t u = (x4 & m2) | ((x4 << (16 - 2 * B)) & (m2 << 16));
        const uint32_t v = (u & m1) | ((u << (8 - B)) & (m1 << 8));
        acc[t] = dp4a_u<XS>(v, xa[t], acc[t]);
      }
    }
  }
  return (acc[0] + acc[1]) + (acc[2] + acc[3]);
}

// x slab -> shared memory: int32 (xs[j]), or on the byte-lane path int8 in
// dp4a order followed by the per-warp partial sums of x (xpart).
template <int B, bool DP>
__device__ __forceinline__ void stage_x(const Args& a, int* xs, int* xpart, uint64_t col0,
                                        uint32_t ncols) {
  const int bx = a.hx->width, sx = a.hx->is_signed;
  if constexpr (DP) {
    int8_t* x8 = reinterpret_cast<int8_t*>(xs);
    int part = 0;
    for (uint32_t j = threadIdx.x; j < ncols; j += blockDim.x) {
      const int v = (int)decode_field(a.wx, col0 + j, bx, sx);
      x8[x8_pos<B>(j)] = (int8_t)v;
      part += v;
    }
    for (int d = 16; d; d >>= 1) part += __shfl_xor_sync(0xffffffffu, part, d);
    if (threadIdx.x % 32 == 0) xpart[threadIdx.x / 32] = part;
  } else {
    for (uint32_t j = threadIdx.x; j < ncols; j += blockDim.x)
      xs[j] = (int)decode_field(a.wx, col0 + j, bx, sx);
  }
}

template <int B, bool SGN, bool NARROW, bool DP>
__device__ __noinline__ void body(const Args& a, uint8_t* smem, int* xs, int* xpart,
                                  uint64_t col0, uint32_t ncols) {
  constexpr int K = ring_depth(B);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int pitch = pitch_bytes(B);
  const int stage_bytes = 32 * pitch;
  uint8_t* wbuf = smem + warp * a.warp_region;  // K * stage_bytes <= warp_region
  const uint32_t nst = ncols / kKC;
  const uint64_t rows_per_cta = (uint64_t)blockDim.x;  // 32 rows per warp
  const uint64_t nrb = (a.m + rows_per_cta - 1) / rows_per_cta;
  bool first = true;
  long long corr = 0;  // 2^(b-1) * (sum of the slab's x) on the signed byte-lane path
  // persistent over row blocks: the CTA keeps its column slab (and x)
  for (uint64_t rb = blockIdx.x; rb < nrb; rb += gridDim.x) {
    const uint64_t row0 = rb * rows_per_cta + (uint64_t)warp * 32;
    long long acc = 0;
    Issuer<(B <= 8 ? B : 1)> is;
    auto issue = [&](uint32_t s) {
      uint8_t* buf = wbuf + (s % K) * stage_bytes;
      if constexpr (B <= 8)
        is.issue(buf, s);
      else
        issue_stage<B>(a, buf, row0, col0 + (uint64_t)s * kKC, lane);
    };
    // the first K-1 stages in flight (one commit group per stage, empty or not)
    if (row0 < a.m) {
      if constexpr (B <= 8) is.init(a, row0, col0, lane);
#pragma unroll
      for (int p = 0; p < K - 1; ++p) {
        if ((uint32_t)p < nst) issue(p);
        cp_async_commit();
      }
    }
    if (first) {
      // x staged while the first stages load
      stage_x<B, DP>(a, xs, xpart, col0, ncols);
      __syncthreads();
      first = false;
      if constexpr (DP && SGN) {
        long long xsum = 0;
        for (int k = 0; k < (int)(blockDim.x / 32); ++k) xsum += xpart[k];
        corr = xsum * (1ll << (B - 1));
      }
    }
    if (row0 < a.m) {
      for (uint32_t s = 0; s < nst; ++s) {
        if (s + K - 1 < nst) issue(s + K - 1);
        cp_async_commit();
        cp_async_wait<K - 1>();  // groups complete in order: stage s has landed
        __syncwarp();
        const uint8_t* row = wbuf + (s % K) * stage_bytes + lane * pitch;
        if constexpr (DP)
          acc += dp4a_stage<B, SGN>(row, xs + s * (kKC / 4));
        else
          decode_mac<B, SGN, NARROW>(row, xs + s * kKC, acc);
        __syncwarp();
      }
      if (row0 + lane < a.m)
        atomicAdd(reinterpret_cast<unsigned long long*>(a.y + row0 + lane),
                  (unsigned long long)(acc - corr));
    }
    cp_async_wait<0>();
    __syncwarp();
  }
  if (first) __syncthreads();  // (a CTA with no row block still meets the barrier)
}

// Calls body<b, sign> for the runtime width b, for widths up to BMAX (up to
// min(BMAX, 8) on the byte-lane path).
template <int BMAX, bool NARROW, bool DP, int B = 1>
__device__ __forceinline__ void dispatch(const Args& a, int b, int sgn, uint8_t* smem, int* xs,
                                         int* xpart, uint64_t col0, uint32_t ncols) {
  constexpr int kTop = DP ? (BMAX < 8 ? BMAX : 8) : BMAX;
  if constexpr (B <= kTop) {
    if (b == B) {
      if (sgn)
        body<B, true, NARROW, DP>(a, smem, xs, xpart, col0, ncols);
      else
        body<B, false, NARROW, DP>(a, smem, xs, xpart, col0, ncols);
      return;
    }
    dispatch<BMAX, NARROW, DP, B + 1>(a, b, sgn, smem, xs, xpart, col0, ncols);
  } else {
    // a width the buffer sizes ruled out: report it, never read past them
    if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) set_status(a.out, CCM_E_INPUT);
  }
}

// One kernel per width class (widths <= BMAX), so that the register budget
// of the narrow classes is not set by the 32-bit instances.
template <int BMAX, bool NARROW>
__global__ void __launch_bounds__(256, BMAX <= 8 ? 2 : 1) k_matvec_fast(Args a) {
  extern __shared__ __align__(16) uint8_t smem[];
  if (a.out->status != CCM_OK) return;
  const int b = a.ha->width, sgn = a.ha->is_signed;
  const int bx = a.hx->width, sx = a.hx->is_signed;
  const uint64_t col0 = (uint64_t)blockIdx.y * a.kslab;
  if (col0 >= a.n) return;
  const uint32_t ncols = (uint32_t)umin(a.kslab, a.n - col0);
  // x slab -> shared memory after the stage buffers (staged inside body(),
  // once the first stages are in flight).  The region holds ncols int32; the
  // int8 staging of the byte-lane path uses its first quarter and keeps the
  // per-warp partial sums of x after it.
  int* xs = reinterpret_cast<int*>(smem + a.stage_region);
  int* xpart = xs + ncols / 4;
  if (b <= 8 && (sx ? bx <= 8 : bx <= 7))
    dispatch<BMAX, NARROW, true>(a, b, sgn, smem, xs, xpart, col0, ncols);
  else
    dispatch<BMAX, NARROW, false>(a, b, sgn, smem, xs, xpart, col0, ncols);
}

// CTAs of the class kernel for bmax that fit on one SM with `threads`
// threads and `smem` bytes of dynamic shared memory (host).
int resident_ctas(int bmax, int threads, size_t smem);

// Host launchers, one translation unit per class (matvec_fast{8,16,32}.cu).
// `narrow`: the width bounds give b_a + b_x + 7 <= 31, so 128 products add up
// in 32 bits before each int64 flush.
void launch_matvec_fast8(const Args& a, bool narrow, dim3 grid, int threads, size_t smem,
                         cudaStream_t st);
void launch_matvec_fast16(const Args& a, bool narrow, dim3 grid, int threads, size_t smem,
                          cudaStream_t st);
void launch_matvec_fast32(const Args& a, bool narrow, dim3 grid, int threads, size_t smem,
                          cudaStream_t st);

// ---------------------------------------------------------------------------
// Row-streaming kernel (the whole of x fits in shared memory).
//
// The row-major packed A is cut into warp-stages of up to 32 consecutive
// 128-field chunks of one row: 4096 columns, 512*b contiguous bytes (the last
// stage of a row holds the rest).  Warp w of the W warps of the grid takes
// the contiguous range [T w / W, T (w + 1) / W) of the T warp-stages, so each
// warp streams one contiguous stretch of A through its cp.async ring
// (coalesced 16-byte copies; chunk q of a stage lands at q * pitch, the same
// odd-multiple-of-16 pitch as above) and the work is balanced to one stage.
// Lane l decodes chunk l of the stage against its own 128 x values, staged
// once per CTA for all columns with rows of 128 padded to an odd multiple of
// 16 bytes (conflict-free 16-byte shared loads across the lanes).  A row's
// partial sums are reduced across the warp and added to y when the warp
// leaves the row (atomically: a row may be split between two warps).
//
// Byte-lane path when b <= 8 and b_x <= 8: x staged as bytes (int8 or
// uint8), dp4a per four fields; signed fields in offset binary, corrected by
// 2^(b-1) times the sum of x over each 128-column chunk (kept beside x).
// Otherwise x is staged as int32 and fields are multiplied one by one.
namespace rows {

constexpr int kChunksPerStage = 32;
constexpr int kXPitch8 = 144;   // 128 x bytes + 16 pad
constexpr int kXPitch32 = 528;  // 128 x int32 + 16 pad

struct RowArgs {
  ccm_header* out;
  const ccm_header* ha;
  const uint32_t* wa;
  const ccm_header* hx;
  const uint32_t* wx;
  uint64_t m, n;
  uint32_t warp_region;  // ring bytes per warp (warp_region_bytes of the width bound)
  uint32_t x_offset;     // byte offset of the x staging: after every warp's ring
  int64_t* y;            // int64 sums, zeroed before launch
  const uint8_t* ximg;   // the x staging image (k_xprep), copied to shared memory as is
};

// Byte position of x_j in a 128-column chunk for field width b (runtime b;
// x8_pos<B> with B = b).
__device__ __forceinline__ uint32_t x8_pos_rt(uint32_t f, int b) {
  if (b == 1 || b == 2 || b == 4) {
    const uint32_t per = 32u / b, r = 8u / b;
    const uint32_t i = f / per, q = f % per;
    return i * per + (q % r) * 4 + q / r;
  }
  return f;
}

// Shared bytes of the x staging (x rows plus the per-chunk sums of x).
__host__ __device__ constexpr uint64_t x_region_bytes(uint64_t n, bool bytes) {
  return n / kKC * ((bytes ? kXPitch8 : kXPitch32) + 4);
}

__device__ __forceinline__ void flush_row(long long& acc, int64_t* y, uint64_t row, int lane) {
  for (int d = 16; d; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if (lane == 0 && acc != 0) atomicAdd(reinterpret_cast<unsigned long long*>(y + row),
                                      (unsigned long long)acc);
  acc = 0;
}

template <int B, bool SGN, bool NARROW, bool DP, bool XS>
__device__ __noinline__ void body(const RowArgs& a, uint8_t* smem) {
  constexpr int K = ring_depth(B);
  constexpr int pitch = pitch_bytes(B);
  constexpr int stage_bytes = kChunksPerStage * pitch;
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  uint8_t* ring = smem + warp * a.warp_region;  // K * stage_bytes <= warp_region
  uint8_t* xb = smem + a.x_offset;
  const uint32_t nchunks = (uint32_t)(a.n / kKC);
  int* csum = reinterpret_cast<int*>(xb + (uint64_t)nchunks * (DP ? kXPitch8 : kXPitch32));
  const uint32_t S = (nchunks + kChunksPerStage - 1) / kChunksPerStage;  // stages per row
  const uint64_t T = a.m * S;
  const uint64_t nw = blockDim.x / 32;
  const uint64_t GW = (uint64_t)gridDim.x * nw, gw = (uint64_t)blockIdx.x * nw + warp;
  const uint64_t t0 = T / GW * gw + umin(gw, T % GW);
  const uint64_t t1 = t0 + T / GW + (gw < T % GW ? 1 : 0);
  const uint64_t row_bytes = a.n / 8 * B;
  const uint8_t* A = reinterpret_cast<const uint8_t*>(a.wa);
  // where this lane's 16-byte pieces q = lane + 32 j of a stage land
  uint32_t soff[B <= 8 ? B : 1];
  if constexpr (B <= 8) {
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const int q = lane + 32 * j;
      soff[j] = (uint32_t)((q / B) * pitch + 16 * (q % B));
    }
  }
  // producer position (row, stage of the row) of the next stage to issue
  uint64_t prow = t0 / S;
  uint32_t pseg = (uint32_t)(t0 % S);
  auto issue_next = [&](uint32_t slot) {
    const uint32_t ch = umin(kChunksPerStage, nchunks - pseg * kChunksPerStage);
    const uint8_t* g = A + prow * row_bytes + (uint64_t)pseg * (512 * B);
    const unsigned sb = (unsigned)__cvta_generic_to_shared(ring + slot * stage_bytes);
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const uint32_t q = lane + 32 * j;
      if (q < ch * B) {
        uint32_t so;
        if constexpr (B <= 8)
          so = soff[j];
        else
          so = (q / B) * pitch + 16 * (q % B);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sb + so), "l"(g + 16 * q)
                     : "memory");
      }
    }
    if (++pseg == S) pseg = 0, ++prow;
  };
  // x image -> shared memory (one commit group), then the first K-1 stages
  {
    const unsigned xs = (unsigned)__cvta_generic_to_shared(xb);
    const uint32_t xbytes = (nchunks * ((DP ? kXPitch8 : kXPitch32) + 4) + 15) & ~15u;
    for (uint32_t o = 16 * threadIdx.x; o < xbytes; o += 16 * blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(xs + o), "l"(a.ximg + o)
                   : "memory");
    cp_async_commit();
  }
#pragma unroll
  for (int p = 0; p < K - 1; ++p) {
    if (t0 + p < t1) issue_next(p);
    cp_async_commit();
  }
  cp_async_wait<K - 1>();  // this thread's share of x has landed
  __syncthreads();         // and everyone's
  long long acc = 0;
  uint64_t row = t0 / S;
  uint32_t seg = (uint32_t)(t0 % S);
  for (uint64_t t = t0; t < t1; ++t) {
    const uint32_t k = (uint32_t)(t - t0);
    if (t + K - 1 < t1) issue_next((k + K - 1) % K);
    cp_async_commit();
    cp_async_wait<K - 1>();  // groups complete in order: stage t has landed
    __syncwarp();
    const uint32_t ch = umin(kChunksPerStage, nchunks - seg * kChunksPerStage);
    if ((uint32_t)lane < ch) {
      const uint32_t c = seg * kChunksPerStage + lane;
      const uint8_t* rp = ring + (k % K) * stage_bytes + lane * pitch;
      if constexpr (DP) {
        acc += dp4a_stage<B, SGN, XS>(rp, reinterpret_cast<const int*>(xb + c * kXPitch8));
        if constexpr (SGN) acc -= (long long)csum[c] * (1ll << (B - 1));
      } else {
        decode_mac<B, SGN, NARROW>(rp, reinterpret_cast<const int*>(xb + c * kXPitch32), acc);
      }
    }
    __syncwarp();
    if (++seg == S || t + 1 == t1) {  // leaving the row (or the range)
      flush_row(acc, a.y, row, lane);
      seg = 0;
      ++row;
    }
  }
  cp_async_wait<0>();
}

template <int BMAX, bool NARROW, bool DP, bool XS, int B = 1>
__device__ __forceinline__ void dispatch(const RowArgs& a, int b, int sgn, uint8_t* smem) {
  constexpr int kTop = DP ? (BMAX < 8 ? BMAX : 8) : BMAX;
  if constexpr (B <= kTop) {
    if (b == B) {
      if (sgn)
        body<B, true, NARROW, DP, XS>(a, smem);
      else
        body<B, false, NARROW, DP, XS>(a, smem);
      return;
    }
    dispatch<BMAX, NARROW, DP, XS, B + 1>(a, b, sgn, smem);
  } else {
    // a width the buffer sizes ruled out: report it, never read past them
    if (threadIdx.x == 0 && blockIdx.x == 0) set_status(a.out, CCM_E_INPUT);
  }
}

template <int BMAX, bool NARROW>
__global__ void __launch_bounds__(256, BMAX <= 8 ? 2 : 1) k_matvec_rows(RowArgs a) {
  extern __shared__ __align__(16) uint8_t smem[];
  if (a.out->status != CCM_OK) return;
  const int b = a.ha->width, sgn = a.ha->is_signed;
  const int bx = a.hx->width, sx = a.hx->is_signed;
  if (b <= 8 && bx <= 8) {
    if (sx)
      dispatch<BMAX, NARROW, true, true>(a, b, sgn, smem);
    else
      dispatch<BMAX, NARROW, true, false>(a, b, sgn, smem);
  } else {
    dispatch<BMAX, NARROW, false, true>(a, b, sgn, smem);
  }
}

// Host side, one translation unit per class (matvec_rows{8,16,32}.cu); the
// x image kernel k_xprep lives in matvec.cu.
int resident_ctas(int bmax, int threads, size_t smem);
void launch(int bmax, const RowArgs& a, bool narrow, unsigned grid, int threads, size_t smem,
            cudaStream_t st);

}  // namespace rows

}  // namespace mvf
}  // namespace ccm
