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
#pragma once

#include "ccm_device.cuh"

namespace ccm {
namespace mvf {

constexpr int kKC = 128;   // columns per stage
constexpr int kStages = 2;  // cp.async double buffering

__host__ __device__ __forceinline__ int pitch_bytes(int b) { return (b & 1) ? 16 * b : 16 * (b + 1); }

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
  int64_t* y;                  // int64 partial sums, zeroed before launch
};

// Issue the cp.async copies of one stage (32 rows x 16*B bytes) of a warp.
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

template <int B, bool SGN, bool NARROW>
__device__ __noinline__ void body(const Args& a, uint8_t* smem, int* xs, uint64_t col0,
                                  uint32_t ncols) {
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int pitch = pitch_bytes(B);
  const int stage_bytes = 32 * pitch;
  uint8_t* wbuf = smem + warp * kStages * stage_bytes;
  const uint32_t nst = ncols / kKC;
  const uint64_t rows_per_cta = (uint64_t)blockDim.x;  // 32 rows per warp
  const uint64_t nrb = (a.m + rows_per_cta - 1) / rows_per_cta;
  bool first = true;
  // persistent over row blocks: the CTA keeps its column slab (and x)
  for (uint64_t rb = blockIdx.x; rb < nrb; rb += gridDim.x) {
    const uint64_t row0 = rb * rows_per_cta + (uint64_t)warp * 32;
    long long acc = 0;
    if (row0 < a.m) {
      issue_stage<B>(a, wbuf, row0, col0, lane);
      cp_async_commit();
    }
    if (first) {
      __syncthreads();  // x slab decoded by the whole CTA
      first = false;
    }
    if (row0 < a.m) {
      for (uint32_t s = 0; s < nst; ++s) {
        if (s + 1 < nst) issue_stage<B>(a, wbuf + ((s + 1) % kStages) * stage_bytes, row0,
                                        col0 + (uint64_t)(s + 1) * kKC, lane);
        cp_async_commit();
        cp_async_wait<1>();
        __syncwarp();
        decode_mac<B, SGN, NARROW>(wbuf + (s % kStages) * stage_bytes + lane * pitch, xs + s * kKC,
                                   acc);
        __syncwarp();
      }
      if (row0 + lane < a.m)
        atomicAdd(reinterpret_cast<unsigned long long*>(a.y + row0 + lane), (unsigned long long)acc);
    }
    cp_async_wait<0>();
    __syncwarp();
  }
  if (first) __syncthreads();  // (a CTA with no row block still meets the barrier)
}

// Calls body<b, sign> for the runtime width b, for widths up to BMAX.
template <int BMAX, bool NARROW, int B = 1>
__device__ __forceinline__ void dispatch(const Args& a, int b, int sgn, uint8_t* smem, int* xs,
                                         uint64_t col0, uint32_t ncols) {
  if constexpr (B <= BMAX) {
    if (b == B) {
      if (sgn)
        body<B, true, NARROW>(a, smem, xs, col0, ncols);
      else
        body<B, false, NARROW>(a, smem, xs, col0, ncols);
      return;
    }
    dispatch<BMAX, NARROW, B + 1>(a, b, sgn, smem, xs, col0, ncols);
  } else {
    // a width the buffer sizes ruled out: report it, never read past them
    if (threadIdx.x == 0 && blockIdx.x == 0 && blockIdx.y == 0) set_status(a.out, CCM_E_INPUT);
  }
}

// One kernel per width class (widths <= BMAX), so that the register budget
// of the narrow classes is not set by the 32-bit instances.
template <int BMAX, bool NARROW>
__global__ void __launch_bounds__(256) k_matvec_fast(Args a) {
  extern __shared__ __align__(16) uint8_t smem[];
  if (a.out->status != CCM_OK) return;
  const int b = a.ha->width, sgn = a.ha->is_signed;
  const int bx = a.hx->width, sx = a.hx->is_signed;
  const uint64_t col0 = (uint64_t)blockIdx.y * a.kslab;
  if (col0 >= a.n) return;
  const uint32_t ncols = (uint32_t)umin(a.kslab, a.n - col0);
  // x slab -> shared int32 (after the stage buffers); the barrier that
  // publishes it is inside body(), after the first stage is in flight
  int* xs = reinterpret_cast<int*>(smem + a.stage_region);
  for (uint32_t j = threadIdx.x; j < ncols; j += blockDim.x)
    xs[j] = (int)decode_field(a.wx, col0 + j, bx, sx);
  dispatch<BMAX, NARROW>(a, b, sgn, smem, xs, col0, ncols);
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

}  // namespace mvf
}  // namespace ccm
