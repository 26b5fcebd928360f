// matmul_tc.cu -- exact integer C = A B on the tcgen05 tensor cores.
//
// GB300 (sm_103a) has no integer tensor-core MMA (tcgen05.mma .kind::i8 is
// rejected by ptxas for this target), so the product is computed through an
// exact decomposition into 4-bit digits, which e4m3 represents exactly:
//
//   a = sum_{l < L} d_l 16^l,  d_l in [0, 15] for l < L-1,  d_{L-1} = a >> 4(L-1)
//
// (two's complement bits for the low digits, an arithmetic shift for the top
// one, so the top digit is in [-8, 7] for signed fields and [0, 15] for
// unsigned ones; L = ceil(b / 4)).  Then
//
//   C = sum_c 16^c S_c,   S_c = sum_{l + m = c} A_l B_m,
//
// and every S_c is a dense e4m3 x e4m3 GEMM accumulated in fp32 in tensor
// memory.  Each product of two digits is at most 225 in magnitude, so an
// S_c entry is at most L * k * 225 < 2^24 whenever k * L * 225 < 2^24: every
// partial sum is an integer that fp32 holds exactly, and the epilogue
// converts S_c to int64 and combines the classes exactly.
//
// Pipeline (one CTA of 4 warps per 128 x BN output tile):
//   k_limbs_a / k_limbs_bt  packed A, B -> digit planes in e4m3, K-major,
//                           zero padded to the tile sizes (B transposed)
//   k_mm_tc                 warp 0: TMA producer (128-byte swizzled tiles of
//                           every digit plane, mbarrier pipeline); warp 1:
//                           one thread issues tcgen05.mma for every digit
//                           pair into the accumulator of its class; all four
//                           warps: epilogue (tcgen05.ld, exact int64 combine,
//                           width statistics of C merged into C's header)
// The int64 C is then packed by the pack pass of the pack engine.
//
// Every wait on an mbarrier is bounded; a wait that gives up records
// CCM_E_TIMEOUT in C's header and the CTA frees its tensor memory and exits.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "ccm_device.cuh"
#include "kernels.h"
#include "matmul_tc.h"

namespace ccm {
namespace tc {

constexpr int kBM = 128;    // rows of A / C per tile (UMMA M)
constexpr int kBK = 128;    // K elements (= bytes of e4m3) per pipeline stage
constexpr uint32_t kSpinLimit = 1u << 26;  // bounded mbarrier waits
constexpr uint32_t kGroupM = 8;            // tile rows per raster group

// Tile geometry for L digits per operand.
struct Geo {
  int L = 0;        // digits per field
  int classes = 0;  // 2L - 1 accumulators
  int bn = 0;       // UMMA N
  int stages = 0;
  int accs = 0;     // accumulator sets in tensor memory (2: a tile's epilogue
                    // overlaps the next tile's MMAs)
  int tmem_cols = 0;
};

__host__ __device__ constexpr Geo geometry(int L) {
  Geo g;
  g.L = L;
  g.classes = 2 * L - 1;
  g.bn = L == 1 ? 256 : (L == 2 ? 128 : 64);
  const int stage_bytes = L * kBK * (kBM + g.bn);
  g.stages = 200 * 1024 / stage_bytes;
  if (g.stages > 4) g.stages = 4;
  const int cols = g.classes * g.bn;
  g.accs = 2 * cols <= 512 ? 2 : 1;
  int p = 32;
  while (p < g.accs * cols) p <<= 1;
  g.tmem_cols = p;
  return g;
}

__host__ __device__ inline uint64_t round_up(uint64_t v, uint64_t m) { return (v + m - 1) / m * m; }

// ---------------------------------------------------------------------------
// e4m3 encoding of a digit in [-8, 15] (exact: at most 4 significant bits).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint8_t e4m3_of_digit(int d) {
  if (d == 0) return 0;
  uint32_t sign = d < 0 ? 0x80u : 0u;
  uint32_t v = (uint32_t)(d < 0 ? -d : d);  // 1..15
  int e = 31 - __clz(v);                    // 0..3
  uint32_t mant = (v << (3 - e)) & 7u;
  return (uint8_t)(sign | ((uint32_t)(e + 7) << 3) | mant);
}

__device__ __forceinline__ int digit(int64_t a, int l, int L) {
  return l == L - 1 ? (int)(a >> (4 * l)) : (int)((a >> (4 * l)) & 15);
}

// ---------------------------------------------------------------------------
// Fields of exactly 4L bits: digit l of field f is nibble f L + l of the
// packed stream (the stream is LSB-first and the digits are the value's
// nibbles, the top one taken as signed for two's complement fields), so the
// digit planes are a strided nibble gather.  Four nibbles become four e4m3
// bytes by table lookup with byte permutes: the low three bits of a nibble
// select a byte of an 8-byte table (entries 0..7, or 8..15 / the negative
// digits -8..-1), bit 3 picks which table.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t e4m3_of_nibbles(uint32_t x, bool top_signed) {
  // e4m3 of 0..7, 8..15, and of -8..-1 (nibbles 8..15 of a signed digit)
  constexpr uint32_t kLo0 = 0x44403800u, kLo1 = 0x4E4C4A48u;
  constexpr uint32_t kHi0 = 0x53525150u, kHi1 = 0x57565554u;
  constexpr uint32_t kNeg0 = 0xCACCCED0u, kNeg1 = 0xB8C0C4C8u;
  const uint32_t sel = x & 0x7777u;
  const uint32_t lo = __byte_perm(kLo0, kLo1, sel);
  const uint32_t hi = top_signed ? __byte_perm(kNeg0, kNeg1, sel) : __byte_perm(kHi0, kHi1, sel);
  const uint32_t big = __byte_perm(0u, 0xFFFFFFFFu, (x >> 1) & 0x4444u);  // 0xFF where bit 3
  return (lo & ~big) | (hi & big);
}

// The 8 digit bytes of plane l for 8 consecutive fields held in w[0..L)
// (32 L bits: 8 fields of 4L bits), as two words (fields 0..3, 4..7).
template <int L>
__device__ __forceinline__ uint2 plane_bytes8(const uint32_t (&w)[L], int l, bool top_signed) {
  uint32_t x0 = 0, x1 = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int j = q * L + l;  // nibble index in the 8-field group
    const uint32_t nib = (w[j >> 3] >> (4 * (j & 7))) & 15u;
    if (q < 4)
      x0 |= nib << (4 * q);
    else
      x1 |= nib << (4 * (q - 4));
  }
  return make_uint2(e4m3_of_nibbles(x0, top_signed), e4m3_of_nibbles(x1, top_signed));
}

// The L words holding fields [f0, f0 + 8) of a stream of 4L-bit fields (f0 a
// multiple of 8, so the group starts on a word).
template <int L>
__device__ __forceinline__ void load_group8(const uint32_t* __restrict__ w, uint64_t f0,
                                            uint32_t (&out)[L]) {
  const uint32_t* p = w + f0 * L / 8;
  if constexpr (L == 1) {
    out[0] = __ldg(p);
  } else if constexpr (L == 2) {
    const uint2 v = __ldg(reinterpret_cast<const uint2*>(p));
    out[0] = v.x;
    out[1] = v.y;
  } else if constexpr (L == 4) {
    const uint4 v = __ldg(reinterpret_cast<const uint4*>(p));
    out[0] = v.x;
    out[1] = v.y;
    out[2] = v.z;
    out[3] = v.w;
  } else {
#pragma unroll
    for (int i = 0; i < L; ++i) out[i] = __ldg(p + i);
  }
}

// A (m x k, row-major, k % 8 == 0) with fields of exactly 4L bits ->
// planes [L][m_pad][k_pad]: thread per 8 consecutive fields of a row.
template <int L>
__device__ void limbs_a_nibbles(const uint32_t* __restrict__ w, int sgn, uint64_t m, uint64_t k,
                                uint64_t m_pad, uint64_t k_pad, uint8_t* __restrict__ planes) {
  const uint64_t plane = m_pad * k_pad;
  const uint32_t groups = (uint32_t)(k_pad / 8);
  for (uint64_t i = blockIdx.x; i < m_pad; i += gridDim.x) {
    for (uint32_t q = threadIdx.x; q < groups; q += blockDim.x) {
      const uint64_t kk = 8ull * q;
      uint2 out[L];
      if (i < m && kk < k) {
        uint32_t wg[L];
        load_group8<L>(w, i * k + kk, wg);
#pragma unroll
        for (int l = 0; l < L; ++l) out[l] = plane_bytes8<L>(wg, l, sgn && l == L - 1);
      } else {
#pragma unroll
        for (int l = 0; l < L; ++l) out[l] = make_uint2(0u, 0u);
      }
#pragma unroll
      for (int l = 0; l < L; ++l)
        *reinterpret_cast<uint2*>(planes + l * plane + i * k_pad + kk) = out[l];
    }
  }
}

// A (m x k, row-major) -> planes [L][m_pad][k_pad] of e4m3 digits.
__global__ void k_limbs_a(const ccm_header* out, const ccm_header* h, const uint32_t* __restrict__ w,
                          uint64_t m, uint64_t k, uint64_t m_pad, uint64_t k_pad, int L,
                          uint8_t* __restrict__ planes) {
  if (out->status != CCM_OK) return;
  const int b = h->width, sgn = h->is_signed;
  if (b == 4 * L && k % 8 == 0) {  // nibble-aligned fields
    switch (L) {
      case 1: limbs_a_nibbles<1>(w, sgn, m, k, m_pad, k_pad, planes); return;
      case 2: limbs_a_nibbles<2>(w, sgn, m, k, m_pad, k_pad, planes); return;
      case 3: limbs_a_nibbles<3>(w, sgn, m, k, m_pad, k_pad, planes); return;
      case 4: limbs_a_nibbles<4>(w, sgn, m, k, m_pad, k_pad, planes); return;
      default: break;
    }
  }
  const uint64_t quads = m_pad * k_pad / 4;
  const uint64_t plane = m_pad * k_pad;
  for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < quads;
       q += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t e0 = 4 * q, i = e0 / k_pad, kk = e0 % k_pad;
    int64_t v[4];
#pragma unroll
    for (int t = 0; t < 4; ++t)
      v[t] = (i < m && kk + t < k) ? decode_field(w, i * k + kk + t, b, sgn) : 0;
    for (int l = 0; l < L; ++l) {
      uint32_t word = 0;
#pragma unroll
      for (int t = 0; t < 4; ++t) word |= (uint32_t)e4m3_of_digit(digit(v[t], l, L)) << (8 * t);
      *reinterpret_cast<uint32_t*>(planes + l * plane + e0) = word;
    }
  }
}

// B (k x n, row-major) -> planes [L][n_pad][k_pad] (transposed, K-major).
__global__ void __launch_bounds__(256) k_limbs_bt(const ccm_header* out, const ccm_header* h,
                                                  const uint32_t* __restrict__ w, uint64_t k,
                                                  uint64_t n, uint64_t n_pad, uint64_t k_pad, int L,
                                                  uint8_t* __restrict__ planes) {
  __shared__ uint8_t tile[4][32][64 + 4];  // [digit][j][kk]
  if (out->status != CCM_OK) return;
  const int b = h->width, sgn = h->is_signed;
  const uint64_t plane = n_pad * k_pad;
  const uint64_t tiles_k = k_pad / 64, tiles_n = n_pad / 32;
  // nibble-aligned fields (b = 4L <= 16) and rows of whole 8-field groups:
  // thread t reads fields j = 8 (t % 4) .. + 7 of row kk = t / 4 of the tile
  const bool nib = b == 4 * L && L <= 4 && n % 8 == 0;
  for (uint64_t t = blockIdx.x; t < tiles_k * tiles_n; t += gridDim.x) {
    const uint64_t k0 = (t % tiles_k) * 64, j0 = (t / tiles_k) * 32;
    for (int l0 = 0; l0 < L; l0 += 4) {
      if (nib) {
        const int kk = threadIdx.x / 4, jg = 8 * (threadIdx.x % 4);
        const uint64_t gk = k0 + kk, gj = j0 + jg;
        uint2 bytes[4] = {};
        const bool live = gk < k && gj < n;
        switch (L) {
#define CCM_TC_NIB(LL)                                                           \
  case LL:                                                                       \
    if (live) {                                                                  \
      uint32_t wg[LL];                                                           \
      load_group8<LL>(w, gk * n + gj, wg);                                       \
      _Pragma("unroll") for (int l = 0; l < LL; ++l) bytes[l] =                  \
          plane_bytes8<LL>(wg, l, sgn && l == LL - 1);                           \
    }                                                                            \
    break;
          CCM_TC_NIB(1) CCM_TC_NIB(2) CCM_TC_NIB(3) CCM_TC_NIB(4)
#undef CCM_TC_NIB
          default: break;
        }
        for (int l = 0; l < L; ++l) {
#pragma unroll
          for (int q = 0; q < 8; ++q)
            tile[l][jg + q][kk] = (uint8_t)((q < 4 ? bytes[l].x : bytes[l].y) >> (8 * (q & 3)));
        }
      } else {
        // read: thread covers (kk = threadIdx.x / 32 + 8 r, j = threadIdx.x % 32)
        for (int r = 0; r < 8; ++r) {
          const int kk = threadIdx.x / 32 + 8 * r, j = threadIdx.x % 32;
          const uint64_t gk = k0 + kk, gj = j0 + j;
          const int64_t v = (gk < k && gj < n) ? decode_field(w, gk * n + gj, b, sgn) : 0;
          for (int l = l0; l < L && l < l0 + 4; ++l)
            tile[l - l0][j][kk] = e4m3_of_digit(digit(v, l, L));
        }
      }
      __syncthreads();
      // write: 32 rows (j) x 64 bytes per digit plane, 16 bytes per thread
      for (int l = l0; l < L && l < l0 + 4; ++l) {
        const int j = threadIdx.x / 4, part = threadIdx.x % 4;
        if (threadIdx.x < 128) {
          const uint8_t* src = &tile[l - l0][j][16 * part];
          uint4 v;
          v.x = src[0] | src[1] << 8 | src[2] << 16 | (uint32_t)src[3] << 24;
          v.y = src[4] | src[5] << 8 | src[6] << 16 | (uint32_t)src[7] << 24;
          v.z = src[8] | src[9] << 8 | src[10] << 16 | (uint32_t)src[11] << 24;
          v.w = src[12] | src[13] << 8 | src[14] << 16 | (uint32_t)src[15] << 24;
          *reinterpret_cast<uint4*>(planes + l * plane + (j0 + j) * k_pad + k0 + 16 * part) = v;
        }
      }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// PTX wrappers (sm_100+ family: tcgen05, TMA, mbarrier)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;\n" : "=l"(t));
  return t;
}

// Bounded wait for the phase with parity `parity`: gives up (returns false)
// after about two seconds, or after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t addr = smem_u32(bar);
  uint64_t t0 = 0;
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 1023) == 0) {
      const uint64_t now = globaltimer_ns();
      if (it == 0)
        t0 = now;
      else if (now - t0 > 2000000000ull)
        return false;
    }
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];\n" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, rows of 128 bytes in the
// 128-byte swizzle pattern, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);  // start address
  d |= (uint64_t)1 << 16;                    // leading byte offset (unused for this layout)
  d |= (uint64_t)(1024 >> 4) << 32;          // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                    // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                    // swizzle: 128 bytes
  return d;
}

// Instruction descriptor: kind::f8f6f4, A = B = e4m3, D = f32, both K-major.
__host__ __device__ constexpr uint32_t idesc_e4m3_f32(int m, int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(bar))
      : "memory");
}

// tcgen05.ld of 32 columns without the wait (several in flight, then
// tmem_ld_wait before the registers are used).
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

struct MmArgs {
  ccm_header* out;      // C header: status, width statistics
  int64_t* c;           // int64 C, m x n row-major
  uint64_t m, n;
  uint32_t k_blocks;    // k_pad / kBK
  uint32_t a_rows_pad;  // rows per A digit plane (m_pad)
  uint32_t b_rows_pad;  // rows per B digit plane (n_pad)
  uint32_t tiles_n;     // n_pad / bn
  uint32_t tiles_m;     // m_pad / kBM
  int L;
  int c32;              // 1: C is written as int32 (the output capacity bounds its width by 31)
};

// Output tile t (grouped raster): consecutive tiles sweep the tile columns
// of a group of kGroupM tile rows before the next group.
__device__ __forceinline__ void tile_coords(uint32_t t, uint32_t tiles_m, uint32_t tiles_n,
                                            uint32_t& tm, uint32_t& tn) {
  const uint32_t per_group = kGroupM * tiles_n, group = t / per_group;
  const uint32_t first_m = group * kGroupM;
  const uint32_t gm = tiles_m - first_m < kGroupM ? tiles_m - first_m : kGroupM;
  const uint32_t in_group = t - group * per_group;
  tm = first_m + in_group % gm;
  tn = in_group / gm;
}

// Persistent, warp-specialised: one CTA per SM walks the output tiles t =
// blockIdx.x, + gridDim.x, ...  Warp 0 (one thread) streams the digit-plane
// tiles of every k block of every tile through the S-stage ring (TMA,
// mbarriers); warp 1 allocates tensor memory and one of its threads issues
// the MMAs of tile i into accumulator set i % accs, once the epilogue has
// emptied that set; warps 2-5 (tensor-memory lane quadrants 2, 3, 0, 1) read
// the classes of each finished tile, combine them exactly and store C.  The
// producer runs on into the next tile's loads while the current one is
// finished, and with two accumulator sets (one digit) the next tile's MMAs
// run during the previous tile's epilogue.
constexpr int kThreadsP = 192;

template <int L>
__global__ void __launch_bounds__(kThreadsP, 1)
    k_mm_tc(const __grid_constant__ CUtensorMap tm_a, const __grid_constant__ CUtensorMap tm_b,
            MmArgs args) {
  constexpr Geo G = geometry(L);
  constexpr int BN = G.bn, S = G.stages, C = G.classes, NACC = G.accs;
  constexpr uint32_t ACC_COLS = (uint32_t)(C * BN);          // columns of one accumulator set
  constexpr uint32_t A_TILE = kBM * kBK, B_TILE = BN * kBK;  // bytes per digit plane tile
  constexpr uint32_t STAGE = L * (A_TILE + B_TILE);
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~(uintptr_t)1023);
  __shared__ uint64_t full_bar[S], empty_bar[S], acc_full[NACC], acc_empty[NACC];
  __shared__ uint32_t tmem_base_s;
  __shared__ int skip_s;
  __shared__ volatile int abort_s;
  __shared__ uint32_t issued_s;  // k blocks whose loads the producer issued (all tiles)

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  // one read of the status for the whole CTA (another CTA may change it)
  if (threadIdx.x == 0) skip_s = args.out->status != CCM_OK;
  __syncthreads();
  if (skip_s) return;
  const uint32_t tiles = args.tiles_m * args.tiles_n;
  const uint32_t nk = args.k_blocks;

  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);  // one arrival per epilogue warp
    }
    abort_s = 0;
    issued_s = 0;
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(&tmem_base_s)),
                 "r"((uint32_t)G.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  const uint32_t tmem = tmem_base_s;

  uint64_t orv = 0;
  uint32_t neg = 0;
  if (warp == 0) {
    if (lane == 0) {
      // TMA producer over every k block of every tile of this CTA
      uint32_t g = 0;
      for (uint32_t t = blockIdx.x; t < tiles && !abort_s; t += gridDim.x) {
        uint32_t tm, tn;
        tile_coords(t, args.tiles_m, args.tiles_n, tm, tn);
        for (uint32_t kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % S;
          if (g >= (uint32_t)S && !mbar_wait(&empty_bar[s], ((g / S) - 1) & 1)) {
            abort_s = 1;
            break;
          }
          if (abort_s) break;
          uint8_t* st = smem + s * STAGE;
          mbar_expect_tx(&full_bar[s], STAGE);
          for (int l = 0; l < L; ++l) {
            tma_load_2d(st + l * A_TILE, &tm_a, &full_bar[s], kb * kBK,
                        l * args.a_rows_pad + tm * kBM);
            tma_load_2d(st + L * A_TILE + l * B_TILE, &tm_b, &full_bar[s], kb * kBK,
                        l * args.b_rows_pad + tn * BN);
          }
          issued_s = g + 1;
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // MMA issuer
      constexpr uint32_t idesc = idesc_e4m3_f32(kBM, BN);
      uint32_t g = 0, i = 0;
      bool ok = true;
      for (uint32_t t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++i) {
        const uint32_t a = i % NACC;
        if (i >= (uint32_t)NACC && !mbar_wait(&acc_empty[a], ((i / NACC) - 1) & 1)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        const uint32_t acc0 = tmem + a * ACC_COLS;
        uint32_t started = 0;  // classes already holding a partial sum
        for (uint32_t kb = 0; kb < nk; ++kb, ++g) {
          const int s = g % S;
          if (abort_s || !mbar_wait(&full_bar[s], (g / S) & 1)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
          const uint32_t st = smem_u32(smem + s * STAGE);
#pragma unroll
          for (int l = 0; l < L; ++l) {
#pragma unroll
            for (int mm = 0; mm < L; ++mm) {
              const int c = l + mm;
              const uint32_t a0 = st + l * A_TILE, b0 = st + L * A_TILE + mm * B_TILE;
#pragma unroll
              for (int kk = 0; kk < kBK / 32; ++kk) {
                const uint32_t acc = ((started >> c) & 1u) | (kk > 0 ? 1u : 0u);
                mma_e4m3(acc0 + c * BN, smem_desc_sw128(a0 + 32 * kk),
                         smem_desc_sw128(b0 + 32 * kk), idesc, acc);
              }
              started |= 1u << c;
            }
          }
          mma_commit(&empty_bar[s]);  // frees the stage once these MMAs have read it
        }
        mma_commit(&acc_full[a]);  // (also when giving up: the MMAs issued so far complete)
      }
      if (!ok) abort_s = 1;
    }
  } else {
    // epilogue: tensor-memory lane quadrant q of every finished tile
    const int q = warp % 4;
    const uint32_t lane_base = (uint32_t)(q * 32) << 16;
    uint32_t i = 0;
    for (uint32_t t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
      const uint32_t a = i % NACC;
      // (one decision for the whole warp: the tensor-memory loads are warp-wide)
      if (!__all_sync(0xffffffffu, mbar_wait(&acc_full[a], (i / NACC) & 1))) {
        abort_s = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
      if (__any_sync(0xffffffffu, abort_s != 0)) break;
      uint32_t tm, tn;
      tile_coords(t, args.tiles_m, args.tiles_n, tm, tn);
      const uint64_t row = (uint64_t)tm * kBM + q * 32 + lane;
      const uint32_t acc0 = tmem + lane_base + a * ACC_COLS;
#pragma unroll 1
      for (int col0 = 0; col0 < BN; col0 += 32) {
        int64_t acc[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] = 0;
        if constexpr (C <= 3) {
          // two classes' loads in flight at a time (for more classes the
          // registers this takes cost more than the overlap gains)
#pragma unroll 1
          for (int c = 0; c < C; c += 2) {
            uint32_t r0[32], r1[32];
            tmem_ld32_async(acc0 + c * BN + col0, r0);
            if (c + 1 < C) tmem_ld32_async(acc0 + (c + 1) * BN + col0, r1);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j)
              acc[j] += (int64_t)__float2ll_rn(__uint_as_float(r0[j])) * (int64_t)(1ll << (4 * c));
            if (c + 1 < C) {
#pragma unroll
              for (int j = 0; j < 32; ++j)
                acc[j] += (int64_t)__float2ll_rn(__uint_as_float(r1[j])) *
                          (int64_t)(1ll << (4 * (c + 1)));
            }
          }
        } else {
#pragma unroll 1
          for (int c = 0; c < C; ++c) {
            uint32_t r[32];
            tmem_ld32(acc0 + c * BN + col0, r);
#pragma unroll
            for (int j = 0; j < 32; ++j)
              acc[j] += (int64_t)__float2ll_rn(__uint_as_float(r[j])) * (int64_t)(1ll << (4 * c));
          }
        }
        const uint64_t col = (uint64_t)tn * BN + col0;
        if (row < args.m) {
          int64_t* dst = args.c + row * args.n + col;
          int32_t* dst32 = reinterpret_cast<int32_t*>(args.c) + row * args.n + col;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (col + j < args.n) {
              if (args.c32)
                dst32[j] = (int32_t)acc[j];  // (statistics from the exact value below)
              else
                dst[j] = acc[j];
              orv |= fold(acc[j]);
              neg |= (uint32_t)(acc[j] < 0);
            }
          }
        }
      }
      // this set's tensor memory has been read: the MMAs of tile i + accs may start
      asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_u32(&acc_empty[a]))
                     : "memory");
    }
    orv = warp_or64(orv);
    neg = __reduce_or_sync(0xffffffffu, neg);
    if (lane == 0) {
      if (orv) atomicOr(reinterpret_cast<unsigned long long*>(&args.out->stat_or),
                        (unsigned long long)orv);
      if (neg) atomicOr(&args.out->stat_neg, 1u);
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
  __syncthreads();
  if (abort_s && threadIdx.x == 0) {
    // a wait gave up: let the copies already issued land (bounded) before the
    // CTA's shared memory is released, and report it
    const uint32_t issued = issued_s;
    for (uint32_t g = issued > (uint32_t)S ? issued - S : 0; g < issued; ++g)
      mbar_wait(&full_bar[g % S], (g / S) & 1);
    set_status(args.out, CCM_E_TIMEOUT);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "r"((uint32_t)G.tmem_cols));
  }
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
struct Plan {
  int L;
  uint64_t m_pad, n_pad, k_pad;
  size_t a_bytes, b_bytes;
};

Plan plan_for(uint64_t m, uint64_t k, uint64_t n, int L) {
  Geo g = geometry(L);
  Plan p;
  p.L = L;
  p.m_pad = round_up(m, kBM);
  p.n_pad = round_up(n, (uint64_t)g.bn);
  p.k_pad = round_up(k, kBK);
  p.a_bytes = (size_t)L * p.m_pad * p.k_pad;
  p.b_bytes = (size_t)L * p.n_pad * p.k_pad;
  return p;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map(CUtensorMap* map, void* base, uint64_t inner, uint64_t rows, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {inner};
  cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int digits_for(int bmax) { return (bmax + 3) / 4; }

}  // namespace tc

// The tensor path needs both widths bounded by 16 bits (at most 4 digits) and
// every class sum below 2^24.
bool matmul_c32(const ccm_matrix& c) { return width_bound(c.capacity, c.rows * c.cols) <= 31; }

bool matmul_tc_supported(const ccm_matrix& a, const ccm_matrix& b) {
  const uint64_t m = a.rows, k = a.cols, n = b.cols;
  if (!m || !n || !k) return false;
  const int ba = width_bound(a.capacity, m * k), bb = width_bound(b.capacity, k * n);
  const int L = tc::digits_for(ba > bb ? ba : bb);
  if (L < 1 || L > 4) return false;
  if ((double)k * L * 225.0 >= 16777216.0) return false;
  if (ba + bb + bitlen_host(k) > 62) return false;
  return tc::encode_fn() != nullptr;
}

size_t matmul_tc_workspace(const ccm_matrix& a, const ccm_matrix& b) {
  if (!matmul_tc_supported(a, b)) return 0;
  const uint64_t m = a.rows, k = a.cols, n = b.cols;
  const int ba = width_bound(a.capacity, m * k), bb = width_bound(b.capacity, k * n);
  tc::Plan p = tc::plan_for(m, k, n, tc::digits_for(ba > bb ? ba : bb));
  return tc::round_up(p.a_bytes, 256) + tc::round_up(p.b_bytes, 256);
}

size_t matmul_tc_workspace_upper(uint64_t m, uint64_t k, uint64_t n) {
  if (!m || !n || !k) return 0;
  tc::Plan p = tc::plan_for(m, k, n, 4);
  return tc::round_up(p.a_bytes, 256) + tc::round_up(p.b_bytes, 256);
}

template <int L>
static void launch_mm(const CUtensorMap& ta, const CUtensorMap& tb, const tc::MmArgs& args,
                      unsigned grid, cudaStream_t st) {
  constexpr tc::Geo g = tc::geometry(L);
  const size_t smem = (size_t)g.stages * L * tc::kBK * (tc::kBM + g.bn) + 1024;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(tc::k_mm_tc<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  tc::k_mm_tc<L><<<grid, tc::kThreadsP, smem, st>>>(ta, tb, args);
}

int run_matmul_tc(const ccm_matrix& a, const ccm_matrix& b, const ccm_matrix& c,
                  int64_t* c_scratch, void* ws, cudaStream_t st) {
  const uint64_t m = a.rows, k = a.cols, n = b.cols;
  const int ba = width_bound(a.capacity, m * k), bb = width_bound(b.capacity, k * n);
  const int L = tc::digits_for(ba > bb ? ba : bb);
  tc::Plan p = tc::plan_for(m, k, n, L);
  uint8_t* pa = (uint8_t*)ws;
  uint8_t* pb = pa + tc::round_up(p.a_bytes, 256);
  {
    const uint64_t quads = p.m_pad * p.k_pad / 4;
    int g = (int)umin((quads + 255) / 256, (uint64_t)num_sms() * 16);
    tc::k_limbs_a<<<g, 256, 0, st>>>(c.hdr, a.hdr, a.words, m, k, p.m_pad, p.k_pad, L, pa);
    const uint64_t tiles = (p.k_pad / 64) * (p.n_pad / 32);
    int g2 = (int)umin(tiles, (uint64_t)num_sms() * 16);
    tc::k_limbs_bt<<<g2, 256, 0, st>>>(c.hdr, b.hdr, b.words, k, n, p.n_pad, p.k_pad, L, pb);
    note_launch(2);
  }
  const tc::Geo g = tc::geometry(L);
  CUtensorMap ta, tb;
  if (!tc::make_map(&ta, pa, p.k_pad, (uint64_t)L * p.m_pad, tc::kBM) ||
      !tc::make_map(&tb, pb, p.k_pad, (uint64_t)L * p.n_pad, (uint32_t)g.bn))
    return CCM_E_CUDA;
  tc::MmArgs args{c.hdr, c_scratch, m, n, (uint32_t)(p.k_pad / tc::kBK), (uint32_t)p.m_pad,
                  (uint32_t)p.n_pad, (uint32_t)(p.n_pad / g.bn), (uint32_t)(p.m_pad / tc::kBM),
                  L, matmul_c32(c) ? 1 : 0};
  // persistent: one CTA per SM (the stages fill its shared memory), or one
  // per tile when there are fewer tiles
  const uint64_t tiles = (p.m_pad / tc::kBM) * (p.n_pad / g.bn);
  const unsigned grid = (unsigned)umin(tiles, (uint64_t)num_sms());
  profile_begin(st);
  switch (L) {
    case 1: launch_mm<1>(ta, tb, args, grid, st); break;
    case 2: launch_mm<2>(ta, tb, args, grid, st); break;
    case 3: launch_mm<3>(ta, tb, args, grid, st); break;
    default: launch_mm<4>(ta, tb, args, grid, st); break;
  }
  profile_end(st);
  note_launch();
  return CCM_OK;
}

}  // namespace ccm
