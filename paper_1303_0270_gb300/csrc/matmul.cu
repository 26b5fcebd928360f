// matmul.cu -- C = A B on the compressed form, CUDA-core path: tiles of A
// and B are decoded from their words into shared memory and multiplied with
// integer multiply-adds.  c_ij = sum_l a_il b_lj exactly (int64 when the
// operand widths bound every partial sum below 2^63, 128-bit otherwise), into
// an int64 scratch matrix that the pack engine re-packs at C's own width.
#include <type_traits>

#include "pack_engine.cuh"
#include "kernels.h"
#include "matmul_tc.h"

namespace ccm {

namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;
constexpr int kMmThreads = 256;  // 16 x 16 threads, 4 x 4 outputs each

__device__ __forceinline__ bool fits64(__int128 v) {
  return v >= -((__int128)1 << 63) && v < ((__int128)1 << 63);
}

template <bool kWide>
__device__ __forceinline__ void mm_tile(ccm_header* out, const uint32_t* __restrict__ wa, int ba,
                                        int sa, const uint32_t* __restrict__ wb, int bb, int sb,
                                        uint64_t m, uint64_t k, uint64_t n, int64_t* __restrict__ c,
                                        uint64_t tm, uint64_t tn, int64_t (*sA)[kBM + 1],
                                        int64_t (*sB)[kBN + 1]) {
  using Acc = typename std::conditional<kWide, __int128, int64_t>::type;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  Acc acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = 0;
  for (uint64_t k0 = 0; k0 < k; k0 += kBK) {
    // decode A[tm .. tm+64) x [k0 .. k0+16) transposed into sA[kk][r]
    for (int e = threadIdx.x; e < kBM * kBK; e += kMmThreads) {
      int r = e / kBK, kk = e % kBK;
      uint64_t gi = tm + r, gk = k0 + kk;
      sA[kk][r] = (gi < m && gk < k) ? decode_field(wa, gi * k + gk, ba, sa) : 0;
    }
    for (int e = threadIdx.x; e < kBK * kBN; e += kMmThreads) {
      int kk = e / kBN, q = e % kBN;
      uint64_t gk = k0 + kk, gj = tn + q;
      sB[kk][q] = (gk < k && gj < n) ? decode_field(wb, gk * n + gj, bb, sb) : 0;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kBK; ++kk) {
      int64_t av[4], bv[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) av[r] = sA[kk][ty + 16 * r];
#pragma unroll
      for (int q = 0; q < 4; ++q) bv[q] = sB[kk][tx + 16 * q];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[r][q] += (Acc)av[r] * (Acc)bv[q];
    }
    __syncthreads();
  }
  int ovf = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint64_t gi = tm + ty + 16 * r, gj = tn + tx + 16 * q;
      if (gi < m && gj < n) {
        if (kWide && !fits64((__int128)acc[r][q])) ovf = 1;
        c[gi * n + gj] = (int64_t)acc[r][q];
      }
    }
  if (ovf) set_status(out, CCM_E_OVERFLOW);
}

__global__ void __launch_bounds__(kMmThreads) k_matmul_cc(ccm_header* out, const ccm_header* ha,
                                                          const uint32_t* __restrict__ wa,
                                                          const ccm_header* hb,
                                                          const uint32_t* __restrict__ wb,
                                                          uint64_t m, uint64_t k, uint64_t n,
                                                          int64_t* __restrict__ c) {
  __shared__ int64_t sA[kBK][kBM + 1];
  __shared__ int64_t sB[kBK][kBN + 1];
  if (out->status != CCM_OK) return;
  const int ba = ha->width, sa = ha->is_signed, bb = hb->width, sb = hb->is_signed;
  const bool wide = ba + bb + bitlen64(k) > 63;
  const uint64_t tiles_n = (n + kBN - 1) / kBN;
  const uint64_t tiles = ((m + kBM - 1) / kBM) * tiles_n;
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    uint64_t tm = (t / tiles_n) * kBM, tn = (t % tiles_n) * kBN;
    if (wide)
      mm_tile<true>(out, wa, ba, sa, wb, bb, sb, m, k, n, c, tm, tn, sA, sB);
    else
      mm_tile<false>(out, wa, ba, sa, wb, bb, sb, m, k, n, c, tm, tn, sA, sB);
  }
}

// CUDA-core path for fields of at most 31 bits (bounded by the capacities):
// 128 x 128 output tiles, 256 threads with 8 x 8 outputs each; A and B tiles
// decoded to int32 in shared memory; every product a 32 x 32 -> 64-bit
// multiply-add.  The host selects it only when b_a + b_b + bitlen(k) <= 63,
// so every partial sum fits the int64 accumulators.
constexpr int kCB = 128, kCK = 16;
__global__ void __launch_bounds__(256) k_matmul_cc32(ccm_header* out, const ccm_header* ha,
                                                     const uint32_t* __restrict__ wa,
                                                     const ccm_header* hb,
                                                     const uint32_t* __restrict__ wb,
                                                     uint64_t m, uint64_t k, uint64_t n,
                                                     int64_t* __restrict__ c) {
  __shared__ __align__(16) int sA[kCK][kCB + 4];
  __shared__ __align__(16) int sB[kCK][kCB + 4];
  __shared__ int s_skip;
  if (threadIdx.x == 0) s_skip = out->status != CCM_OK;
  __syncthreads();
  if (s_skip) return;
  const int ba = ha->width, sa = ha->is_signed, bb = hb->width, sb = hb->is_signed;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const uint64_t tiles_n = (n + kCB - 1) / kCB;
  const uint64_t tiles = ((m + kCB - 1) / kCB) * tiles_n;
  for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    const uint64_t tm = (t / tiles_n) * kCB, tn = (t % tiles_n) * kCB;
    long long acc[8][8];
#pragma unroll
    for (int r = 0; r < 8; ++r)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[r][q] = 0;
    for (uint64_t k0 = 0; k0 < k; k0 += kCK) {
      for (int e = threadIdx.x; e < kCB * kCK; e += 256) {
        const int r = e / kCK, kk = e % kCK;
        const uint64_t gi = tm + r, gk = k0 + kk;
        sA[kk][r] = (gi < m && gk < k) ? (int)decode_field(wa, gi * k + gk, ba, sa) : 0;
        const int kk2 = e / kCB, q = e % kCB;
        const uint64_t gk2 = k0 + kk2, gj = tn + q;
        sB[kk2][q] = (gk2 < k && gj < n) ? (int)decode_field(wb, gk2 * n + gj, bb, sb) : 0;
      }
      __syncthreads();
#pragma unroll 4
      for (int kk = 0; kk < kCK; ++kk) {
        const int4 a0 = *reinterpret_cast<const int4*>(&sA[kk][ty * 4]);
        const int4 a1 = *reinterpret_cast<const int4*>(&sA[kk][64 + ty * 4]);
        const int4 b0 = *reinterpret_cast<const int4*>(&sB[kk][tx * 4]);
        const int4 b1 = *reinterpret_cast<const int4*>(&sB[kk][64 + tx * 4]);
        const int av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const int bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[r][q] += (long long)av[r] * bv[q];
      }
      __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const uint64_t gi = tm + (r < 4 ? ty * 4 + r : 64 + ty * 4 + r - 4);
      if (gi >= m) continue;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const uint64_t gj = tn + (q < 4 ? tx * 4 + q : 64 + tx * 4 + q - 4);
        if (gj < n) c[gi * n + gj] = acc[r][q];
      }
    }
  }
}

}  // namespace

size_t matmul_workspace(const ccm_matrix& a, const ccm_matrix& b) {
  const uint64_t m = a.rows, n = b.cols;
  size_t c_bytes = ((m * n * sizeof(int64_t)) + 255) & ~(size_t)255;
  return c_bytes + matmul_tc_workspace(a, b) + 256;
}

size_t matmul_workspace_upper(uint64_t m, uint64_t k, uint64_t n) {
  size_t c_bytes = ((m * n * sizeof(int64_t)) + 255) & ~(size_t)255;
  return c_bytes + matmul_tc_workspace_upper(m, k, n) + 256;
}

int run_matmul(const ccm_matrix& a, const ccm_matrix& b, const ccm_matrix& c, int path, void* ws,
               cudaStream_t st) {
  const uint64_t m = a.rows, k = a.cols, n = b.cols;
  const bool tc_ok = matmul_tc_supported(a, b);
  if (path == CCM_MATMUL_TENSOR && !tc_ok) return CCM_E_SHAPE;
  const bool tc = tc_ok && (path == CCM_MATMUL_TENSOR || path == CCM_MATMUL_AUTO);
  int64_t* cs = (int64_t*)ws;
  InitArgs ia{};
  ia.out = c.hdr;
  ia.in0 = a.hdr;
  ia.in0_rows = a.rows;
  ia.in0_cols = a.cols;
  ia.in0_capacity = a.capacity;
  ia.in1 = b.hdr;
  ia.in1_rows = b.rows;
  ia.in1_cols = b.cols;
  ia.in1_capacity = b.capacity;
  ia.out_rows = c.rows;
  ia.out_cols = c.cols;
  if (k == 0) {
    ia.zero_ptr = cs;
    ia.zero_count = m * n;
  }
  launch_init(ia, st);
  if (m && n && k) {
    if (tc) {
      size_t c_bytes = ((m * n * sizeof(int64_t)) + 255) & ~(size_t)255;
      int rc = run_matmul_tc(a, b, c, cs, (char*)ws + c_bytes, st);
      if (rc != CCM_OK) return rc;
      if (matmul_c32(c))
        run_pack_scratch32(reinterpret_cast<const int32_t*>(cs), c, st);
      else
        run_pack_scratch(cs, c, st, /*stats_done=*/true);
      return CCM_OK;
    } else {
      const int ba = width_bound(a.capacity, m * k), bb = width_bound(b.capacity, k * n);
      profile_begin(st);
      if (ba <= 31 && bb <= 31 && ba + bb + bitlen_host(k) <= 63) {
        uint64_t tiles = ((m + kCB - 1) / kCB) * ((n + kCB - 1) / kCB);
        int g = (int)umin(tiles, (uint64_t)num_sms() * 2);
        k_matmul_cc32<<<g, 256, 0, st>>>(c.hdr, a.hdr, a.words, b.hdr, b.words, m, k, n, cs);
      } else {
        uint64_t tiles = ((m + kBM - 1) / kBM) * ((n + kBN - 1) / kBN);
        int g = (int)umin(tiles, (uint64_t)num_sms() * 4);
        k_matmul_cc<<<g, kMmThreads, 0, st>>>(c.hdr, a.hdr, a.words, b.hdr, b.words, m, k, n, cs);
      }
      profile_end(st);
      note_launch();
    }
  }
  run_pack_scratch(cs, c, st);
  return CCM_OK;
}

}  // namespace ccm
