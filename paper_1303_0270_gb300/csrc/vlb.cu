// vlb.cu -- the paper's second encoding, Variable Length Blocks (Methods,
// "Method 2: Variable Length Blocks", Eq. 9-13): every entry is stored as a
// fixed k-bit prefix holding its bit length L, followed by the entry in
// exactly L bits, LSB-first in one bit stream (the same stream convention as
// SM).  k is the bit length of the largest L; the bit length of 0 is 1
// (Eq. 1).  Non-negative entries, as in the paper.
//
// A VLB stream has no random access: entry e starts after the lengths of all
// entries before it.  On the GPU the encoder is therefore a scan --
//   k_vlb_lens   per 1024-entry block: sum of L, global max of L
//   k_vlb_scan   one CTA: k, block bit offsets (exclusive scan), header
//   k_vlb_write  per block: in-block scan of k + L, bits assembled in shared
//                memory, interior words stored, the two boundary words OR-ed
// -- and it also writes an index: the bit offset of every 64th entry (plus
// the total), which lets the decoder k_vlb_unpack run one thread per 64
// entries.  The index is this library's addition (the paper has none).
#include "ccm_device.cuh"
#include "kernels.h"
#include "pack_engine.cuh"

namespace ccm {
namespace vlb {

constexpr int kBlock = 1024;   // entries per encoder block
constexpr int kThreads = 256;  // 4 entries per thread
constexpr int kStride = CCM_VLB_INDEX_STRIDE;
// shared words of one block: 1024 entries of at most 7 + 63 bits, plus slack
constexpr int kBlockWords = (kBlock * 70 + 31) / 32 + 4;

__device__ __forceinline__ int vlb_len(uint64_t v) { return v ? 64 - __clzll((long long)v) : 1; }

template <typename T>
__global__ void __launch_bounds__(kThreads) k_vlb_lens(const T* __restrict__ src, uint64_t n,
                                                       uint64_t* __restrict__ block_sum,
                                                       ccm_header* hdr) {
  __shared__ uint64_t s_sum[kThreads / 32];
  __shared__ int s_max[kThreads / 32];
  __shared__ int s_neg[kThreads / 32];
  const uint64_t nblocks = (n + kBlock - 1) / kBlock;
  for (uint64_t blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
    uint64_t sum = 0;
    int mx = 1, neg = 0;
    for (int j = 0; j < kBlock / kThreads; ++j) {
      const uint64_t e = blk * kBlock + threadIdx.x + j * kThreads;
      if (e < n) {
        const int64_t v = (int64_t)src[e];
        neg |= v < 0;
        const int L = vlb_len((uint64_t)v);
        sum += L;
        mx = max(mx, L);
      }
    }
    for (int d = 16; d; d >>= 1) {
      sum += __shfl_down_sync(0xffffffffu, sum, d);
      mx = max(mx, __shfl_down_sync(0xffffffffu, mx, d));
      neg |= __shfl_down_sync(0xffffffffu, neg, d);
    }
    if (threadIdx.x % 32 == 0) {
      s_sum[threadIdx.x / 32] = sum;
      s_max[threadIdx.x / 32] = mx;
      s_neg[threadIdx.x / 32] = neg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < kThreads / 32; ++w) {
        sum += s_sum[w];
        mx = max(mx, s_max[w]);
        neg |= s_neg[w];
      }
      block_sum[blk] = sum;
      atomicMax(reinterpret_cast<unsigned int*>(&hdr->reserved0), (unsigned int)mx);
      if (neg) set_status(hdr, CCM_E_RANGE);
    }
    __syncthreads();
  }
}

// One CTA: k from the largest bit length, bit offset of every block, header.
__global__ void __launch_bounds__(1024) k_vlb_scan(uint64_t* __restrict__ block_off,
                                                   uint64_t nblocks, uint64_t n, ccm_header* hdr,
                                                   uint64_t capacity, uint64_t* __restrict__ index,
                                                   uint64_t index_entries) {
  __shared__ uint64_t s_part[32];
  __shared__ uint64_t s_carry;
  if (hdr->status != CCM_OK) return;
  const int k = 32 - __clz((int)hdr->reserved0);  // bit length of the largest L
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (uint64_t base = 0; base < nblocks; base += blockDim.x) {
    const uint64_t b = base + threadIdx.x;
    uint64_t v = 0;
    if (b < nblocks) {
      const uint64_t cnt = umin((uint64_t)kBlock, n - b * kBlock);
      v = block_off[b] + (uint64_t)k * cnt;
    }
    // inclusive warp scan, then across warps
    uint64_t x = v;
    for (int d = 1; d < 32; d <<= 1) {
      const uint64_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (threadIdx.x % 32 >= d) x += y;
    }
    if (threadIdx.x % 32 == 31) s_part[threadIdx.x / 32] = x;
    __syncthreads();
    if (threadIdx.x < 32) {
      uint64_t p = threadIdx.x < blockDim.x / 32 ? s_part[threadIdx.x] : 0;
      for (int d = 1; d < 32; d <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, p, d);
        if (threadIdx.x >= d) p += y;
      }
      s_part[threadIdx.x] = p;
    }
    __syncthreads();
    const uint64_t warp_prefix = threadIdx.x >= 32 ? s_part[threadIdx.x / 32 - 1] : 0;
    const uint64_t carry = s_carry;
    if (b < nblocks) block_off[b] = carry + warp_prefix + x - v;  // exclusive
    __syncthreads();
    if (threadIdx.x == 0) s_carry = carry + s_part[blockDim.x / 32 - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const uint64_t total = s_carry;
    const uint64_t nw = ((total + 31) / 32 + 3) & ~3ull;
    hdr->width = k;
    hdr->is_signed = 0;
    hdr->nwords = nw;
    hdr->stat_or = total;
    hdr->magic = CCM_VLB_MAGIC;
    if (nw > capacity) hdr->status = CCM_E_CAPACITY;
    if (index) index[index_entries - 1] = total;
  }
}

__global__ void k_vlb_zero(const ccm_header* hdr, uint32_t* __restrict__ words, uint64_t capacity) {
  if (hdr->status != CCM_OK) return;
  const uint64_t nw = umin(hdr->nwords, capacity);
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nw;
       i += (uint64_t)gridDim.x * blockDim.x)
    words[i] = 0;
}

template <typename T>
__global__ void __launch_bounds__(kThreads) k_vlb_write(const T* __restrict__ src, uint64_t n,
                                                        const uint64_t* __restrict__ block_off,
                                                        const ccm_header* hdr,
                                                        uint32_t* __restrict__ words,
                                                        uint64_t* __restrict__ index) {
  __shared__ uint32_t s_words[kBlockWords];
  __shared__ uint32_t s_part[kThreads / 32];
  if (hdr->status != CCM_OK) return;
  const int k = hdr->width;
  const uint64_t nblocks = (n + kBlock - 1) / kBlock;
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  for (uint64_t blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
    const uint64_t bo = block_off[blk];
    const uint64_t w0 = bo / 32;
    const int shift0 = (int)(bo % 32);
    // this thread's 4 consecutive entries
    const uint64_t e0 = blk * kBlock + 4 * (uint64_t)threadIdx.x;
    uint64_t v[4];
    int bits[4];
    uint32_t mine = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const bool live = e0 + j < n;
      v[j] = live ? (uint64_t)(int64_t)src[e0 + j] : 0;
      bits[j] = live ? k + vlb_len(v[j]) : 0;
      mine += bits[j];
    }
    // block exclusive scan of the per-thread bit counts
    uint32_t x = mine;
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= d) x += y;
    }
    if (lane == 31) s_part[warp] = x;
    for (uint32_t i = threadIdx.x; i < kBlockWords; i += kThreads) s_words[i] = 0;
    __syncthreads();
    uint32_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_part[w];
    uint32_t off = before + x - mine;  // bit offset of entry e0 within the block
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (bits[j]) {
        const uint64_t e = e0 + j;
        if (index && e % kStride == 0) index[e / kStride] = bo + off;
        const int L = bits[j] - k;
        // prefix (k bits) then the value (L bits): up to 70 bits
        const uint64_t lo = (uint64_t)L | (k < 64 ? (v[j] << k) : 0);
        const uint64_t hi = k ? (v[j] >> (64 - k)) : 0;
        const uint32_t p = (uint32_t)shift0 + off;
        const uint32_t wi = p / 32, s = p % 32;
        // 70 bits starting at bit s of word wi: up to four words
        atomicOr(&s_words[wi], (uint32_t)(lo << s));
        const uint64_t t1 = s ? (lo >> (32 - s)) | (hi << (32 + s)) : (lo >> 32);
        const int need = (int)((s + bits[j] + 31) / 32);
        if (need > 1) atomicOr(&s_words[wi + 1], (uint32_t)t1);
        if (need > 2) {
          const uint64_t t2 = s ? (lo >> (64 - s)) | (hi << s) : hi;
          atomicOr(&s_words[wi + 2], (uint32_t)t2);
        }
        if (need > 3) atomicOr(&s_words[wi + 3], (uint32_t)(hi >> (32 - s)));
        off += bits[j];
      }
    }
    __syncthreads();
    uint32_t block_bits = 0;
    for (int w = 0; w < kThreads / 32; ++w) block_bits += s_part[w];
    const uint32_t nwords_blk = (uint32_t)((shift0 + block_bits + 31) / 32);
    for (uint32_t i = threadIdx.x; i < nwords_blk; i += kThreads) {
      const uint32_t val = s_words[i];
      if (i == 0 || i == nwords_blk - 1)
        atomicOr(&words[w0 + i], val);  // shared with the neighbouring blocks
      else
        words[w0 + i] = val;
    }
    __syncthreads();
  }
}

// Reads `len` (<= 64) bits at bit position `pos` of the stream.
__device__ __forceinline__ uint64_t read_bits(const uint32_t* __restrict__ w, uint64_t pos,
                                              int len) {
  const uint64_t wi = pos / 32;
  const int s = (int)(pos % 32);
  uint64_t r = (uint64_t)__ldg(w + wi) >> s;
  int have = 32 - s;
  if (have < len) {
    r |= (uint64_t)__ldg(w + wi + 1) << have;
    have += 32;
    if (have < len) r |= (uint64_t)__ldg(w + wi + 2) << have;
  }
  return len >= 64 ? r : (r & ((1ull << len) - 1ull));
}

// A valid VLB header for the expected shape and buffer.
__device__ __forceinline__ int check_vlb(const ccm_header* hdr, uint64_t rows, uint64_t cols,
                                         uint64_t capacity) {
  if (hdr->magic != CCM_VLB_MAGIC) return CCM_E_INPUT;
  if (hdr->status != CCM_OK) return hdr->status;
  if (hdr->rows != rows || hdr->cols != cols) return CCM_E_INPUT;
  if (hdr->width < 1 || hdr->width > 7 || hdr->nwords > capacity) return CCM_E_INPUT;
  if (hdr->stat_or > hdr->nwords * 32ull) return CCM_E_INPUT;
  return CCM_OK;
}

template <typename T>
__global__ void __launch_bounds__(256) k_vlb_unpack(const ccm_header* hdr,
                                                    const uint32_t* __restrict__ words,
                                                    const uint64_t* __restrict__ index,
                                                    uint64_t rows, uint64_t cols, uint64_t capacity,
                                                    T* __restrict__ out, int32_t* err) {
  const uint64_t n = rows * cols;
  int st = check_vlb(hdr, rows, cols, capacity);
  if (st == CCM_OK && sizeof(T) == 4 && (int)hdr->reserved0 > 31) st = CCM_E_WIDTH;
  if (err && blockIdx.x == 0 && threadIdx.x == 0) *err = st;
  if (st != CCM_OK) return;
  const int k = hdr->width;
  const uint64_t chunks = (n + kStride - 1) / kStride;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks;
       c += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t pos = index[c];
    const uint64_t limit = hdr->stat_or;  // total bits: never read past the stream
    const uint64_t e_end = umin(n, (c + 1) * kStride);
    for (uint64_t e = c * kStride; e < e_end; ++e) {
      if (pos + k > limit) break;
      const int L = (int)read_bits(words, pos, k);
      if (L < 1 || pos + k + L > limit) break;
      const uint64_t v = read_bits(words, pos + k, L);
      out[e] = (T)v;
      pos += k + L;
    }
  }
}

}  // namespace vlb

size_t vlb_workspace(uint64_t n) {
  const uint64_t nblocks = (n + vlb::kBlock - 1) / vlb::kBlock;
  return ((nblocks * 8 + 255) & ~(size_t)255) + 256;
}

// words == nullptr: measure only (k, total bits and word count in the header).
void run_vlb_pack(const void* dense, int dtype, uint64_t rows, uint64_t cols, ccm_header* hdr,
                  uint32_t* words, uint64_t capacity, uint64_t* index, void* ws, cudaStream_t st) {
  const uint64_t n = rows * cols;
  const uint64_t nblocks = (n + vlb::kBlock - 1) / vlb::kBlock;
  uint64_t* block = (uint64_t*)ws;
  InitArgs ia{};
  ia.out = hdr;
  ia.out_rows = rows;
  ia.out_cols = cols;
  launch_init(ia, st);  // also clears reserved0 (the largest bit length)
  const int g = (int)umin(umax(nblocks, 1), (uint64_t)num_sms() * 8);
  if (dtype == CCM_I64)
    vlb::k_vlb_lens<int64_t><<<g, vlb::kThreads, 0, st>>>((const int64_t*)dense, n, block, hdr);
  else
    vlb::k_vlb_lens<int32_t><<<g, vlb::kThreads, 0, st>>>((const int32_t*)dense, n, block, hdr);
  const uint64_t entries = (n + vlb::kStride - 1) / vlb::kStride + 1;
  vlb::k_vlb_scan<<<1, 1024, 0, st>>>(block, nblocks, n, hdr, words ? capacity : ~0ull,
                                      index, entries);
  note_launch(2);
  if (!words) return;
  vlb::k_vlb_zero<<<(int)umin((capacity + 255) / 256 + 1, (uint64_t)num_sms() * 8), 256, 0, st>>>(
      hdr, words, capacity);
  profile_begin(st);
  if (dtype == CCM_I64)
    vlb::k_vlb_write<int64_t><<<g, vlb::kThreads, 0, st>>>((const int64_t*)dense, n, block, hdr,
                                                           words, index);
  else
    vlb::k_vlb_write<int32_t><<<g, vlb::kThreads, 0, st>>>((const int32_t*)dense, n, block, hdr,
                                                           words, index);
  profile_end(st);
  note_launch(2);
}

void run_vlb_unpack(const ccm_header* hdr, const uint32_t* words, uint64_t capacity,
                    const uint64_t* index, uint64_t rows, uint64_t cols, void* dense, int dtype,
                    int32_t* err, cudaStream_t st) {
  const uint64_t n = rows * cols;
  const uint64_t chunks = (n + vlb::kStride - 1) / vlb::kStride;
  const int g = (int)umin(umax((chunks + 255) / 256, 1), (uint64_t)num_sms() * 8);
  profile_begin(st);
  if (dtype == CCM_I64)
    vlb::k_vlb_unpack<int64_t><<<g, 256, 0, st>>>(hdr, words, index, rows, cols, capacity,
                                                   (int64_t*)dense, err);
  else
    vlb::k_vlb_unpack<int32_t><<<g, 256, 0, st>>>(hdr, words, index, rows, cols, capacity,
                                                   (int32_t*)dense, err);
  profile_end(st);
  note_launch();
}

}  // namespace ccm
