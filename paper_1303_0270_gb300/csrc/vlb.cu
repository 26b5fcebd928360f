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
// entries (a warp's 32 x 64 values staged in shared memory and stored
// coalesced).  The index is this library's addition (the paper has none).
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

// Sequential reader of the stream from a bit position: a 64-bit buffer
// refilled one 32-bit word at a time (one load per 32 bits consumed).
struct BitReader {
  const uint32_t* __restrict__ w;
  uint64_t buf;
  uint64_t next;  // index of the next word to load
  int have;       // valid bits in buf
  __device__ __forceinline__ BitReader(const uint32_t* words, uint64_t pos) : w(words) {
    const uint64_t wi = pos / 32;
    const int s = (int)(pos % 32);
    buf = (uint64_t)__ldg(w + wi) >> s;
    have = 32 - s;
    next = wi + 1;
  }
  // the next len (<= 32) bits
  __device__ __forceinline__ uint32_t take(int len) {
    if (have < len) {
      buf |= (uint64_t)__ldg(w + next++) << have;
      have += 32;
    }
    const uint32_t v = (uint32_t)(buf & ((1ull << len) - 1ull));
    buf >>= len;
    have -= len;
    return v;
  }
  // the next len (1..64) bits
  __device__ __forceinline__ uint64_t take64(int len) {
    if (len <= 32) return take(len);
    const uint64_t lo = take(32);
    return lo | ((uint64_t)take(len - 32) << 32);
  }
};

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

// Decode: thread c walks the 64 entries of index chunk c from their indexed
// bit offset (prefix, then value).  The 32 lanes of a warp hold 32
// consecutive chunks; each lane decodes its chunk in two halves of 32
// entries, staged in shared memory (33 slots per lane) and then stored by the
// warp one chunk-half at a time with consecutive lanes on consecutive entries
// (coalesced 128- or 256-byte runs), only the entries a lane decoded.
constexpr int kUnpackWarps = 8;
constexpr int kHalf = kStride / 2;

template <typename T>
__global__ void __launch_bounds__(kUnpackWarps * 32) k_vlb_unpack(
    const ccm_header* hdr, const uint32_t* __restrict__ words, const uint64_t* __restrict__ index,
    uint64_t rows, uint64_t cols, uint64_t capacity, T* __restrict__ out, int32_t* err) {
  extern __shared__ __align__(16) uint8_t s_raw[];
  T* stage = reinterpret_cast<T*>(s_raw) + (threadIdx.x / 32) * 32 * (kHalf + 1);
  const uint64_t n = rows * cols;
  int st = check_vlb(hdr, rows, cols, capacity);
  if (st == CCM_OK && sizeof(T) == 4 && (int)hdr->reserved0 > 31) st = CCM_E_WIDTH;
  if (st != CCM_OK) {
    if (err && blockIdx.x == 0 && threadIdx.x == 0) *err = st;  // (*err holds CCM_OK before)
    return;
  }
  const int k = hdr->width;
  const uint64_t limit = hdr->stat_or;  // total bits: never read past the stream
  const uint64_t chunks = (n + kStride - 1) / kStride;
  const int lane = threadIdx.x % 32;
  const uint64_t nwarps = (uint64_t)gridDim.x * kUnpackWarps;
  T* mine = stage + lane * (kHalf + 1);
  uint64_t wc = (uint64_t)blockIdx.x * kUnpackWarps + threadIdx.x / 32;
  // the bit offsets of the chunks of this warp's next group, loaded one group
  // ahead (its decode hides their latency)
  uint64_t npos = wc * 32 + lane < chunks ? __ldg(index + wc * 32 + lane) : 0;
  for (; wc * 32 < chunks; wc += nwarps) {
    const uint64_t c = wc * 32 + lane;
    const int e_cnt = c < chunks ? (int)umin(kStride, n - c * kStride) : 0;
    uint64_t pos = npos;
    const uint64_t wn = wc + nwarps;
    npos = wn * 32 + lane < chunks ? __ldg(index + wn * 32 + lane) : 0;
    BitReader br(words, pos);
    bool ok = true;
    const uint64_t e0 = wc * 32 * kStride;
    for (int h = 0; h < 2; ++h) {
      if (h == 1 && wn * 32 < chunks) {
        // the stream lines of the next group into L1 (its chunks are
        // contiguous: from its first chunk's offset to past its last one's)
        const uint64_t b0 = __shfl_sync(0xffffffffu, npos, 0);
        const uint64_t cl = umin(chunks - wn * 32, 32) - 1;  // its last chunk (lane)
        const uint64_t bl = __shfl_sync(0xffffffffu, npos, (int)cl);
        const uint64_t l0 = b0 / 1024, l1 = umin((bl + (uint64_t)kStride * (k + 64)) / 1024,
                                                 (limit + 1023) / 1024);
        for (uint64_t ln = l0 + lane; ln < l1; ln += 32)
          asm volatile("prefetch.global.L1 [%0];\n" ::"l"(words + ln * 32));
      }
      int cnt = 0;  // entries of this half the lane decoded
      for (; ok && cnt < kHalf && h * kHalf + cnt < e_cnt; ++cnt) {
        if (pos + k > limit) {
          ok = false;
          break;
        }
        const int L = (int)br.take(k);
        if (L < 1 || L > 64 || pos + k + L > limit) {
          ok = false;
          break;
        }
        mine[cnt] = (T)br.take64(L);
        pos += k + L;
      }
      __syncwarp();
      // chunk-half by chunk-half: lane j stores entry j of the owner's half
#pragma unroll 4
      for (int owner = 0; owner < 32; ++owner) {
        const int oc = __shfl_sync(0xffffffffu, cnt, owner);
        const uint64_t e = e0 + (uint64_t)owner * kStride + h * kHalf + lane;
        if (lane < oc) out[e] = stage[owner * (kHalf + 1) + lane];
      }
      __syncwarp();
    }
    // a chunk parses to the next index entry, or the stream is damaged
    if (c < chunks && (!ok || pos != __ldg(index + c + 1)) && err)
      atomicCAS(err, CCM_OK, CCM_E_INPUT);
  }
}

// y = A x with A in VLB form: one warp per row; lane l takes the 64-entry
// index blocks l, l + 32, ... that overlap the row, decodes them from the
// block's indexed bit offset (skipping the entries before the row start) and
// accumulates a_ij * x_j in 128 bits; the warp's sum is checked against the
// int64 range and stored in the int64 y scratch.  x is read straight from
// its packed form.
__device__ __forceinline__ __int128 shfl_xor_i128(__int128 v, int d) {
  uint64_t lo = (uint64_t)v, hi = (uint64_t)((unsigned __int128)v >> 64);
  lo = __shfl_xor_sync(0xffffffffu, lo, d);
  hi = __shfl_xor_sync(0xffffffffu, hi, d);
  return (__int128)(((unsigned __int128)hi << 64) | lo);
}

__global__ void __launch_bounds__(256) k_vlb_matvec(const ccm_header* hdr,
                                                    const uint32_t* __restrict__ words,
                                                    const uint64_t* __restrict__ index,
                                                    uint64_t rows, uint64_t cols,
                                                    uint64_t capacity, ccm_header* out,
                                                    const ccm_header* hx,
                                                    const uint32_t* __restrict__ wx,
                                                    int64_t* __restrict__ y,
                                                    const unsigned long long* done) {
  if (out->status != CCM_OK || (done && *done)) return;
  const int st = check_vlb(hdr, rows, cols, capacity);
  if (st != CCM_OK) {
    if (blockIdx.x == 0 && threadIdx.x == 0) set_status(out, st);
    return;
  }
  const int k = hdr->width;
  const int bx = hx->width, sx = hx->is_signed;
  const uint64_t limit = hdr->stat_or;  // total bits: never read past the stream
  // every partial sum inside int64 when (largest L) + b_x + bitlen(cols) <= 63
  const bool narrow = (int)hdr->reserved0 + bx + bitlen64(cols) <= 63;
  const int lane = threadIdx.x % 32;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
  int bad = 0, ovf = 0;
  for (uint64_t i = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32; i < rows;
       i += warps) {
    const uint64_t rs = i * cols, re = rs + cols;
    __int128 acc = 0;
    for (uint64_t c = rs / kStride + lane; c * kStride < re; c += 32) {
      uint64_t pos = index[c];
      const uint64_t e_end = umin(re, (c + 1) * kStride);
      BitReader br(words, pos);
      long long acc64 = 0;
      for (uint64_t e = c * kStride; e < e_end; ++e) {
        if (pos + k > limit) { bad = 1; break; }
        const int L = (int)br.take(k);
        if (L < 1 || L > 64 || pos + k + L > limit) { bad = 1; break; }
        const uint64_t v = br.take64(L);
        if (e >= rs) {
          const int64_t xj = decode_field(wx, e - rs, bx, sx);
          if (narrow)
            acc64 += (long long)v * xj;
          else
            acc += (__int128)(int64_t)v * (__int128)xj;
        }
        pos += k + L;
      }
      acc += acc64;
    }
    for (int d = 16; d; d >>= 1) acc += shfl_xor_i128(acc, d);
    if (lane == 0) {
      if (acc < -((__int128)1 << 63) || acc >= ((__int128)1 << 63)) ovf = 1;
      y[i] = (int64_t)acc;
    }
  }
  if (bad) set_status(out, CCM_E_INPUT);
  if (ovf) set_status(out, CCM_E_OVERFLOW);
}

// ---------------------------------------------------------------------------
// Decoder and matvec, fast path.  A warp takes 32 consecutive index chunks
// (2048 entries), one per lane.  Each lane walks its chunk in steps: the 64
// stream bits from its position (two funnel shifts over the current and the
// next 8-byte block, held in registers), then E entries cut from them with
// shifts and a bit mask -- E = 8, 4 or 2 when E (k + largest L) <= 64 bits,
// one entry of up to 64 bits otherwise, and the prefix and the value from two
// windows when k + largest L > 64.  The blocks come through a small per-lane
// ring in shared memory that cp.async keeps several steps ahead.  Lane 0 asks
// L2 for the next group's stream bytes with one bulk prefetch.  Every lane
// checks its chunk: each L in [1, largest L], and the bits it used equal to
// the distance to the next index entry.

constexpr int kRound = 8;  // entries per lane between two staged stores

__device__ __forceinline__ uint32_t bmsk32(uint32_t width) {
  uint32_t m;
  asm("bmsk.clamp.b32 %0, 0, %1;" : "=r"(m) : "r"(width));
  return m;
}

// The reader's stream comes in 16-byte blocks through a per-lane ring of
// kSlots in shared memory (lane-interleaved: slot j of lane l at j * 32 + l),
// filled by 16-byte cp.async copies (L2 to shared memory) that the whole warp
// commits once per step.  Taking block b reads its slot and copies block
// b + kSlots - 1 into the slot of block b - 1 (read, and its value used, one
// take earlier), so each block is copied kSlots - 1 takes before it is read.
// A step consumes at most 71 bits, so it takes at most one block, and the
// chunk's first step starts after at most two takes: a block is read at
// least kSlots - 3 steps after the step (or the start) that copied it, and a
// wait for all but the last kWait = kSlots - 3 groups at the start of a step
// covers every block the step reads.  Copies stop one block past the chunk.
constexpr uint32_t kSlots = 5;
constexpr int kWait = kSlots - 3;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, uint32_t bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(smem)),
               "l"(gmem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// A lane's position in its chunk: the current and the next 8 bytes of the
// stream in registers (plus the upper half of the last 16-byte block taken,
// while unused) and the bit position p (< 64) in the current 8 bytes, so that
// the 64 bits from p are two funnel shifts away.
struct LaneReader {
  uint4* ring;        // this lane's slot 0; slot j at ring[j * 32]
  const uint4* src;   // the 16-byte block holding the chunk's first bit
  uint32_t cap;       // blocks worth copying from src (zeros past them)
  uint32_t rd, slot;  // next block to take (relative to src) and its slot
  uint32_t c0, c1, n0, n1, h0, h1;  // current, next, held (low word first)
  uint32_t p;
  bool held;

  __device__ __forceinline__ void copy(uint32_t b, uint32_t sl) {
    const uint32_t bytes = b < cap ? 16u : 0u;
    cp_async16(ring + sl * 32, src + (bytes ? b : 0u), bytes);
  }
  __device__ __forceinline__ uint4 take() {
    const uint4 v = ring[slot * 32];
    copy(rd + kSlots - 1, slot == 0 ? kSlots - 1 : slot - 1);
    ++rd;
    slot = slot == kSlots - 1 ? 0 : slot + 1;
    return v;
  }
  // Chunk bits [pos, end) of `words` (16-byte aligned, nwords a multiple of
  // 4); `ring_lane`: the lane's slot 0.  Waits for the previous chunk's copies
  // and for the first kSlots - 1 blocks.
  __device__ __forceinline__ void init(const uint32_t* words, uint64_t nwords, uint64_t pos,
                                       uint64_t end, uint4* ring_lane) {
    ring = ring_lane;
    const uint64_t nall = nwords / 4, q = pos >> 7;
    src = reinterpret_cast<const uint4*>(words) + (q < nall ? q : 0);
    const uint64_t last = end > pos ? ((end - 1) >> 7) + 2 : q + 1;  // one block past the chunk
    cap = q < nall ? (uint32_t)umin(umin(last, nall) - q, 1u << 20) : 0u;
    cp_async_wait<0>();
#pragma unroll
    for (uint32_t b = 0; b < kSlots - 1; ++b) copy(b, b);
    cp_async_commit();
    cp_async_wait<0>();
    rd = 0;
    slot = 0;
    const uint4 a = take();
    if (pos & 64) {
      c0 = a.z, c1 = a.w;
      const uint4 b = take();
      n0 = b.x, n1 = b.y, h0 = b.z, h1 = b.w;
      held = true;
    } else {
      c0 = a.x, c1 = a.y, n0 = a.z, n1 = a.w;
      held = false;
    }
    p = (uint32_t)(pos & 63);
    cp_async_commit();
  }
  // the 64 bits from p
  __device__ __forceinline__ uint64_t window() const {
    const bool h = p >= 32;
    const uint32_t a = h ? c1 : c0, b = h ? n0 : c1, c = h ? n1 : n0;
    return ((uint64_t)__funnelshift_r(b, c, p) << 32) | __funnelshift_r(a, b, p);
  }
  // t <= 64
  __device__ __forceinline__ void advance(uint32_t t) {
    p += t;
    if (p >= 64) {
      c0 = n0, c1 = n1;
      if (held) {
        n0 = h0, n1 = h1;
      } else {
        const uint4 v = take();
        n0 = v.x, n1 = v.y, h0 = v.z, h1 = v.w;
      }
      held = !held;
      p -= 64;
    }
  }
};

// x >> s for any s (PTX clamps shifts past 64: zero), so that the shift
// stays defined on a damaged stream.
__device__ __forceinline__ uint64_t shr64(uint64_t x, uint32_t s) {
  uint64_t r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
  return r;
}

// The low l bits of x (1 <= l <= 64).
__device__ __forceinline__ uint64_t low_bits(uint64_t x, uint32_t l) {
  return x & ((2ull << (l - 1u)) - 1ull);
}

template <int E>
__device__ __forceinline__ void take_short(LaneReader& r, uint32_t k, uint32_t km, uint32_t* v,
                                           uint32_t& umax, uint32_t& used) {
  cp_async_wait<kWait>();
  const uint64_t x = r.window();
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < E; ++i) {
    const uint32_t xi = (uint32_t)shr64(x, s);
    const uint32_t L = xi & km;
    v[i] = (xi >> k) & bmsk32(L);
    umax = max(umax, L - 1u);
    s += k + L;
  }
  s = min(s, 64u);  // (a valid chunk never reaches the clamp)
  r.advance(s);
  used += s;
  cp_async_commit();
}

// One entry of k + L <= 64 bits from one window.
__device__ __forceinline__ uint64_t take_medium(LaneReader& r, uint32_t k, uint32_t km,
                                                uint32_t& umax, uint32_t& used) {
  cp_async_wait<kWait>();
  const uint64_t x = r.window();
  const uint32_t L = (uint32_t)x & km;
  umax = max(umax, L - 1u);
  const uint64_t v = low_bits(x >> k, min(max(L, 1u), 64u));
  const uint32_t t = min(k + L, 64u);
  r.advance(t);
  used += t;
  cp_async_commit();
  return v;
}

// One entry of up to k + 64 bits: the prefix, then the value from a second
// window.
__device__ __forceinline__ uint64_t take_long(LaneReader& r, uint32_t k, uint32_t km,
                                              uint32_t& umax, uint32_t& used) {
  cp_async_wait<kWait>();
  const uint32_t L = (uint32_t)r.window() & km;
  umax = max(umax, L - 1u);
  r.advance(k);
  const uint32_t l = min(max(L, 1u), 64u);
  const uint64_t v = low_bits(r.window(), l);
  r.advance(l);
  used += k + l;
  cp_async_commit();
  return v;
}

// Entries per step for k + largest L bits (1: one entry of up to 64 bits;
// 0: the long form).
__device__ __forceinline__ int entries_per_step(int bits) {
  return bits <= 8 ? 8 : (bits <= 16 ? 4 : (bits <= 32 ? 2 : (bits <= 64 ? 1 : 0)));
}

// Asks L2 for the stream bytes of bits [b0, b1) and the reader's lookahead.
__device__ __forceinline__ void prefetch_span(const uint32_t* words, uint64_t nwords, uint64_t b0,
                                              uint64_t b1) {
  const uint64_t lo = (b0 / 128) * 16;
  const uint64_t hi = umin((b1 + 127) / 128 * 16 + 16, nwords * 4);
  if (hi > lo) {
    const uint32_t size = (uint32_t)umin(hi - lo, 1ull << 20);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(
                     reinterpret_cast<const char*>(words) + lo),
                 "r"(size)
                 : "memory");
  }
}

// The entries of a chunk that ends early (the last one, when rows x cols is
// not a multiple of the index stride), one by one.  False on a bad stream.
template <typename T>
__device__ bool decode_tail(const uint32_t* words, uint64_t limit, uint64_t pos, int cnt, int k,
                            T* out) {
  if (pos >= limit) return false;
  BitReader br(words, pos);
  for (int i = 0; i < cnt; ++i) {
    if (pos + k > limit) return false;
    const int L = (int)br.take(k);
    if (L < 1 || L > 64 || pos + k + L > limit) return false;
    out[i] = (T)br.take64(L);
    pos += k + L;
  }
  return true;
}

// Bounds of the stream span of group g (its chunks' first bit to the bit
// after its last chunk), from the index values its lanes hold.
struct GroupIndex {
  uint64_t pos, end;
};

__device__ __forceinline__ GroupIndex load_group(const uint64_t* index, uint64_t g, uint64_t chunks,
                                                 int lane) {
  const uint64_t c = g * 32 + lane;
  GroupIndex gi{0, 0};
  if (c < chunks) {
    gi.pos = __ldg(index + c);
    gi.end = __ldg(index + c + 1);
  }
  return gi;
}

__device__ __forceinline__ void prefetch_group(const uint32_t* words, uint64_t nwords,
                                               const GroupIndex& gi, uint64_t g, uint64_t chunks,
                                               int lane) {
  if (g * 32 >= chunks) return;
  const int last = (int)umin(chunks - g * 32, 32) - 1;
  const uint64_t b0 = __shfl_sync(0xffffffffu, gi.pos, 0);
  const uint64_t b1 = __shfl_sync(0xffffffffu, gi.end, last);
  if (lane == 0) prefetch_span(words, nwords, b0, b1);
}

template <typename T, int E>
__device__ __forceinline__ void decode_body(const uint32_t* __restrict__ words, uint64_t nwords,
                                            uint64_t limit, const uint64_t* __restrict__ index,
                                            uint64_t n, uint32_t k, uint32_t maxl, T* stage,
                                            uint4* ring_warp, T* __restrict__ out, int32_t* err) {
  const uint32_t km = (1u << k) - 1u;
  const uint64_t chunks = (n + kStride - 1) / kStride;
  const int lane = threadIdx.x % 32;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
  uint64_t wc = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  T* mine = stage + lane * (kRound + 1);
  uint4* ring = ring_warp + lane;
  // index values one group ahead of use, and the L2 prefetch of a group's
  // stream issued one group ahead from values loaded the iteration before
  GroupIndex gi = load_group(index, wc, chunks, lane);
  GroupIndex gn = load_group(index, wc + nwarps, chunks, lane);
  prefetch_group(words, nwords, gi, wc, chunks, lane);
  for (; wc * 32 < chunks; wc += nwarps) {
    const uint64_t c = wc * 32 + lane;
    const GroupIndex cur = gi;
    prefetch_group(words, nwords, gn, wc + nwarps, chunks, lane);
    gi = gn;
    gn = load_group(index, wc + 2 * nwarps, chunks, lane);
    const bool full = (c + 1) * kStride <= n;
    LaneReader r;
    r.init(words, nwords, cur.pos, full ? cur.end : 0, ring);
    uint32_t umax = 0, used = 0;
    for (int rd = 0; rd < kStride / kRound; ++rd) {
      if constexpr (E > 1) {
#pragma unroll
        for (int i = 0; i < kRound; i += E) {
          uint32_t v[E];
          take_short<E>(r, k, km, v, umax, used);
#pragma unroll
          for (int j = 0; j < E; ++j) mine[i + j] = (T)v[j];
        }
      } else if constexpr (E == 1) {
#pragma unroll 4
        for (int i = 0; i < kRound; ++i) mine[i] = (T)take_medium(r, k, km, umax, used);
      } else {
#pragma unroll 4
        for (int i = 0; i < kRound; ++i) mine[i] = (T)take_long(r, k, km, umax, used);
      }
      __syncwarp();
      // 32 / kRound owners' kRound entries per pass: consecutive lanes on
      // consecutive entries
      constexpr int kOwners = 32 / kRound;
#pragma unroll
      for (int j = 0; j < kRound; ++j) {
        const int owner = kOwners * j + lane / kRound, ii = lane % kRound;
        const uint64_t oc = wc * 32 + owner;
        if ((oc + 1) * kStride <= n)
          out[oc * kStride + rd * kRound + ii] = stage[owner * (kRound + 1) + ii];
      }
      __syncwarp();
    }
    bool bad = full && (umax >= maxl || (uint64_t)used != cur.end - cur.pos);
    if (c < chunks && !full)
      bad = !decode_tail<T>(words, limit, cur.pos, (int)(n - c * kStride), (int)k,
                            out + c * kStride);
    if (bad && err) atomicCAS(err, CCM_OK, CCM_E_INPUT);
  }
  cp_async_wait<0>();  // no copy into the ring outlives the CTA
}

// Shared bytes of the decoder (8 warps): the output staging, then the rings.
__host__ __device__ constexpr size_t decode_stage_bytes(size_t elem) {
  return (size_t)8 * 32 * (kRound + 1) * elem;
}
__host__ __device__ constexpr size_t ring_bytes() { return (size_t)8 * 32 * kSlots * 16; }

template <typename T>
__global__ void __launch_bounds__(256) k_vlb_decode(const ccm_header* hdr,
                                                    const uint32_t* __restrict__ words,
                                                    const uint64_t* __restrict__ index,
                                                    uint64_t rows, uint64_t cols,
                                                    uint64_t capacity, T* __restrict__ out,
                                                    int32_t* err) {
  extern __shared__ __align__(16) uint8_t s_raw[];
  T* stage = reinterpret_cast<T*>(s_raw) + (threadIdx.x / 32) * 32 * (kRound + 1);
  uint4* ring = reinterpret_cast<uint4*>(s_raw + decode_stage_bytes(sizeof(T))) +
                (threadIdx.x / 32) * 32 * kSlots;
  int st = check_vlb(hdr, rows, cols, capacity);
  if (st == CCM_OK && sizeof(T) == 4 && (int)hdr->reserved0 > 31) st = CCM_E_WIDTH;
  if (st != CCM_OK) {
    if (err && blockIdx.x == 0 && threadIdx.x == 0) *err = st;
    return;
  }
  const uint32_t k = (uint32_t)hdr->width, maxl = (uint32_t)hdr->reserved0;
  const uint64_t nwords = hdr->nwords, limit = hdr->stat_or, n = rows * cols;
  switch (entries_per_step((int)(k + maxl))) {
    case 8: decode_body<T, 8>(words, nwords, limit, index, n, k, maxl, stage, ring, out, err); break;
    case 4: decode_body<T, 4>(words, nwords, limit, index, n, k, maxl, stage, ring, out, err); break;
    case 2: decode_body<T, 2>(words, nwords, limit, index, n, k, maxl, stage, ring, out, err); break;
    case 1: decode_body<T, 1>(words, nwords, limit, index, n, k, maxl, stage, ring, out, err); break;
    default: decode_body<T, 0>(words, nwords, limit, index, n, k, maxl, stage, ring, out, err); break;
  }
}

// y = A x, fast path: cols a multiple of the index stride (no chunk crosses a
// row), x of at most 32 bits staged in shared memory as int32 (one pad word
// per 64 columns, so that the lanes' columns 64 apart fall in different
// banks), and every partial sum inside int64 (largest L + b_x + bitlen(cols)
// <= 63).  Each lane accumulates its chunk in int64; a warp whose 32 chunks
// lie in one row adds their sum with one atomic, otherwise each lane adds its
// own.  When the conditions hold (decided from the headers, the same in every
// CTA) block 0 sets *done and the general kernel after it returns at once.
template <int E>
__device__ __forceinline__ void mv_body(const uint32_t* __restrict__ words, uint64_t nwords,
                                        const uint64_t* __restrict__ index, uint64_t rows,
                                        uint64_t cols, uint32_t k, uint32_t maxl,
                                        const int32_t* xs, uint4* ring_warp,
                                        int64_t* __restrict__ y, ccm_header* out) {
  const uint32_t km = (1u << k) - 1u;
  const uint64_t chunks = rows * cols / kStride;
  const int lane = threadIdx.x % 32;
  const uint64_t nwarps = (uint64_t)gridDim.x * (blockDim.x / 32);
  uint64_t wc = (uint64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  uint4* ring = ring_warp + lane;
  // index values one group ahead of use, and the L2 prefetch of a group's
  // stream issued one group ahead from values loaded the iteration before
  GroupIndex gi = load_group(index, wc, chunks, lane);
  GroupIndex gn = load_group(index, wc + nwarps, chunks, lane);
  prefetch_group(words, nwords, gi, wc, chunks, lane);
  int bad = 0;
  for (; wc * 32 < chunks; wc += nwarps) {
    const uint64_t c = wc * 32 + lane;
    const GroupIndex cur = gi;
    prefetch_group(words, nwords, gn, wc + nwarps, chunks, lane);
    gi = gn;
    gn = load_group(index, wc + 2 * nwarps, chunks, lane);
    const bool active = c < chunks;
    const uint64_t row = active ? c * kStride / cols : 0;
    const uint64_t col0 = active ? c * kStride - row * cols : 0;
    const int32_t* xr = xs + col0 + col0 / kStride;
    LaneReader r;
    r.init(words, nwords, cur.pos, active ? cur.end : 0, ring);
    uint32_t umax = 0, used = 0;
    long long acc = 0;
    for (int rd = 0; rd < kStride / kRound; ++rd, xr += kRound) {
      if constexpr (E > 1) {
#pragma unroll
        for (int i = 0; i < kRound; i += E) {
          uint32_t v[E];
          take_short<E>(r, k, km, v, umax, used);
#pragma unroll
          for (int j = 0; j < E; ++j) acc += (long long)(int32_t)v[j] * xr[i + j];
        }
      } else if constexpr (E == 1) {
#pragma unroll 4
        for (int i = 0; i < kRound; ++i)
          acc += (long long)take_medium(r, k, km, umax, used) * (long long)xr[i];
      } else {
#pragma unroll 4
        for (int i = 0; i < kRound; ++i)
          acc += (long long)take_long(r, k, km, umax, used) * (long long)xr[i];
      }
    }
    bad |= active && (umax >= maxl || (uint64_t)used != cur.end - cur.pos);
    if (!active) acc = 0;  // (lanes past the last chunk walked the stream start)
    const uint64_t row0 = __shfl_sync(0xffffffffu, row, 0);
    if (__all_sync(0xffffffffu, !active || row == row0)) {
      for (int d = 16; d; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
      if (lane == 0 && acc)
        atomicAdd(reinterpret_cast<unsigned long long*>(y + row0), (unsigned long long)acc);
    } else if (active && acc) {
      atomicAdd(reinterpret_cast<unsigned long long*>(y + row), (unsigned long long)acc);
    }
  }
  cp_async_wait<0>();  // no copy into the ring outlives the CTA
  if (bad) set_status(out, CCM_E_INPUT);
}

// int32 words of the staged x (one pad word per 64 columns, a multiple of 4).
__host__ __device__ constexpr uint64_t mv_x_words(uint64_t cols) {
  return (cols + cols / kStride + 3) & ~3ull;
}

__global__ void __launch_bounds__(256) k_vlb_mv_fast(const ccm_header* hdr,
                                                     const uint32_t* __restrict__ words,
                                                     const uint64_t* __restrict__ index,
                                                     uint64_t rows, uint64_t cols,
                                                     uint64_t capacity, ccm_header* out,
                                                     const ccm_header* hx,
                                                     const uint32_t* __restrict__ wx,
                                                     int64_t* __restrict__ y,
                                                     unsigned long long* done) {
  extern __shared__ __align__(16) int32_t s_x[];
  uint4* ring = reinterpret_cast<uint4*>(s_x + mv_x_words(cols)) + (threadIdx.x / 32) * 32 * kSlots;
  if (out->status != CCM_OK || check_vlb(hdr, rows, cols, capacity) != CCM_OK) return;
  const uint32_t k = (uint32_t)hdr->width, maxl = (uint32_t)hdr->reserved0;
  const int bx = hx->width, sx = hx->is_signed;
  if (bx > 32 || (int)maxl + bx + bitlen64(cols) > 63) return;  // the general kernel
  if (blockIdx.x == 0 && threadIdx.x == 0) *done = 1;
  for (uint64_t j = threadIdx.x; j < cols; j += blockDim.x)
    s_x[j + j / kStride] = (int32_t)decode_field(wx, j, bx, sx);
  __syncthreads();
  const uint64_t nwords = hdr->nwords;
  switch (entries_per_step((int)(k + maxl))) {
    case 8: mv_body<8>(words, nwords, index, rows, cols, k, maxl, s_x, ring, y, out); break;
    case 4: mv_body<4>(words, nwords, index, rows, cols, k, maxl, s_x, ring, y, out); break;
    case 2: mv_body<2>(words, nwords, index, rows, cols, k, maxl, s_x, ring, y, out); break;
    case 1: mv_body<1>(words, nwords, index, rows, cols, k, maxl, s_x, ring, y, out); break;
    default: mv_body<0>(words, nwords, index, rows, cols, k, maxl, s_x, ring, y, out); break;
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

namespace {

__global__ void k_vlb_err_init(int32_t* err) { *err = CCM_OK; }

// Resident CTAs per SM of `kern` with `smem` dynamic bytes (at least 1).
template <class K>
int resident(K kern, int threads, size_t smem) {
  int per = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem) != cudaSuccess ||
      per < 1)
    per = 1;
  return per;
}

template <typename T>
void launch_decode(const ccm_header* hdr, const uint32_t* words, uint64_t capacity,
                   const uint64_t* index, uint64_t rows, uint64_t cols, T* out, int32_t* err,
                   cudaStream_t st) {
  const uint64_t n = rows * cols;
  const uint64_t groups = (n + 32 * vlb::kStride - 1) / (32 * vlb::kStride);
  const size_t smem = vlb::decode_stage_bytes(sizeof(T)) + vlb::ring_bytes();
  static int dev_done = -1, per_sm = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev_done != dev) {
    cudaFuncSetAttribute(vlb::k_vlb_decode<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    per_sm = resident(vlb::k_vlb_decode<T>, 256, smem);
    dev_done = dev;
  }
  const int g = (int)umin(umax((groups + 7) / 8, 1), (uint64_t)num_sms() * per_sm);
  if (err) {
    k_vlb_err_init<<<1, 1, 0, st>>>(err);
    note_launch();
  }
  profile_begin(st);
  vlb::k_vlb_decode<T><<<g, 256, smem, st>>>(hdr, words, index, rows, cols, capacity, out, err);
  profile_end(st);
  note_launch();
}

}  // namespace

// The fast decoder reads the stream 8 bytes at a time and prefetches it with
// 16-byte aligned bulk requests: it takes `words` 16-byte aligned; the
// one-thread-per-chunk decoder below takes any 4-byte alignment.
void run_vlb_unpack(const ccm_header* hdr, const uint32_t* words, uint64_t capacity,
                    const uint64_t* index, uint64_t rows, uint64_t cols, void* dense, int dtype,
                    int32_t* err, cudaStream_t st) {
  const uint64_t n = rows * cols;
  if (reinterpret_cast<uintptr_t>(words) % 16 == 0) {
    if (dtype == CCM_I64)
      launch_decode<int64_t>(hdr, words, capacity, index, rows, cols, (int64_t*)dense, err, st);
    else
      launch_decode<int32_t>(hdr, words, capacity, index, rows, cols, (int32_t*)dense, err, st);
    return;
  }
  const uint64_t chunks = (n + vlb::kStride - 1) / vlb::kStride;
  const uint64_t warp_groups = (chunks + 31) / 32;
  if (err) {
    k_vlb_err_init<<<1, 1, 0, st>>>(err);
    note_launch();
  }
  const int g = (int)umin(umax((warp_groups + vlb::kUnpackWarps - 1) / vlb::kUnpackWarps, 1),
                          (uint64_t)num_sms() * 8);
  const int threads = vlb::kUnpackWarps * 32;
  const size_t per = (size_t)vlb::kUnpackWarps * 32 * (vlb::kHalf + 1);
  profile_begin(st);
  if (dtype == CCM_I64) {
    static int attr_dev = -1;
    int dev = 0;
    cudaGetDevice(&dev);
    if (attr_dev != dev) {
      cudaFuncSetAttribute(vlb::k_vlb_unpack<int64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)(per * sizeof(int64_t)));
      attr_dev = dev;
    }
    vlb::k_vlb_unpack<int64_t><<<g, threads, per * sizeof(int64_t), st>>>(
        hdr, words, index, rows, cols, capacity, (int64_t*)dense, err);
  } else {
    vlb::k_vlb_unpack<int32_t><<<g, threads, per * sizeof(int32_t), st>>>(
        hdr, words, index, rows, cols, capacity, (int32_t*)dense, err);
  }
  profile_end(st);
  note_launch();
}

}  // namespace ccm

namespace ccm {

size_t vlb_matvec_workspace(uint64_t rows) { return ((rows * 8 + 255) & ~(size_t)255) + 256; }

// Widest x the fast matvec stages in shared memory (66.5 KB as int32).
constexpr uint64_t kFastMaxCols = 16384;

void run_vlb_matvec(const ccm_header* hdr, const uint32_t* words, uint64_t capacity,
                    const uint64_t* index, uint64_t rows, uint64_t cols, const ccm_matrix& x,
                    const ccm_matrix& y, void* ws, cudaStream_t st) {
  int64_t* yv = (int64_t*)ws;
  InitArgs ia{};
  ia.out = y.hdr;
  ia.in0 = x.hdr;
  ia.in0_rows = x.rows;
  ia.in0_cols = x.cols;
  ia.in0_capacity = x.capacity;
  ia.out_rows = y.rows;
  ia.out_cols = y.cols;
  ia.zero_ptr = yv;
  ia.zero_count = rows + 1;  // y, then the fast kernel's flag
  launch_init(ia, st);
  if (rows && cols) {
    unsigned long long* done = reinterpret_cast<unsigned long long*>(yv + rows);
    // fast kernel: chunks within rows, x staged in shared memory, aligned stream
    const bool fast = cols % vlb::kStride == 0 && cols <= kFastMaxCols &&
                      reinterpret_cast<uintptr_t>(words) % 16 == 0;
    const int g = (int)umin((rows + 7) / 8, (uint64_t)num_sms() * 8);
    profile_begin(st);
    if (fast) {
      const size_t smem = vlb::mv_x_words(cols) * sizeof(int32_t) + vlb::ring_bytes();
      static int dev_done = -1;
      int dev = 0;
      cudaGetDevice(&dev);
      if (dev_done != dev) {
        cudaFuncSetAttribute(vlb::k_vlb_mv_fast, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(vlb::mv_x_words(kFastMaxCols) * sizeof(int32_t) +
                                   vlb::ring_bytes()));
        dev_done = dev;
      }
      const uint64_t groups = (rows * cols / vlb::kStride + 31) / 32;
      const int gf = (int)umin(umax((groups + 7) / 8, 1),
                               (uint64_t)num_sms() * resident(vlb::k_vlb_mv_fast, 256, smem));
      vlb::k_vlb_mv_fast<<<gf, 256, smem, st>>>(hdr, words, index, rows, cols, capacity, y.hdr,
                                                 x.hdr, x.words, yv, done);
      note_launch();
    }
    vlb::k_vlb_matvec<<<g, 256, 0, st>>>(hdr, words, index, rows, cols, capacity, y.hdr, x.hdr,
                                         x.words, yv, fast ? done : nullptr);
    profile_end(st);
    note_launch();
  }
  run_pack_scratch(yv, y, st);
}

}  // namespace ccm
