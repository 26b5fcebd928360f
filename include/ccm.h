/*
 * ccm.h -- C ABI of libccm: computable compressed matrices on one GPU.
 *
 * A matrix of integers is stored in the paper's "Supreme Minimum" (SM) form
 * (Methods, "Method 1: The Supreme Minimum"): every entry takes the same
 * number of bits b, the smallest that holds every entry (Eq. 1), and the
 * entries, unravelled row-major, are laid end to end in one LSB-first bit
 * stream -- entry e owns bits [e*b, (e+1)*b) -- cut into 32-bit little-endian
 * words (Eq. 3 and the step-by-step example after it: fields fill each word
 * from its least significant bit upward, and a field that does not fit in the
 * rest of a word straddles into the next one, low bits first).  32-bit little-endian words
 * are byte-for-byte the paper's 64-bit bitstrings.
 *
 * Sign: the paper only treats non-negative entries (Methods, Matrix
 * compression).  This library reads Eq. 1 as follows.  When no entry is
 * negative the fields are unsigned and b = max(1, bitlen(max)), exactly
 * Eq. 1.  Otherwise the fields are two's complement and
 * b = 1 + max over entries of bitlen(a >= 0 ? a : -a - 1), the smallest b
 * whose range [-2^(b-1), 2^(b-1)-1] holds every entry.  Widths run 1..64.
 *
 * Word count: ceil(rows*cols*b/32) data words, zero padded to a multiple of 4
 * words (16 bytes); bits above the last field and the pad words are zero, so
 * a packed matrix has exactly one representation.
 *
 * Operations on the compressed form (add, scale, matvec, matmul) compute the
 * same integers as the operation on the uncompressed matrices (Introduction:
 * the compressed form is meant to support the same mathematics as the
 * original), exactly, and re-pack the result at its own new width by the rule
 * above.
 *
 * Conventions for every entry point:
 *  - All data pointers are DEVICE pointers on the current CUDA device and are
 *    owned by the caller (the library never frees them).  `ccm_matrix` and
 *    `ccm_header` pointers passed as arguments are HOST pointers to small
 *    structs that carry those device pointers.
 *  - Calls are asynchronous on `stream` (NULL = the legacy default stream)
 *    unless documented as synchronous.
 *  - Host-detectable errors (NULL pointers, bad dtype, shape mismatch,
 *    too-small capacity or workspace) return a negative ccm_status at once and
 *    launch nothing.  A shape whose rows*cols exceeds 2^57 fields (or wraps
 *    uint64) is CCM_E_INVAL; ccm_workspace_bytes returns SIZE_MAX for it. 
 *  - Data-dependent errors (int64 overflow of a result, a result whose width
 *    needs more words than the output capacity, an input header that is not a
 *    valid matrix) are written by the GPU into the output header's `status`;
 *    the output words are then left unwritten.  An input whose header carries
 *    an error passes that error on to the output, so a chain of calls needs no
 *    host synchronisation and still reports the first failure.
 *  - No call traps, asserts or spins on the GPU.
 */
#ifndef CCM_H
#define CCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* ccm_stream_t; /* the same handle as cudaStream_t */

typedef enum ccm_status {
  CCM_OK = 0,
  CCM_E_INVAL = -1,    /* NULL pointer, bad dtype/path/op code */
  CCM_E_SHAPE = -2,    /* operand shapes do not agree */
  CCM_E_WIDTH = -3,    /* a width outside 1..64, or int32 output for a field that needs more */
  CCM_E_OVERFLOW = -4, /* an exact result does not fit int64 */
  CCM_E_CAPACITY = -5, /* output words or workspace too small */
  CCM_E_RANGE = -6,    /* element index out of range */
  CCM_E_CUDA = -7,     /* a CUDA runtime call failed */
  CCM_E_TIMEOUT = -8,  /* a bounded device wait gave up */
  CCM_E_INPUT = -9     /* an input header is not a valid packed matrix */
} ccm_status;

typedef enum ccm_dtype { CCM_I32 = 0, CCM_I64 = 1 } ccm_dtype;

#define CCM_MAGIC 0x314D4343u /* "CCM1" */
#define CCM_HEADER_BYTES 64

/* Device-resident header of a packed matrix (64 bytes, 16-byte aligned).
 * Written by the library; callers read it with ccm_header_read(). */
typedef struct ccm_header {
  uint32_t magic;     /* CCM_MAGIC once a call has produced the matrix */
  int32_t width;      /* b, 1..64 */
  int32_t is_signed;  /* 0: unsigned fields (Eq. 1); 1: two's complement */
  int32_t status;     /* CCM_OK or the data-dependent error of the producing call */
  uint64_t rows;
  uint64_t cols;
  uint64_t nwords;    /* ccm_words_for(rows, cols, width) */
  uint64_t stat_or;   /* internal: OR over the result of (a >= 0 ? a : ~a) */
  uint32_t stat_neg;  /* internal: 1 when some entry of the result is negative */
  uint32_t reserved0;  /* internal (VLB: the largest entry bit length; add/scale written
                          by the lane pass: the width that pass wrote) */
  uint64_t reserved1;  /* internal (1: an add/scale was written by its lane pass; pack: a
                          tile reached the width the capacity bounds) */
} ccm_header;

/* Host-side handle of one packed matrix: where it lives and its shape.
 * `hdr` and `words` are device pointers, both 16-byte aligned; `capacity`
 * counts the uint32 words available at `words`.  `rows`/`cols` are the shape the caller expects; the
 * library checks them against each other on the host and against the header
 * on the GPU. */
typedef struct ccm_matrix {
  ccm_header* hdr;
  uint32_t* words;
  uint64_t capacity;
  uint64_t rows;
  uint64_t cols;
} ccm_matrix;

/* Operation codes for ccm_workspace_bytes. */
typedef enum ccm_op {
  CCM_OP_MATVEC = 1,
  CCM_OP_MATMUL = 2,
  CCM_OP_PACK = 3,
  CCM_OP_VLB = 4,
  CCM_OP_VLB_MATVEC = 5
} ccm_op;

/* Matmul paths. */
typedef enum ccm_matmul_path {
  CCM_MATMUL_AUTO = 0,
  CCM_MATMUL_TENSOR = 1,  /* exact 4-bit limb decomposition on the tcgen05 tensor cores */
  CCM_MATMUL_CUDACORE = 2 /* decode-and-multiply on the integer ALUs */
} ccm_matmul_path;

/* Words needed for rows*cols fields of `width` bits: ceil(n*width/32) rounded
 * up to a multiple of 4 (Methods, Method 1: the paper's bitstring count,
 * restated for 32-bit words and 16-byte padding).  0 for an empty matrix or a
 * width outside 1..64. */
uint64_t ccm_words_for(uint64_t rows, uint64_t cols, int width);

/* Result-width bounds (Methods, Method 1: Eq. 1, with this library's signed
 * reading, applied to the range of every result that operands of the given
 * widths and sign modes allow; a b-bit field holds [0, 2^b - 1] unsigned or
 * [-2^(b-1), 2^(b-1) - 1] signed).  Each returns the smallest width that holds
 * any possible result, so an output of ccm_words_for(rows, cols, bound) words
 * can never be short of capacity; the exact width of an actual result may be
 * smaller.  The bound is capped at 64: a result beyond int64 is reported by
 * the operation itself as CCM_E_OVERFLOW.  A width outside 1..64 returns
 * CCM_E_WIDTH (negative).  Pure host functions: no GPU, no synchronisation
 * (read the operand widths with ccm_header_read first).
 *  ccm_bound_add:    C = A + B; range [lo_A + lo_B, hi_A + hi_B].
 *  ccm_bound_scale:  C = s A; range s * [lo_A, hi_A].
 *  ccm_bound_matvec: y = A x with `cols` columns: cols times the smallest and
 *                    the largest product of the range ends (1 when cols = 0).
 *  ccm_bound_matmul: C = A B with inner size `inner`, the same rule. */
int ccm_bound_add(int width_a, int signed_a, int width_b, int signed_b);
int ccm_bound_scale(int width_a, int signed_a, int64_t s);
int ccm_bound_matvec(int width_a, int signed_a, int width_x, int signed_x, uint64_t cols);
int ccm_bound_matmul(int width_a, int signed_a, int width_b, int signed_b, uint64_t inner);

/* Human-readable name of a status code (static storage). */
const char* ccm_status_str(int status);

/* Library version, major*10000 + minor*100 + patch. */
int ccm_version(void);

/* Width selection only (Eq. 1 with the signed reading): scans rows*cols
 * dense entries (`dtype` CCM_I32 or CCM_I64, row-major, device) and writes
 * width, is_signed, nwords, rows, cols and status into `hdr` (device).
 * Lets a caller size the output exactly before ccm_pack. */
ccm_status ccm_measure(const void* dense, int dtype, uint64_t rows, uint64_t cols,
                       ccm_header* hdr, ccm_stream_t stream);

/* SM compression (Methods, Method 1; Eq. 1 and Eq. 3): width selection over
 * the dense matrix, then every entry written as a b-bit field at bit e*b of
 * the stream.  `dense` is rows*cols entries of `dtype`, row-major, device.
 * Output in `out` (header + words).  If the exact width needs more than
 * out->capacity words the header gets CCM_E_CAPACITY and no words.
 * `ws` (optional, device, 256-byte aligned) of at least
 * ccm_workspace_bytes(CCM_OP_PACK, rows, cols, out->capacity) bytes lets the
 * dense input be read once instead of twice (tiles packed at their own width,
 * then re-coded); NULL or a smaller workspace takes the two-pass route.  The
 * result is the same either way. */
ccm_status ccm_pack(const void* dense, int dtype, uint64_t rows, uint64_t cols,
                    const ccm_matrix* out, void* ws, size_t ws_bytes, ccm_stream_t stream);

/* Decompression: every field read back and sign- or zero-extended to
 * `dtype`, row-major into `dense` (rows*cols entries, device).  CCM_I32
 * output needs signed b <= 32 or unsigned b <= 31; otherwise CCM_E_WIDTH is
 * written to `*err` (device int32, may be NULL) and `dense` is untouched.
 * `*err` is set to CCM_OK on success when given. */
ccm_status ccm_unpack(const ccm_matrix* a, void* dense, int dtype, int32_t* err,
                      ccm_stream_t stream);

/* Element access by row and column (Methods, Matrix compression: access to
 * any element given its row i and column j).  `idx` holds `count` flat
 * row-major indices i*cols + j (device uint64); `out` receives `count` int64
 * entries (device).  An index >= rows*cols yields 0 and CCM_E_RANGE in
 * `*err` (device int32, may be NULL). */
ccm_status ccm_get(const ccm_matrix* a, const uint64_t* idx, uint64_t count, int64_t* out,
                   int32_t* err, ccm_stream_t stream);

/* C = A + B, exact, entrywise; A, B and C have the same shape; A and B may
 * have different widths and sign modes.  C is re-packed at its own width.
 * One pass writes C at the width the input ranges bound the sum to; a second
 * pass re-packs only when the exact width is smaller (and when that bound
 * needs more than c->capacity words).  `ws`, `ws_bytes`: not used (any
 * value, NULL included). */
ccm_status ccm_add(const ccm_matrix* a, const ccm_matrix* b, const ccm_matrix* c, void* ws,
                   size_t ws_bytes, ccm_stream_t stream);

/* C = s * A for an int64 scalar s, exact; CCM_E_OVERFLOW when an entry does
 * not fit int64.  C is re-packed at its own width, in one pass when s times
 * the range of A's width is the result's exact width, as for ccm_add.
 * `ws`, `ws_bytes`: not used. */
ccm_status ccm_scale(const ccm_matrix* a, int64_t s, const ccm_matrix* c, void* ws,
                     size_t ws_bytes, ccm_stream_t stream);

/* y = A x: A is m x n, x is a packed n x 1 matrix, y a packed m x 1 matrix,
 * y_i = sum_j a_ij x_j exactly (CCM_E_OVERFLOW when y_i does not fit int64).
 * `ws` is device workspace of at least ccm_workspace_bytes(CCM_OP_MATVEC,
 * m, n, 1) bytes, 256-byte aligned; its contents need no initialisation. */
ccm_status ccm_matvec(const ccm_matrix* a, const ccm_matrix* x, const ccm_matrix* y, void* ws,
                      size_t ws_bytes, ccm_stream_t stream);

/* y = A x + B z in one chain that stays compressed: A is m x n1, B is
 * m x n2, x and z packed n1 x 1 and n2 x 1; both products are summed exactly
 * in one int64 scratch and y is packed once, at the sum's exact width (no
 * intermediate vector is packed or unpacked).  The paper's setting of
 * producing, compressing and then manipulating data (Introduction) as one
 * operation; CCM_E_OVERFLOW when y_i does not fit int64.  `ws`: at least
 * ccm_workspace_bytes(CCM_OP_MATVEC, m, max(n1, n2), 1) bytes, 256-byte
 * aligned. */
ccm_status ccm_matvec2(const ccm_matrix* a, const ccm_matrix* x, const ccm_matrix* b,
                       const ccm_matrix* z, const ccm_matrix* y, void* ws, size_t ws_bytes,
                       ccm_stream_t stream);

/* C = A B: A is m x k, B is k x n, C is m x n, exact int64 entries
 * (CCM_E_OVERFLOW otherwise), re-packed at C's own width.  `path` selects the
 * tensor-core limb path or the CUDA-core path (AUTO = tensor when the inputs
 * allow it).  `ws` as for ccm_matvec with CCM_OP_MATMUL and (m, k, n). */
ccm_status ccm_matmul(const ccm_matrix* a, const ccm_matrix* b, const ccm_matrix* c, int path,
                      void* ws, size_t ws_bytes, ccm_stream_t stream);

/* Device workspace needed by `op` on an m x k by k x n problem (matvec: n = 1
 * is the vector, k the inner size).  An upper bound over all operand widths
 * (for matmul: the tensor path's digit planes at 4 digits per field).  For
 * CCM_OP_PACK the arguments are (rows, cols, output capacity in words). */
size_t ccm_workspace_bytes(int op, uint64_t m, uint64_t k, uint64_t n);

/* Synchronous copy of a device header to host memory (waits for `stream`). */
ccm_status ccm_header_read(const ccm_header* dev, ccm_header* host, ccm_stream_t stream);

/* Synthetic inputs, generated on the GPU by the counter-based SplitMix64
 * scheme of the test-input generator: entry i of stream `stream_id` under
 * `seed` is mix(key + (i + 1) * 0x9E3779B97F4A7C15) with
 * key = mix(seed + (stream_id + 1) * 0x9E3779B97F4A7C15) and mix the
 * SplitMix64 finaliser (Steele, Lea and Flood 2014).  `start` offsets i.
 * ccm_gen_uniform: int64 in [lo, hi] by the multiply-high map.
 * ccm_gen_poisson: inversion of `table` (float64 CDF, `table_len` entries,
 * device) on u = (draw >> 11) * 2^-53: the count of entries <= u. */
ccm_status ccm_gen_uniform(int64_t* out, uint64_t count, uint64_t seed, uint64_t stream_id,
                           uint64_t start, int64_t lo, int64_t hi, ccm_stream_t stream);
ccm_status ccm_gen_poisson(int64_t* out, uint64_t count, uint64_t seed, uint64_t stream_id,
                           uint64_t start, const double* table, uint32_t table_len,
                           ccm_stream_t stream);

/* Re-pack at a given width (Methods, Method 1: the same fields written with
 * b = `width` bits each, two's complement when `is_signed`), into rows
 * [row_offset, row_offset + in->rows) of `out` (out->rows >= that, same
 * cols).  Every other word of out (its other rows, the bits above the block's
 * last field, the pad words) is set to zero, and out's header describes the
 * whole out->rows x cols matrix at `width`.  This is the assembly step of a
 * matvec split by rows across devices: each device re-packs its block of y at
 * the width all blocks agree on (the maximum of their width statistics), and
 * since the blocks occupy disjoint word ranges, a sum (or OR) of the devices'
 * word buffers is the packed y.  Host checks: width 1..64 (CCM_E_WIDTH),
 * row_offset*cols*width a multiple of 32 for a non-empty block, i.e. the
 * block starts on a word boundary (CCM_E_SHAPE; row_offset a multiple of 32
 * always qualifies), out
 * capacity for the whole matrix at `width` (CCM_E_CAPACITY).  On the GPU: an
 * input whose width or sign mode does not fit the target gets CCM_E_WIDTH in
 * out's header and no words are written.  out's stat_or/stat_neg are zero. */
ccm_status ccm_repack(const ccm_matrix* in, int width, int is_signed, const ccm_matrix* out,
                      uint64_t row_offset, ccm_stream_t stream);

/* ---------------------------------------------------------------------------
 * Batched matvec: y_i = A_i x_i for many packed matrices of uneven shapes and
 * widths in one persistent launch (same arithmetic as ccm_matvec, applied to
 * every entry).  Limits per entry: cols <= 8192 (checked on the host);
 * width(A) <= 32, width(x) <= 31 and width(A) + width(x) + bitlen(cols) <= 63
 * so that every sum fits int64 (checked on the GPU: an entry outside them gets
 * CCM_E_WIDTH in its y header and the other entries are unaffected).
 *
 * ccm_batch_plan (synchronous) validates every entry on the host, cuts each
 * matrix into work units of `unit_segments` row segments (a multiple of 32;
 * a segment is up to 32 consecutive fields of one row) and writes the plan
 * (entry descriptors + unit list) to `plan`, a device buffer of at least
 * ccm_batch_plan_bytes(...) bytes, 256-byte aligned; `info` (host) receives
 * the counts the launch needs.  The entries' device pointers are baked into
 * the plan: the buffers must stay where they are while the plan is used.
 *
 * ccm_batch_matvec launches an initialisation kernel (validates the headers,
 * clears y headers and the scratch, decodes every x into an image in `ws`:
 * bytes when x fits 8 signed or 7 unsigned bits and width(A) <= 24, else
 * int32), a one-CTA kernel that orders the valid entries' units by width and
 * sign, and the persistent kernel (`grid` CTAs; <= 0 picks one resident
 * wave).  Each warp of the persistent kernel takes work units in that order
 * from an atomic ticket and streams their words through info->slots ring slots in shared
 * memory, each stage one bulk copy of about info->stage_bytes bytes (the
 * segments per lane follow from the width).  The slots are sized for A widths
 * up to info->max_width.  An info with max_width outside 1..32 or max_cols
 * above 8192, slots other than 0 (= 3) or 2..4, stage_bytes other than 0
 * (= 3072) or 128..16384, or a ring whose shared memory exceeds the
 * device's: CCM_E_INVAL.  `ws` is device workspace of at least
 * ccm_batch_workspace_bytes(...) bytes, 256-byte aligned.  Each y_i header
 * receives its own status (CCM_E_TIMEOUT if a bounded wait on a copy gave
 * up).  The three launches are stream-ordered and can be captured in a CUDA
 * graph. */
typedef struct ccm_batch_entry {
  ccm_matrix a; /* m x n */
  ccm_matrix x; /* n x 1 */
  ccm_matrix y; /* m x 1 (output) */
} ccm_batch_entry;

typedef struct ccm_batch_info {
  uint32_t count;         /* entries */
  uint32_t units;         /* work units */
  uint64_t y_rows;        /* sum of the entries' rows */
  uint32_t unit_segments; /* segments per unit */
  uint32_t max_cols;      /* widest entry (at most 8192 columns) */
  uint64_t plan_bytes;
  uint32_t max_width;     /* widest A the capacities admit, <= 32 (sizes the staging) */
  uint32_t slots;         /* ring slots per warp: 0 (default 3) or 2..4; set to 0 by the
                             plan, the caller may change it before ccm_batch_matvec */
  uint64_t x_ints;        /* ints of the decoded-x images in the workspace */
  uint32_t stage_bytes;   /* bytes of A per warp stage: 0 (default 3072) or 128..16384;
                             set to 0 by the plan, the caller may change it */
  uint32_t reserved;      /* 0 */
} ccm_batch_info;

size_t ccm_batch_plan_bytes(const ccm_batch_entry* entries, int count, uint32_t unit_segments);
size_t ccm_batch_workspace_bytes(const ccm_batch_entry* entries, int count);
ccm_status ccm_batch_plan(const ccm_batch_entry* entries, int count, uint32_t unit_segments,
                          void* plan, size_t plan_bytes, ccm_batch_info* info);
ccm_status ccm_batch_matvec(const void* plan, const ccm_batch_info* info, void* ws,
                            size_t ws_bytes, int grid, ccm_stream_t stream);

/* ---------------------------------------------------------------------------
 * VLB, the paper's second encoding (Methods, "Method 2: Variable Length
 * Blocks", Eq. 9-13): each entry is a k-bit prefix holding its bit length L
 * (the bit length of 0 is 1, Eq. 1) followed by the entry in L bits, LSB-first
 * in one stream of 32-bit words; k is the bit length of the largest L.
 * Non-negative entries only (a negative entry: CCM_E_RANGE in the header).
 * Header: magic CCM_VLB_MAGIC, width = k, nwords, rows, cols, stat_or = total
 * bits of the stream, reserved0 = largest L.  Because entries have no fixed
 * position, the encoder also writes an index: the bit offset of every
 * CCM_VLB_INDEX_STRIDE-th entry, plus the total bits as the last entry
 * (ccm_vlb_index_entries(rows, cols) uint64 values, device) -- the decoder
 * needs it; the paper's format has no index.
 * ccm_vlb_pack: `dense` as for ccm_pack; `words` NULL measures only (header
 * gets k, total bits and nwords: the size to compare with SM's rows*cols*b
 * bits, Eq. 15 vs Eq. 16).  `ws`: ccm_workspace_bytes(CCM_OP_VLB, rows,
 * cols, 0) bytes, 256-byte aligned.  A stream needing more than `capacity`
 * words: CCM_E_CAPACITY in the header.
 * ccm_vlb_unpack: entries back to `dense` (`dtype`); CCM_I32 needs L <= 31.
 * Status to `*err` (device, may be NULL) as for ccm_unpack; a stream that does
 * not parse (a length outside [1, largest L], or an index chunk that does not
 * end where the next index entry says) sets CCM_E_INPUT.  `words` 16-byte
 * aligned takes the fast decoder (a register bit window per lane, the stream
 * staged by cp.async); any 4-byte alignment is accepted. */
#define CCM_VLB_MAGIC 0x31564343u /* "CCV1" */
#define CCM_VLB_INDEX_STRIDE 64
uint64_t ccm_vlb_index_entries(uint64_t rows, uint64_t cols);
ccm_status ccm_vlb_pack(const void* dense, int dtype, uint64_t rows, uint64_t cols,
                        ccm_header* hdr, uint32_t* words, uint64_t capacity, uint64_t* index,
                        void* ws, size_t ws_bytes, ccm_stream_t stream);
ccm_status ccm_vlb_unpack(const ccm_header* hdr, const uint32_t* words, uint64_t capacity,
                          const uint64_t* index, uint64_t rows, uint64_t cols, void* dense,
                          int dtype, int32_t* err, ccm_stream_t stream);

/* y = A x with A (rows x cols) in VLB form -- the operation of Introduction
 * ("computable": work on the compressed matrix) on Method 2's encoding: each
 * entry is decoded from the stream as it is used (the index locates every
 * 64th entry), never stored densely.  x and y are SM matrices as for
 * ccm_matvec (x: cols x 1, y: rows x 1, y re-packed at its exact width).
 * `ws`: ccm_workspace_bytes(CCM_OP_VLB_MATVEC, rows, cols, 0) bytes,
 * 256-byte aligned.  Errors as for ccm_matvec; a VLB header that does not
 * match (rows, cols, capacity) or a stream that ends early: CCM_E_INPUT in
 * y's header. */
ccm_status ccm_vlb_matvec(const ccm_header* hdr, const uint32_t* words, uint64_t capacity,
                          const uint64_t* index, uint64_t rows, uint64_t cols,
                          const ccm_matrix* x, const ccm_matrix* y, void* ws, size_t ws_bytes,
                          ccm_stream_t stream);

/* Matvec that allocates nothing (the paper has no counterpart; this is a
 * service of the library).  For callers that cannot hand ccm_matvec a device
 * workspace because they must not allocate device memory: a process whose
 * GPU memory is reserved in full by another component's allocator, or a
 * latency-critical path that cannot afford the device-wide synchronisation a
 * cudaMalloc/cudaFree may cause.  Same operation, arguments and results as
 * ccm_matvec, minus the workspace: the scratch is a fixed array of
 * CCM_STATIC_SCRATCH_BYTES compiled into libccm, present on every GPU that
 * loads the library until the process exits.
 *  - Size limit: A (rows x cols) needs up256(8*cols) + up256(8*rows) + 256
 *    bytes of it (up256 rounds up to a multiple of 256), as
 *    ccm_workspace_bytes(CCM_OP_MATVEC, rows, cols, 1) reports; larger
 *    problems return CCM_E_CAPACITY at once, before any other check but the
 *    NULL and shape checks (rows + cols up to about 131,000: rows = 4 allows
 *    up to 131,520 columns).  The other host checks are ccm_matvec's.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current); make that first call
 *    before any stream capture.
 *  - All calls on a device share the one array and find in it whatever the
 *    previous call left; the kernels clear what must start at zero.  Calls
 *    that overlap on the GPU (for example on two unordered streams) race on
 *    the array: order them.
 *  - No cudaMalloc, cudaFree or other allocating call is made. */
#define CCM_STATIC_SCRATCH_BYTES ((1u << 20) + 4096u)
ccm_status ccm_matvec_static(const ccm_matrix* a, const ccm_matrix* x, const ccm_matrix* y,
                             ccm_stream_t stream);

/* Runtime instrumentation (no counterpart in the paper).
 * ccm_launch_count: number of kernels this library has launched in this
 * process so far (all devices, all threads).
 * ccm_profile_next: brackets the main kernel of the NEXT ccm_* call made by
 * the calling host thread with cudaEventRecord(start) before it and
 * cudaEventRecord(stop) after it, on that call's stream, so the caller can
 * time that one kernel with cudaEventElapsedTime.  `start` and `stop` are
 * cudaEvent_t handles owned by the caller; NULL, NULL cancels.  The main
 * kernel is: for ccm_pack the local pack (with a workspace; the re-code to
 * the matrix width that follows is not bracketed) or the pack pass (without
 * one), every pass of ccm_add/ccm_scale after the initialisation
 * (together: the lane pass and the general passes), k_stats for
 * ccm_measure, k_unpack, k_get, and the product kernel of
 * ccm_matvec/ccm_matmul. */
uint64_t ccm_launch_count(void);
ccm_status ccm_profile_next(void* start_event, void* stop_event);

#ifdef __cplusplus
}
#endif

#endif /* CCM_H */
