/*
 * ccm_oracle.c -- plain, slow CPU oracle for the Supreme Minimum (SM)
 * fixed-width compression of integer matrices and for linear algebra on it.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the bench's CPU-baseline leg and the smoke
 * check do.  It shares no code, header or table with the CUDA path.
 *
 * Everything here follows the plain definitions, one bit or one element at a
 * time, in the order the paper states them:
 *
 *  - bit length of a non-negative integer (Table 1) and the SM width rule,
 *    Eq. 1: b = 1 when sup M is 0 or 1, else floor(log2 sup M) + 1, computed
 *    by counting bits, never by a floating-point logarithm;
 *  - signed reading (the paper only treats non-negative entries): when some
 *    entry is negative, fields are two's complement and b is one more than the
 *    largest bit length of a (a >= 0) or -a - 1 (a < 0), the smallest b whose
 *    range [-2^(b-1), 2^(b-1) - 1] holds every entry; on non-negative data the
 *    rule is exactly Eq. 1;
 *  - SM layout (Methods, "Method 1: The Supreme Minimum", Eq. 3 and the
 *    step-by-step example after it): the matrix is unravelled row-major and
 *    entry e occupies bits [e*b, (e+1)*b) of one LSB-first bit stream (the
 *    paper fills each bitstring from its least significant end); a field that
 *    does not fit in what is left of a word straddles into the next one, low
 *    bits first.  The stream is cut into
 *    32-bit little-endian words, which is byte-for-byte the paper's 64-bit
 *    bitstrings on a little-endian machine;
 *  - the word count: ceil(n*b/32) data words, zero-padded to a multiple of 4
 *    words (the paper's floor(n*b/64)+1 over-allocates when 64 divides n*b);
 *  - operations on the compressed form are defined as the same operation on
 *    the uncompressed integers (Introduction: the compressed form is meant to
 *    support the same mathematics as the original), carried out here on
 *    unpacked int64 with 128-bit accumulation and an explicit int64 overflow
 *    check.  The result is re-packed with the width rule above.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_OVERFLOW (-4)
#define ORACLE_RANGE (-6)

/* Number of binary digits of v (Table 1: 900 -> 10, 256 -> 9, 1 -> 1); 0 -> 0. */
int ccmo_bitlen_u64(uint64_t v) {
  int len = 0;
  while (v != 0) {
    ++len;
    v >>= 1;
  }
  return len;
}

/* Eq. 1 extended to signed data.  Writes the sign mode to *is_signed. */
int ccmo_width(const int64_t* a, size_t n, int* is_signed) {
  int any_negative = 0;
  for (size_t e = 0; e < n; ++e)
    if (a[e] < 0) any_negative = 1;
  int b = 0;
  if (!any_negative) {
    /* sup M by a plain maximum, then its bit length (Eq. 1). */
    int64_t sup = 0;
    for (size_t e = 0; e < n; ++e)
      if (a[e] > sup) sup = a[e];
    b = (sup <= 1) ? 1 : ccmo_bitlen_u64((uint64_t)sup);
  } else {
    for (size_t e = 0; e < n; ++e) {
      uint64_t magnitude = (a[e] >= 0) ? (uint64_t)a[e] : (uint64_t)(-(a[e] + 1));
      int len = ccmo_bitlen_u64(magnitude) + 1;
      if (len > b) b = len;
    }
  }
  *is_signed = any_negative;
  return b;
}

size_t ccmo_words_for(uint64_t n, int width) {
  uint64_t bits = n * (uint64_t)width;
  uint64_t data = (bits + 31) / 32;
  return (size_t)((data + 3) / 4 * 4);
}

/* SM pack: one bit at a time into the LSB-first stream. */
void ccmo_pack(const int64_t* a, size_t n, int width, uint32_t* words, size_t nwords) {
  memset(words, 0, nwords * sizeof(uint32_t));
  for (size_t e = 0; e < n; ++e) {
    uint64_t pattern = (uint64_t)a[e]; /* two's complement bits of the entry */
    for (int k = 0; k < width; ++k) {
      uint64_t pos = (uint64_t)e * (uint64_t)width + (uint64_t)k;
      uint32_t bit = (uint32_t)((pattern >> k) & 1u);
      words[pos / 32] |= bit << (pos % 32);
    }
  }
}

/* Read field e back, one bit at a time, and extend it to int64. */
int64_t ccmo_field(const uint32_t* words, uint64_t e, int width, int is_signed) {
  uint64_t value = 0;
  for (int k = 0; k < width; ++k) {
    uint64_t pos = e * (uint64_t)width + (uint64_t)k;
    uint64_t bit = (words[pos / 32] >> (pos % 32)) & 1u;
    value |= bit << k;
  }
  if (is_signed && width < 64 && ((value >> (width - 1)) & 1u)) {
    /* two's complement: subtract 2^width */
    value |= ~(uint64_t)0 << width;
  }
  return (int64_t)value;
}

void ccmo_unpack(const uint32_t* words, size_t n, int width, int is_signed, int64_t* out) {
  for (size_t e = 0; e < n; ++e) out[e] = ccmo_field(words, e, width, is_signed);
}

/* Element access by (i, j) on the row-major stream. */
int ccmo_get(const uint32_t* words, uint64_t rows, uint64_t cols, int width, int is_signed,
             uint64_t i, uint64_t j, int64_t* out) {
  if (i >= rows || j >= cols) return ORACLE_RANGE;
  *out = ccmo_field(words, i * cols + j, width, is_signed);
  return ORACLE_OK;
}

static int fits_i64(__int128 v) {
  return v >= -((__int128)1 << 63) && v <= (((__int128)1 << 63) - 1);
}

int ccmo_add(const int64_t* a, const int64_t* b, size_t n, int64_t* c) {
  int status = ORACLE_OK;
  for (size_t e = 0; e < n; ++e) {
    __int128 s = (__int128)a[e] + (__int128)b[e];
    if (!fits_i64(s)) status = ORACLE_OVERFLOW;
    c[e] = (int64_t)s;
  }
  return status;
}

int ccmo_scale(const int64_t* a, size_t n, int64_t s, int64_t* c) {
  int status = ORACLE_OK;
  for (size_t e = 0; e < n; ++e) {
    __int128 p = (__int128)a[e] * (__int128)s;
    if (!fits_i64(p)) status = ORACLE_OVERFLOW;
    c[e] = (int64_t)p;
  }
  return status;
}

/* y_i = sum_j a_ij x_j for the listed rows (all rows when row_list is NULL). */
int ccmo_matvec_rows(const int64_t* a, uint64_t m, uint64_t n, const int64_t* x,
                     const uint64_t* row_list, size_t nrows_listed, int64_t* y) {
  int status = ORACLE_OK;
  size_t count = row_list ? nrows_listed : (size_t)m;
  for (size_t r = 0; r < count; ++r) {
    uint64_t i = row_list ? row_list[r] : r;
    __int128 acc = 0;
    for (uint64_t j = 0; j < n; ++j) acc += (__int128)a[i * n + j] * (__int128)x[j];
    if (!fits_i64(acc)) status = ORACLE_OVERFLOW;
    y[r] = (int64_t)acc;
  }
  return status;
}

/* C = A (m x k) times B (k x n), rows of C listed in row_list (all when NULL).
 * Plain triple loop, i-l-j order so that B is read row-wise; 128-bit sums. */
int ccmo_matmul_rows(const int64_t* a, const int64_t* b, uint64_t m, uint64_t k, uint64_t n,
                     const uint64_t* row_list, size_t nrows_listed, int64_t* c) {
  int status = ORACLE_OK;
  __int128* work = (__int128*)malloc((n ? n : 1) * sizeof(__int128));
  if (!work) return -1;
  size_t count = row_list ? nrows_listed : (size_t)m;
  for (size_t r = 0; r < count; ++r) {
    uint64_t i = row_list ? row_list[r] : r;
    for (uint64_t j = 0; j < n; ++j) work[j] = 0;
    for (uint64_t l = 0; l < k; ++l) {
      __int128 ail = a[i * k + l];
      const int64_t* brow = b + l * n;
      for (uint64_t j = 0; j < n; ++j) work[j] += ail * (__int128)brow[j];
    }
    for (uint64_t j = 0; j < n; ++j) {
      if (!fits_i64(work[j])) status = ORACLE_OVERFLOW;
      c[r * n + j] = (int64_t)work[j];
    }
  }
  free(work);
  return status;
}

/* ---------------------------------------------------------------------------
 * VLB, Method 2 (Methods, "Method 2: Variable Length Blocks", Eq. 9-13):
 * every entry is written as a fixed k-bit prefix holding its bit length L,
 * followed by the entry itself in exactly L bits, both LSB-first into the
 * same stream as SM uses.  k is the bit length of the largest bit length
 * (1023 -> 10 -> k = 4).  The bit length of 0 is taken as 1 (Eq. 1).
 * Non-negative entries only, as in the paper.
 * ------------------------------------------------------------------------- */
static int vlb_len(int64_t v) {
  int len = ccmo_bitlen_u64((uint64_t)v);
  return len ? len : 1;
}

/* k, or -1 when an entry is negative. */
int ccmo_vlb_prefix_width(const int64_t* a, size_t n) {
  int lmax = 1;
  for (size_t e = 0; e < n; ++e) {
    if (a[e] < 0) return -1;
    int len = vlb_len(a[e]);
    if (len > lmax) lmax = len;
  }
  return ccmo_bitlen_u64((uint64_t)lmax);
}

uint64_t ccmo_vlb_bits(const int64_t* a, size_t n, int k) {
  uint64_t bits = 0;
  for (size_t e = 0; e < n; ++e) bits += (uint64_t)k + (uint64_t)vlb_len(a[e]);
  return bits;
}

static void put_bit(uint32_t* words, uint64_t pos, uint32_t bit) {
  words[pos / 32] |= bit << (pos % 32);
}

static uint32_t get_bit(const uint32_t* words, uint64_t pos) {
  return (words[pos / 32] >> (pos % 32)) & 1u;
}

/* Writes the stream one bit at a time; returns the number of bits. */
uint64_t ccmo_vlb_pack(const int64_t* a, size_t n, int k, uint32_t* words, size_t nwords) {
  memset(words, 0, nwords * sizeof(uint32_t));
  uint64_t pos = 0;
  for (size_t e = 0; e < n; ++e) {
    int len = vlb_len(a[e]);
    for (int i = 0; i < k; ++i) put_bit(words, pos++, (uint32_t)((len >> i) & 1));
    for (int i = 0; i < len; ++i) put_bit(words, pos++, (uint32_t)(((uint64_t)a[e] >> i) & 1u));
  }
  return pos;
}

/* Reads n entries back in order (each prefix tells how long the entry is). */
void ccmo_vlb_unpack(const uint32_t* words, size_t n, int k, int64_t* out) {
  uint64_t pos = 0;
  for (size_t e = 0; e < n; ++e) {
    int len = 0;
    for (int i = 0; i < k; ++i) len |= (int)get_bit(words, pos++) << i;
    uint64_t v = 0;
    for (int i = 0; i < len; ++i) v |= (uint64_t)get_bit(words, pos++) << i;
    out[e] = (int64_t)v;
  }
}
