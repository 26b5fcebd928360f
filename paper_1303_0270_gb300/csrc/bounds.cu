// bounds.cu -- result-width bounds of the operations, computed on the host
// from the operand widths alone (the entries themselves live on the GPU).
//
// A b-bit field holds [0, 2^b - 1] (unsigned) or [-2^(b-1), 2^(b-1) - 1]
// (two's complement).  Each bound is Eq. 1 (with the library's signed
// reading) applied to the range of every result those operand ranges allow:
// the smallest width that holds any possible result, so an output buffer of
// ccm_words_for(rows, cols, bound) words never overflows its capacity.
#include "ccm.h"
#include "ccm_device.cuh"

namespace {

typedef __int128 i128;

struct Range {
  i128 lo, hi;
};

bool width_ok(int b) { return b >= 1 && b <= 64; }

Range field_range(int b, int sgn) {
  if (sgn) return {-((i128)1 << (b - 1)), ((i128)1 << (b - 1)) - 1};
  return {0, ((i128)1 << b) - 1};
}

int bitlen128(i128 v) {  // v >= 0
  int l = 0;
  for (; v > 0; v >>= 1) ++l;
  return l;
}

// The width rule on a range: unsigned max(1, bitlen(hi)) when lo >= 0, else
// 1 + the larger bit length of hi and -lo - 1; capped at 64 (a result beyond
// int64 is an error of the operation, not a width).
int range_width(const Range& r) {
  int b;
  if (r.lo >= 0) {
    b = bitlen128(r.hi);
    if (b < 1) b = 1;
  } else {
    const int lh = r.hi > 0 ? bitlen128(r.hi) : 0;
    const int ll = bitlen128(-r.lo - 1);
    b = 1 + (lh > ll ? lh : ll);
  }
  return b > 64 ? 64 : b;
}

// Range of sum_{j<k} a_j x_j for a_j, x_j in the ranges of the two widths:
// k times the smallest and the largest product of the range ends.  Widths
// whose product range could leave 126 bits are beyond int64 anyway.
int dot_bound(int ba, int sa, int bx, int sx, uint64_t k) {
  if (k == 0) return 1;  // every entry is an empty sum
  int lk = 0;
  for (uint64_t v = k; v; v >>= 1) ++lk;
  if (ba + bx + lk > 125) return 64;
  const Range a = field_range(ba, sa), x = field_range(bx, sx);
  const i128 p[4] = {a.lo * x.lo, a.lo * x.hi, a.hi * x.lo, a.hi * x.hi};
  i128 pmin = p[0], pmax = p[0];
  for (int i = 1; i < 4; ++i) {
    if (p[i] < pmin) pmin = p[i];
    if (p[i] > pmax) pmax = p[i];
  }
  return range_width({pmin * (i128)k, pmax * (i128)k});
}

}  // namespace

extern "C" {

int ccm_bound_add(int width_a, int signed_a, int width_b, int signed_b) {
  if (!width_ok(width_a) || !width_ok(width_b)) return CCM_E_WIDTH;
  const Range a = field_range(width_a, signed_a != 0), b = field_range(width_b, signed_b != 0);
  return range_width({a.lo + b.lo, a.hi + b.hi});
}

int ccm_bound_scale(int width_a, int signed_a, int64_t s) {
  if (!width_ok(width_a)) return CCM_E_WIDTH;
  const Range a = field_range(width_a, signed_a != 0);
  const i128 p = a.lo * (i128)s, q = a.hi * (i128)s;
  return range_width({p < q ? p : q, p < q ? q : p});
}

int ccm_bound_matvec(int width_a, int signed_a, int width_x, int signed_x, uint64_t cols) {
  if (!width_ok(width_a) || !width_ok(width_x)) return CCM_E_WIDTH;
  return dot_bound(width_a, signed_a != 0, width_x, signed_x != 0, cols);
}

int ccm_bound_matmul(int width_a, int signed_a, int width_b, int signed_b, uint64_t inner) {
  if (!width_ok(width_a) || !width_ok(width_b)) return CCM_E_WIDTH;
  return dot_bound(width_a, signed_a != 0, width_b, signed_b != 0, inner);
}

}  // extern "C"
