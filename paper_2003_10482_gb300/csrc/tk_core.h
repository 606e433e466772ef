// Combinatorics of the packed symmetric layout, shared by host and device code.
//
// The stored entries of an order-m symmetric tensor over n points are the
// sorted tuples i_1 <= ... <= i_m in lexicographic order (the nested loops of
// Section 5 of the thesis).  Counting arguments:
//
//   multiset(k, r)  = number of sorted r-tuples over k values = C(k+r-1, r)
//   N               = multiset(n, m)
//   before(j, lo, v)= number of sorted tuples that agree with a prefix up to
//                     position j-1 (whose last value is lo) and have a value
//                     in [lo, v) at position j:
//                     sum_{u=lo}^{v-1} multiset(n-u, r) with r = m-1-j,
//                     = multiset(n-lo, r+1) - multiset(n-v, r+1)  (hockey stick)
//   rank(t)         = sum_j before(j, t_{j-1}, t_j),  t_{-1} = 0.
//
// This is the combinatorial number system written for multisets; for m = 2,
// 3, 4 it equals the thesis's v_2d, v_3d, v_4d (eqs. index_2d, v3d, v4d).
#pragma once
#include <stdint.h>

#ifdef __CUDACC__
#define TK_HD __host__ __device__ __forceinline__
#else
#define TK_HD inline
#endif

namespace tk {

constexpr int kMaxOrder = 8;

// x / d for x known to be a multiple of d, 1 <= d <= 16, x < 2^64: strip the
// power of two of d by a shift, then multiply by the inverse of the odd part
// modulo 2^64 (exact division needs no 64-bit divide instruction).
TK_HD uint64_t exact_div_small(uint64_t x, int d) {
  int s = 0;
  while ((d & 1) == 0) {
    d >>= 1;
    ++s;
  }
  x >>= s;
  uint64_t inv;
  switch (d) {
    case 3: inv = 0xAAAAAAAAAAAAAAABull; break;
    case 5: inv = 0xCCCCCCCCCCCCCCCDull; break;
    case 7: inv = 0x6DB6DB6DB6DB6DB7ull; break;
    case 9: inv = 0x8E38E38E38E38E39ull; break;
    case 11: inv = 0x2E8BA2E8BA2E8BA3ull; break;
    case 13: inv = 0x4EC4EC4EC4EC4EC5ull; break;
    case 15: inv = 0xEEEEEEEEEEEEEEEFull; break;
    default: inv = 1ull; break;
  }
  return x * inv;
}

// C(a, k) for 0 <= k <= 16.  Each partial product C(a, i) * (a - i) is a
// multiple of i + 1; callers keep sizes such that it stays below 2^63.
TK_HD int64_t binom(int64_t a, int k) {
  if (k < 0 || a < k) return 0;
  uint64_t c = 1;
  for (int i = 0; i < k; ++i) c = exact_div_small(c * (uint64_t)(a - i), i + 1);
  return (int64_t)c;
}

TK_HD int64_t multiset(int64_t k, int r) {
  if (r == 0) return 1;
  if (k <= 0) return 0;
  return binom(k + r - 1, r);
}

// Number of sorted tuples whose position j (r = m-1-j values follow it) holds
// a value in [lo, v), given the same prefix before j.
TK_HD int64_t before(int64_t n, int r, int64_t lo, int64_t v) {
  return multiset(n - lo, r + 1) - multiset(n - v, r + 1);
}

TK_HD int64_t rank(int m, int64_t n, const int32_t *t) {
  int64_t off = 0, lo = 0;
  for (int j = 0; j < m; ++j) {
    off += before(n, m - 1 - j, lo, t[j]);
    lo = t[j];
  }
  return off;
}

// Sequential unrank (host and tests): at each position, binary-search the
// largest value whose preceding block still lies at or before `off`.
TK_HD void unrank(int m, int64_t n, int64_t off, int32_t *t) {
  int64_t lo = 0;
  for (int j = 0; j < m; ++j) {
    int r = m - 1 - j;
    int64_t a = lo, b = n - 1;  // answer in [a, b]
    while (a < b) {
      int64_t mid = a + (b - a + 1) / 2;
      if (before(n, r, lo, mid) <= off) a = mid; else b = mid - 1;
    }
    off -= before(n, r, lo, a);
    t[j] = (int32_t)a;
    lo = a;
  }
}

// Offset of the first entry of row t (i_m = i_{m-1}) -- i.e. rank with the
// last index replaced by the second-to-last.
TK_HD int64_t row_start(int m, int64_t n, const int32_t *t) {
  int64_t off = 0, lo = 0;
  for (int j = 0; j < m - 1; ++j) {
    off += before(n, m - 1 - j, lo, t[j]);
    lo = t[j];
  }
  return off;
}

// Advance the (len)-tuple q of sorted values in [0, n) to its lexicographic
// successor; returns false after the last tuple.
TK_HD bool next_sorted(int len, int64_t n, int32_t *q) {
  int j = len - 1;
  while (j >= 0 && q[j] == n - 1) --j;
  if (j < 0) return false;
  q[j] += 1;
  for (int i = j + 1; i < len; ++i) q[i] = q[j];
  return true;
}

TK_HD int dtype_size(int dt) { return dt == 0 ? 8 : (dt == 1 ? 4 : 2); }

}  // namespace tk
