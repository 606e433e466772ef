// Index and epilogue arithmetic of the tensor-core batched contraction
// (tk_batched_tc.cu), shared by the device kernel and host-side checks.
//
// Per triangle Q (prefix i_1..i_{m-2}, last value b, kb = cnt_Q(b),
// M' = m!/prod_v cnt_Q(v)!, A_Q = prod_Q a) let S_Q be the full symmetric
// (n-b) x (n-b) matrix of its entries, S_Q[c][d] = K_{Q,min(c,d),max(c,d)},
// and f_d = 1/(kb+1) for d = b, 1 otherwise.  The tensor cores give, for every
// vector, the weighted row dots
//   Rf_c = sum_{d >= b} S_Q[c][d] f_d a_d            (c >= b).
// The multiplicity-weighted sums of the contraction (the same sums as the
// single-vector kernel's triangle/row decomposition) then read
//   g_c  += A_Q (M'/m) Rf_c                                   (c >= b)
//   r_b   = Rf_b - h_b a_b/(kb+1)                (h_b = K_{Qbb}; row-b dot over d > b)
//   P     = sum_{c > b} a_c Rf_c
//   T_rest  = (M'/2) (P - a_b r_b/(kb+1))
//   T_first = (M'/(kb+1)) a_b (r_b + h_b a_b/(kb+2))
//   T     = T_rest + T_first,   S += A_Q T
//   g_l  += (cnt_Q(l)/m) B_{Q,l} (l == b ? T_rest : T)     for distinct l in Q
// (B_{Q,l} = A_Q without one factor a_l).  For m = 2 there is one triangle,
// Q empty, b = -1, A_Q = 1, M' = 2, no first row: T = T_rest = P over all rows.
#pragma once
#include <stdint.h>

namespace tk {
namespace tc {

constexpr int kRowsPerJob = 96;  // rows of S_Q per MMA (N of the instruction, a multiple of 16)

// Offset, relative to the triangle's first entry (b, b), of entry (r, d),
// bb <= r <= d < n (bb = max(b, 0)): row r starts after the rows bb..r-1.
__host__ __device__ inline int64_t tri_entry(int n, int bb, int r, int d) {
  return (int64_t)(r - bb) * (2 * n - bb - r + 1) / 2 + (d - r);
}

// Offset of S_Q[c][d] within the triangle, or -1 when (c, d) lies outside it.
__host__ __device__ inline int64_t sym_entry(int n, int b, int c, int d) {
  const int bb = b < 0 ? 0 : b;
  if (c < bb || d < bb || c >= n || d >= n) return -1;
  return c <= d ? tri_entry(n, bb, c, d) : tri_entry(n, bb, d, c);
}

// The per-triangle finish of the epilogue for one vector (see above): from
// P, Rf_b, h_b, a_b returns T and T_rest.
template <typename CT>
__host__ __device__ inline void finish_triangle(int b, int kb, CT mprime, CT P, CT Rfb, CT hb, CT ab, CT *T,
                                                CT *T_rest) {
  if (b < 0) {
    *T_rest = mprime / CT(2) * P;
    *T = *T_rest;
    return;
  }
  const CT k1 = CT(1) / CT(kb + 1), k2 = CT(1) / CT(kb + 2);
  const CT rb = Rfb - hb * ab * k1;
  *T_rest = mprime / CT(2) * (P - ab * rb * k1);
  *T = *T_rest + mprime * k1 * ab * (rb + hb * ab * k2);
}

}  // namespace tc
}  // namespace tk
