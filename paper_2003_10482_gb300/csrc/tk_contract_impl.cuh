// Packed contraction kernels: K[a^{m-1}] and K[a^m] (and, with a dual
// direction, K[a^{m-2}, v]) over the sorted-tuple layout of Section 5.
//
// What is computed (Section 4, eq. dual_tensor_kernel): the full sums over all
// n^m index tuples, evaluated over the stored sorted tuples.  Fix a "triangle"
// Q = (i_1..i_{m-2}) with last value b and let its rows be c = b..n-1, row c
// holding the entries (Q, c, d) for d = c..n-1 (d = c is the row head).  With
//   M'  = m! / prod_v cnt_Q(v)!,   M_f = M' / (cnt_Q(b) + 1)   (first row c = b)
//   M_c = M_f for c = b, M' otherwise;   cnt_c = cnt_Q(b)+1 for c = b, else 1
//   A_Q = prod_{q in Q} a_q,   B_{Q,l} = A_Q without one factor a_l
//   r_c = sum_{d > c} K_{Qcd} a_d,   h_c = K_{Qcc}
//   R_c = r_c + h_c a_c / (cnt_c + 1)
// the multiplicity-weighted sums reduce to
//   g_d  += K_{Qcd} (M_c/m) A_Q a_c                  for d > c   (per entry)
//   g_c  += A_Q (M_c/m) (a_c h_c + cnt_c r_c)                    (per row)
//   T    += M_c a_c R_c   (T_rest over c > b, T_first for c = b) (per row)
//   S    += A_Q T                                                (per triangle)
//   g_l  += (cnt_Q(l)/m) B_{Q,l} (l == b ? T_rest : T)  for distinct l in Q
// (For m = 2 there is one triangle, Q empty, A_Q = 1, M' = 2, no first row.)
// Replacing a by a + eps v and carrying the eps-coefficient alongside (dual
// numbers) gives d/deps K[(a+eps v)^{m-1}] = (m-1) K[a^{m-2}, v] in the same
// pass.
//
// GB300 mapping.  Every warp owns a contiguous, row-aligned range of the packed
// array and streams it through its own shared-memory ring with
// cp.async.bulk (TMA bulk copies, mbarrier completion), so each SM keeps
// ~100 KB of HBM reads in flight with a handful of instructions.  Within a
// row, lane j owns the columns d = n-1-(32k+j): the last index is counted
// from the end of the row, so every row of a triangle starts at chunk 0.  The
// per-entry scatter to g_d then accumulates in registers (acc[k]) with no
// atomics, the row dot r_c is a per-lane partial sum, and RB = 4 rows are
// processed together so that their dots are reduce-scattered across the
// warp with 6 shuffles.  Per-warp partial g lives in shared memory; blocks
// write FP64 partials that a second kernel sums in a fixed order.
#include <cuda_bf16.h>

#pragma once
#include <algorithm>

#include "tk_internal.h"

namespace tk {

// ------------------------------------------------------------------ PTX
__device__ __forceinline__ uint32_t saddr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          saddr(dst)),
      "l"(src), "r"(bytes), "r"(saddr(bar))
      : "memory");
}

// bounded wait: gives up after ~2^31 cycles (about a second) and reports
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  long long t0 = clock64();
  while (!mbar_try_wait(bar, parity)) {
    if (clock64() - t0 > (1ll << 31)) return false;
  }
  return true;
}

// ------------------------------------------------------------------ numbers
// Value with an optional derivative part (dual number a + eps a').
template <typename T, bool D>
struct Nm {
  T v, d;
};
template <typename T, bool D>
__device__ __forceinline__ Nm<T, D> mk(T v, T d) {
  Nm<T, D> r;
  r.v = v;
  r.d = D ? d : T(0);
  return r;
}
template <typename T, bool D>
__device__ __forceinline__ Nm<T, D> operator+(Nm<T, D> a, Nm<T, D> b) {
  return mk<T, D>(a.v + b.v, D ? a.d + b.d : T(0));
}
template <typename T, bool D>
__device__ __forceinline__ Nm<T, D> operator*(Nm<T, D> a, Nm<T, D> b) {
  return mk<T, D>(a.v * b.v, D ? a.v * b.d + a.d * b.v : T(0));
}
template <typename T, bool D>
__device__ __forceinline__ Nm<T, D> scale(T s, Nm<T, D> a) {
  return mk<T, D>(s * a.v, D ? s * a.d : T(0));
}
// acc += x * a  (x a plain value)
__device__ __forceinline__ float fmx(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return __fma_rn(a, b, c); }
template <typename T, bool D>
__device__ __forceinline__ void fma_acc(Nm<T, D> &acc, T x, Nm<T, D> a) {
  acc.v = fmx(x, a.v, acc.v);
  if (D) acc.d = fmx(x, a.d, acc.d);
}
template <typename T, bool D>
__device__ __forceinline__ Nm<T, D> shfl_xor(Nm<T, D> a, int mask) {
  Nm<T, D> r;
  r.v = __shfl_xor_sync(0xffffffffu, a.v, mask);
  r.d = D ? __shfl_xor_sync(0xffffffffu, a.d, mask) : T(0);
  return r;
}
template <typename T, bool D>
__device__ __forceinline__ Nm<T, D> sel(bool c, Nm<T, D> a, Nm<T, D> b) {
  return c ? a : b;
}
template <typename T, bool D>
__device__ __forceinline__ Nm<T, D> warp_sum(Nm<T, D> a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a = a + shfl_xor(a, o);
  return a;
}

template <typename ST, typename CT>
__device__ __forceinline__ CT ld_ring(const unsigned char *ring, uint32_t idx);
template <>
__device__ __forceinline__ float ld_ring<float, float>(const unsigned char *ring, uint32_t idx) {
  return reinterpret_cast<const float *>(ring)[idx];
}
template <>
__device__ __forceinline__ double ld_ring<double, double>(const unsigned char *ring, uint32_t idx) {
  return reinterpret_cast<const double *>(ring)[idx];
}
template <>
__device__ __forceinline__ float ld_ring<__nv_bfloat16, float>(const unsigned char *ring,
                                                                uint32_t idx) {
  uint32_t h = reinterpret_cast<const unsigned short *>(ring)[idx];
  return __uint_as_float(h << 16);
}

template <typename CT>
__device__ __forceinline__ CT ld_vec(const void *p, int dt, int i) {
  return dt == TK_F64 ? (CT) reinterpret_cast<const double *>(p)[i]
                      : (CT) reinterpret_cast<const float *>(p)[i];
}

// Warp-cooperative unrank (see tk_core.h): each position is located by a
// 32-way search, two rounds for n <= 1024.
static __device__ void warp_unrank(int m, int64_t n, int64_t off, int32_t *t, int lane) {
  int64_t lo = 0;
  for (int j = 0; j < m; ++j) {
    int r = m - 1 - j;
    int64_t a = lo, b = n - 1;
    while (a < b) {
      int64_t step = (b - a + 31) >> 5;
      int64_t cand = a + (int64_t)(lane + 1) * step;
      bool ok = (cand <= b) && (before(n, r, lo, cand) <= off);
      unsigned msk = __ballot_sync(0xffffffffu, ok);
      if (msk == 0) {
        b = a + step - 1;
      } else {
        int hl = 31 - __clz(msk);
        int64_t ch = a + (int64_t)(hl + 1) * step;
        a = ch;
        b = min(b, ch + step - 1);
      }
    }
    off -= before(n, r, lo, a);
    t[j] = (int32_t)a;
    lo = a;
  }
}

struct KParams {
  int m, n;
  const unsigned char *K;  // entry off_lo
  int64_t off_lo, off_hi;
  int64_t bytes;           // (off_hi - off_lo) * ES
  const void *alpha;
  const void *v;
  int vec_dtype;
  double *part;
  int *status;
  int warps;
  int slot_log2, ns_log2;
  int vec_bytes;   // bytes of the staged alpha (and v) region, 128-aligned
  int warp_bytes;  // bytes of one warp's region
};

constexpr int kRB = 4;  // rows per batch

// Threads per block the register budget allows: a base of ~64 registers plus
// the per-lane column state (acc[] and alpha[], doubled for dual numbers and
// for FP64).  Above 120 estimated registers the block is capped at 256 threads.
__host__ __device__ constexpr int max_threads_est(int ct_bytes, bool dual, int nc) {
  return (64 + (dual ? 2 : 1) * (ct_bytes / 4) * 2 * nc <= 120 && !(dual && ct_bytes == 8)) ? 512 : 256;
}
template <typename CT, bool D, int NC>
constexpr int max_threads() {
  return max_threads_est((int)sizeof(CT), D, NC);
}

template <typename ST, typename CT, bool D, int NC>
__global__ void __launch_bounds__(max_threads<CT, D, NC>(), 1) contract_kernel(KParams p) {
  using N = Nm<CT, D>;
  constexpr int ES = sizeof(ST);
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int m = p.m;
  const int n = p.n;

  CT *a_s = reinterpret_cast<CT *>(smem);
  CT *v_s = a_s + n;
  unsigned char *wb = smem + p.vec_bytes + (size_t)wid * p.warp_bytes;
  uint64_t *bar = reinterpret_cast<uint64_t *>(wb);
  unsigned char *ring = wb + 128;
  const uint32_t SLOT = 1u << p.slot_log2;
  const uint32_t NS = 1u << p.ns_log2;
  const uint32_t RING = SLOT * NS;
  CT *g_v = reinterpret_cast<CT *>(ring + RING);
  CT *g_d = g_v + n;

  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a_s[i] = ld_vec<CT>(p.alpha, p.vec_dtype, i);
    if (D) v_s[i] = ld_vec<CT>(p.v, p.vec_dtype, i);
  }
  for (int i = lane; i < n; i += 32) {
    g_v[i] = CT(0);
    if (D) g_d[i] = CT(0);
  }
  if (lane == 0) {
    for (uint32_t s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
    fence_barrier_init();
  }
  __syncthreads();

  auto alpha_at = [&](int i) -> N { return mk<CT, D>(a_s[i], D ? v_s[i] : CT(0)); };

  // ------------------------------------------------------------ warp range
  const int64_t W = (int64_t)gridDim.x * p.warps;
  const int64_t w = (int64_t)blockIdx.x * p.warps + wid;
  const int64_t total = p.off_hi - p.off_lo;
  int64_t o0 = p.off_lo + (w * total) / W;
  int64_t o1 = p.off_lo + ((w + 1) * total) / W;

  int32_t Q[kMaxOrder];
  int32_t tt[kMaxOrder];
  int c = 0;
  int64_t p_row = p.off_hi, p_end = p.off_hi;
  bool have = false;
  if (o0 < p.off_hi) {
    warp_unrank(m, n, o0, tt, lane);
    c = tt[m - 2];
    int dl = tt[m - 1];
    p_row = (dl == c) ? o0 : o0 + (n - dl);
    if (dl != c) c += 1;
    for (int j = 0; j < m - 2; ++j) Q[j] = tt[j];
    if (c == n) {
      // the next row starts a new triangle
      if (m > 2 && next_sorted(m - 2, n, Q)) c = Q[m - 3];
      else p_row = p.off_hi;
    }
    if (o1 < p.off_hi) {
      warp_unrank(m, n, o1, tt, lane);
      int c1 = tt[m - 2], d1 = tt[m - 1];
      p_end = (d1 == c1) ? o1 : o1 + (n - d1);
    }
    have = p_row < p_end;
  }

  // ------------------------------------------------------------ ring
  const int64_t rel0 = (p_row - p.off_lo) * ES;
  const int64_t rel1 = (p_end - p.off_lo) * ES;
  const int64_t sbase = rel0 & ~int64_t(15);
  const int64_t tail_lo = p.bytes & ~int64_t(15);
  const int64_t bulk_lim = min((rel1 + 15) & ~int64_t(15), tail_lo);
  const uint32_t emask = RING / ES - 1;
  const uint32_t ebase = (uint32_t)(p.off_lo + sbase / ES);
  int64_t s_issued = 0, s_ready = 0;
  bool failed = false;

  auto issue = [&](int64_t s) {
    const int64_t lo = sbase + (s << p.slot_log2);
    if (lo >= bulk_lim) return;
    const int64_t rem = bulk_lim - lo;
    const uint32_t sz = rem < (int64_t)SLOT ? (uint32_t)rem : SLOT;
    if (lane == 0) {
      uint64_t *b = &bar[s & (NS - 1)];
      fence_proxy_async();
      mbar_expect_tx(b, sz);
      bulk_g2s(ring + (uint32_t)((s & (NS - 1)) << p.slot_log2), p.K + lo, sz, b);
    }
  };
  auto wait_slot = [&](int64_t s) {
    const int64_t lo = sbase + (s << p.slot_log2);
    if (lo < bulk_lim) {
      bool ok = mbar_wait_bounded(&bar[s & (NS - 1)], (uint32_t)((s >> p.ns_log2) & 1));
      if (!__all_sync(0xffffffffu, ok)) {
        if (lane == 0) {
          atomicExch(&reinterpret_cast<WsHeader *>(p.status)->status, TK_ETIMEOUT);
          reinterpret_cast<WsHeader *>(p.status)->where = 1;
        }
        failed = true;
      }
    }
    // bytes past the last 16-byte boundary of the array are not reachable by
    // the bulk engine: copy them with plain loads
    if (rel1 > tail_lo && tail_lo >= lo && tail_lo < lo + (int64_t)SLOT) {
      const int64_t nb = rel1 - tail_lo;
      if (lane < nb) {
        uint32_t ri = (uint32_t)((tail_lo + lane - sbase) & (RING - 1));
        ring[ri] = p.K[tail_lo + lane];
      }
      __syncwarp();
    }
  };

  if (have) {
    for (int64_t s = 0; s < (int64_t)NS; ++s) issue(s);
    s_issued = NS;
  }

  // ------------------------------------------------------------ accumulators
  N acc[NC];
  N ar[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    acc[k] = mk<CT, D>(CT(0), CT(0));
    int e = 32 * k + lane;
    ar[k] = (e < n) ? alpha_at(n - 1 - e) : mk<CT, D>(CT(0), CT(0));
  }
  double S_v = 0.0, S_d = 0.0;

  // triangle state
  int b = -1;           // last value of Q (-1: m = 2, no first row)
  int kb = 0;           // multiplicity of b in Q
  CT Mprime = CT(2), Mf = CT(2);
  N AQ = mk<CT, D>(CT(1), CT(0));
  N cA = AQ, cAf = AQ;
  N Trest = mk<CT, D>(CT(0), CT(0)), Tfirst = Trest;
  const CT inv_m = CT(1) / CT(m);

  auto setup_triangle = [&]() {
    AQ = mk<CT, D>(CT(1), CT(0));
    double fact_m = 1.0;
    for (int i = 2; i <= m; ++i) fact_m *= i;
    double den = 1.0;
    int run = 0;
    for (int j = 0; j < m - 2; ++j) {
      AQ = AQ * alpha_at(Q[j]);
      run = (j > 0 && Q[j] == Q[j - 1]) ? run + 1 : 1;
      den *= run;  // accumulates prod_v cnt_Q(v)!
    }
    if (m > 2) {
      b = Q[m - 3];
      kb = 0;
      for (int j = 0; j < m - 2; ++j) kb += (Q[j] == b);
    } else {
      b = -1;
      kb = 0;
    }
    Mprime = CT(fact_m / den);
    Mf = Mprime / CT(kb + 1);
    cA = scale(Mprime * inv_m, AQ);
    cAf = scale(Mf * inv_m, AQ);
  };

  auto flush_triangle = [&]() {
    __syncwarp();
    N Tr = warp_sum(Trest);
    N Tf = warp_sum(Tfirst);
    N T = Tr + Tf;
    N SQ = AQ * T;
    S_v += (double)SQ.v;
    if (D) S_d += (double)SQ.d;
    if (lane < m - 2 && (lane == 0 || Q[lane] != Q[lane - 1])) {
      const int l = Q[lane];
      int cnt = 0;
      N B = mk<CT, D>(CT(1), CT(0));
      for (int j = 0; j < m - 2; ++j) {
        cnt += (Q[j] == l);
        if (j != lane) B = B * alpha_at(Q[j]);
      }
      N add = scale(CT(cnt) * inv_m, B * ((l == b) ? Tr : T));
      g_v[l] += add.v;
      if (D) g_d[l] += add.d;
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      int e = 32 * k + lane;
      if (e < n) {
        g_v[n - 1 - e] += acc[k].v;
        if (D) g_d[n - 1 - e] += acc[k].d;
      }
      acc[k] = mk<CT, D>(CT(0), CT(0));
    }
    __syncwarp();
    Trest = mk<CT, D>(CT(0), CT(0));
    Tfirst = Trest;
  };

  if (have) setup_triangle();
  int64_t pos = p_row;
  bool open = have;  // a triangle is open (has unflushed rows)

  while (pos < p_end && !failed) {
    // ---------------------------------------------------- batch of rows
    int nb = 0;
    int64_t pi[kRB];
    int sl[kRB];
    int64_t q = pos;
#pragma unroll
    for (int i = 0; i < kRB; ++i) {
      pi[i] = q;
      bool ok = (c + i < n) && (q < p_end);
      sl[i] = ok ? n - 1 - c - i : 0;
      if (ok) {
        nb = i + 1;
        q += n - c - i;
      }
    }
    const int64_t p_next = q;
    const int64_t s_hi = ((p_next - p.off_lo) * ES - 1 - sbase) >> p.slot_log2;
    if (s_hi >= s_issued) {  // batch larger than the ring: configuration error
      if (lane == 0) {
        atomicExch(&reinterpret_cast<WsHeader *>(p.status)->status, TK_EINVAL);
        reinterpret_cast<WsHeader *>(p.status)->where = 2;
      }
      failed = true;
      break;
    }
    while (s_ready <= s_hi) wait_slot(s_ready++);
    if (failed) break;

    N cf[kRB];
    uint32_t zl[kRB];
#pragma unroll
    for (int i = 0; i < kRB; ++i) {
      const int ci = min(c + i, n - 1);
      cf[i] = ((ci == b) ? cAf : cA) * alpha_at(ci);
      zl[i] = (uint32_t)pi[i] + (uint32_t)sl[i] - (uint32_t)lane - ebase;
    }
    N dot[kRB];
#pragma unroll
    for (int i = 0; i < kRB; ++i) dot[i] = mk<CT, D>(CT(0), CT(0));

#pragma unroll
    for (int k = 0; k < NC; ++k) {
      if (32 * k >= sl[0]) break;
      const int e = 32 * k + lane;
#pragma unroll
      for (int i = 0; i < kRB; ++i) {
        if (e < sl[i]) {
          const CT x = ld_ring<ST, CT>(ring, (zl[i] - 32u * k) & emask);
          fma_acc(acc[k], x, cf[i]);
          fma_acc(dot[i], x, ar[k]);
        }
      }
    }

    // reduce-scatter the 4 row dots: row i ends up on lanes 8i..8i+7
    {
      const bool h16 = lane & 16;
      N k0 = sel(h16, dot[2], dot[0]), k1 = sel(h16, dot[3], dot[1]);
      N s0 = sel(h16, dot[0], dot[2]), s1 = sel(h16, dot[1], dot[3]);
      k0 = k0 + shfl_xor(s0, 16);
      k1 = k1 + shfl_xor(s1, 16);
      const bool h8 = lane & 8;
      N kk = sel(h8, k1, k0), ss = sel(h8, k0, k1);
      kk = kk + shfl_xor(ss, 8);
      kk = kk + shfl_xor(kk, 4);
      kk = kk + shfl_xor(kk, 2);
      kk = kk + shfl_xor(kk, 1);
      const int i = lane >> 3;
      if ((lane & 7) == 0 && i < nb) {
        const int ci = c + i;
        const N ac = alpha_at(ci);
        const CT h = ld_ring<ST, CT>(ring, ((uint32_t)pi[i] - ebase) & emask);
        const bool first = (ci == b);
        const CT cnt = first ? CT(kb + 1) : CT(1);
        const N Rf = kk + scale(h / (cnt + CT(1)), ac);
        const N gadd = (first ? cAf : cA) * (scale(h, ac) + scale(cnt, kk));
        g_v[ci] += gadd.v;
        if (D) g_d[ci] += gadd.d;
        const N tadd = scale(first ? Mf : Mprime, ac * Rf);
        if (first) Tfirst = Tfirst + tadd; else Trest = Trest + tadd;
      }
    }

    // ---------------------------------------------------- advance
    c += nb;
    pos = p_next;
    if (c == n) {
      flush_triangle();
      open = false;
      if (pos < p_end) {
        if (m > 2 && next_sorted(m - 2, n, Q)) {
          c = Q[m - 3];
          setup_triangle();
          open = true;
        } else {
          break;
        }
      }
    }
    __syncwarp();
    const int64_t s_free = ((pos - p.off_lo) * ES - sbase) >> p.slot_log2;
    while (s_issued < s_free + (int64_t)NS) issue(s_issued++);
  }
  if (open) flush_triangle();
  // drain bulk copies still in flight before the block can exit
  while (s_ready < s_issued) {
    const int64_t lo = sbase + (s_ready << p.slot_log2);
    if (lo < bulk_lim) mbar_wait_bounded(&bar[s_ready & (NS - 1)], (uint32_t)((s_ready >> p.ns_log2) & 1));
    ++s_ready;
  }
  __syncwarp();

  // ------------------------------------------------------------ block reduce
  __shared__ double s_S[2][32];
  if (lane == 0) {
    s_S[0][wid] = S_v;
    s_S[1][wid] = S_d;
  }
  __syncthreads();
  const int ld = n + 2;
  double *out = p.part + (size_t)blockIdx.x * 2 * ld;
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    double sv = 0.0, sd = 0.0;
    for (int ww = 0; ww < p.warps; ++ww) {
      const CT *gw = reinterpret_cast<const CT *>(smem + p.vec_bytes + (size_t)ww * p.warp_bytes + 128 + RING);
      sv += (double)gw[l];
      if (D) sd += (double)gw[n + l];
    }
    out[l] = sv;
    out[ld + l] = sd;
  }
  if (threadIdx.x == 0) {
    double sv = 0.0, sd = 0.0;
    for (int ww = 0; ww < p.warps; ++ww) {
      sv += s_S[0][ww];
      sd += s_S[1][ww];
    }
    out[n] = sv;
    out[ld + n] = sd;
  }
}

// ------------------------------------------------------------------ launch
template <typename ST, typename CT, bool D, int NC>
inline int launch_nc(const KParams &kp, int grid, int threads, size_t smem, cudaStream_t st) {
  auto kern = contract_kernel<ST, CT, D, NC>;
  if (threads > max_threads<CT, D, NC>())
    return fail(TK_EINVAL, "contract: %d threads exceed the kernel's bound", threads);
  TK_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, threads, smem, st>>>(kp);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

template <typename ST, typename CT, bool D>
inline int launch_typed(const KParams &kp, int nc, int grid, int threads, size_t smem, cudaStream_t st) {
  switch (nc) {
    case 1: return launch_nc<ST, CT, D, 1>(kp, grid, threads, smem, st);
    case 2: return launch_nc<ST, CT, D, 2>(kp, grid, threads, smem, st);
    case 4: return launch_nc<ST, CT, D, 4>(kp, grid, threads, smem, st);
    case 8: return launch_nc<ST, CT, D, 8>(kp, grid, threads, smem, st);
    case 12: return launch_nc<ST, CT, D, 12>(kp, grid, threads, smem, st);
    case 16: return launch_nc<ST, CT, D, 16>(kp, grid, threads, smem, st);
    case 20: return launch_nc<ST, CT, D, 20>(kp, grid, threads, smem, st);
    case 24: return launch_nc<ST, CT, D, 24>(kp, grid, threads, smem, st);
    case 32: return launch_nc<ST, CT, D, 32>(kp, grid, threads, smem, st);
  }
  return fail(TK_EUNSUPPORTED, "contract: n=%d exceeds %d", kp.n, TK_MAX_POINTS);
}

}  // namespace tk
