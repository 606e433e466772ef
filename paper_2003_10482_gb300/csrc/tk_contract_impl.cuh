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
// GB300 mapping.  The host cuts the packed range into row-aligned pieces
// (16 per warp), balanced by cost (entries + a weight per row + a weight per
// triangle, tk_contract_plan); warp w takes pieces w, w+W, ... (or the next
// free one from a shared ticket).  Each warp walks its rows in blocks of at
// most 32 consecutive rows of one triangle whose entries fit its staging
// buffer; a block that holds a whole triangle also takes the whole triangles
// of at most 32 rows that follow it while they fit (n <= 256: the many small
// triangles of high orders then share one copy and one wait).  Every block is
// fetched by one cp.async.bulk copy (TMA bulk engine,
// mbarrier completion) into one of NBUF linear shared-memory buffers, so
// NBUF-1 blocks are always in flight while the warp computes on the current
// one.  The buffers take all the shared memory the 16 warps leave free.
// Within a row, lane j owns the columns d = n-1-(32k+j): the last index is
// counted from the end of the row, so every row of a triangle starts at chunk
// 0 and the per-entry scatter to g_d accumulates in registers (acc[k]) with no
// atomics.  Rows go four at a time; the loads of each 32-column chunk are
// issued one step ahead of its multiply-adds.  The four partial row dots of a
// quad are summed by a butterfly of shuffles that leaves row i's dot on lane
// i, where the per-row epilogue runs (all rows of a block in parallel).
// Per-warp partial g lives in shared memory; blocks write FP64 partials that
// the last block to finish sums in a fixed order.
#pragma once
#include <cuda_bf16.h>

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
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(bar)) : "memory");
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
// The column accumulators of g: the dual pass returns only the derivative
// part (the Hessian-vector product), so its value part is not accumulated.
template <typename T, bool D>
__device__ __forceinline__ void fma_col(Nm<T, D> &acc, T x, Nm<T, D> a) {
  if (D) acc.d = fmx(x, a.d, acc.d);
  else acc.v = fmx(x, a.v, acc.v);
}
template <typename T, bool D>
__device__ __forceinline__ Nm<T, D> shfl_xor(Nm<T, D> a, int mask) {
  Nm<T, D> r;
  r.v = __shfl_xor_sync(0xffffffffu, a.v, mask);
  r.d = D ? __shfl_xor_sync(0xffffffffu, a.d, mask) : T(0);
  return r;
}
template <typename T, bool D>
__device__ __forceinline__ Nm<T, D> shfl_idx(Nm<T, D> a, int src) {
  Nm<T, D> r;
  r.v = __shfl_sync(0xffffffffu, a.v, src);
  r.d = D ? __shfl_sync(0xffffffffu, a.d, src) : T(0);
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
__device__ __forceinline__ CT ld_elem(const ST *p);
template <>
__device__ __forceinline__ float ld_elem<float, float>(const float *p) {
  return *p;
}
template <>
__device__ __forceinline__ double ld_elem<double, double>(const double *p) {
  return *p;
}
template <>
__device__ __forceinline__ float ld_elem<__nv_bfloat16, float>(const __nv_bfloat16 *p) {
  const uint32_t h = *reinterpret_cast<const unsigned short *>(p);
  return __uint_as_float(h << 16);
}

template <typename CT>
__device__ __forceinline__ CT ld_vec(const void *p, int dt, int i) {
  return dt == TK_F64 ? (CT) reinterpret_cast<const double *>(p)[i]
                      : (CT) reinterpret_cast<const float *>(p)[i];
}


// 1/k for k = 0..15 (entry 0 unused), each the correctly rounded quotient
template <typename CT>
__device__ constexpr CT kInvSmall[16] = {CT(0),      CT(1) / 1,  CT(1) / 2,  CT(1) / 3,  CT(1) / 4,  CT(1) / 5,
                                         CT(1) / 6,  CT(1) / 7,  CT(1) / 8,  CT(1) / 9,  CT(1) / 10, CT(1) / 11,
                                         CT(1) / 12, CT(1) / 13, CT(1) / 14, CT(1) / 15};

constexpr int kRB = 16;    // rows per block of the batched kernel (upper bound)
constexpr int kRows = 32;  // rows per block of the single-vector kernel (upper bound)

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
  const WarpPlan *plan;      // cost-balanced pieces of the range
  int pieces;
  unsigned long long *ticket;  // next piece to hand out (zeroed before the launch)
  unsigned int *done;          // blocks finished (zeroed before the launch)
  int dynamic;                 // 1: shared-ticket schedule, 0: warp w takes w, w+W, ...
  FinalizeArgs fin;            // outputs the last block writes
  int warps;
  int nbuf;         // linear staging buffers per warp
  int buf_bytes;    // bytes of one buffer (block budget + alignment slack)
  int cap;          // block budget in entries
  int vec_bytes;    // bytes of the staged alpha (and v) region, 128-aligned
  int warp_bytes;   // bytes of one warp's region
};

// Threads per block the register budget allows: a base of ~64 registers plus
// the per-lane column state (acc[] and alpha[], doubled for dual numbers and
// for FP64).  Up to 120 estimated registers: 512 threads (128 registers
// each); up to 160: 384 threads (170 registers); above: 256 threads.
__host__ __device__ constexpr int max_threads_est(int ct_bytes, bool dual, int nc) {
  const int est = 64 + (dual ? 2 : 1) * (ct_bytes / 4) * 2 * nc;
  if (dual && ct_bytes == 8) return 256;
  return est <= 120 ? 512 : (est <= 160 ? 384 : 256);
}
template <typename CT, bool D, int NC>
constexpr int max_threads() {
  return max_threads_est((int)sizeof(CT), D, NC);
}

// Per-warp shared-memory header: NBUF mbarriers and the descriptor of each
// issued block: {piece, nb | boff << 6 | LAST | ntri << 11}: nb rows of the
// current triangle, the 16-byte lead of the copy in entries, the last block
// of its piece, and the number of whole triangles that follow those rows in
// the same block.
constexpr int kDescLast = 1 << 10;  // the last block of its piece
constexpr int kDescTriShift = 11;
constexpr int kDescMaxTri = 63;
struct WarpHdr {
  uint64_t bar[8];
  int2 desc[8];
  int pad[32];
};
static_assert(sizeof(WarpHdr) == 256, "warp header");

// Per-row data of the current block, written by lane i for row i and read
// back by the whole warp with one broadcast load.
template <typename CT>
struct __align__(16) RowInfo {
  CT cf_v, cf_d;  // coefficient of the per-entry scatter (value, derivative)
  int rowend;     // index of the row's last entry in the block buffer
  int sl;         // entries after the head
};

template <typename CT, bool D>
__host__ __device__ constexpr int warp_fixed_bytes() {
  // header and row info; 128-byte aligned
  return ((256 + kRows * (int)sizeof(RowInfo<CT>)) + 127) & ~127;
}

// rows of the block that starts at row c (position pos) of its triangle:
// at most kRB, within the triangle, within `cap` entries (rows shrink by one
// entry each, so cap / L0 rows always fit), not past `end`
__device__ __forceinline__ int block_rows(int n, int c, int64_t pos, int64_t end, int cap) {
  const int L0 = n - c;
  int r = min(min(kRB, L0), max(1, (int)__fdividef((float)cap, (float)L0)));
  while (r < min(kRB, L0) && (r + 1) * L0 - ((r + 1) * r) / 2 <= cap) ++r;
  while (r > 1 && pos + (int64_t)(r * L0 - (r * (r - 1)) / 2) > end) --r;
  return r;
}

// One 32-column chunk K of four consecutive rows, software-pipelined: lane j
// holds, in xc[i], the entry of row i at column d = n-1-(32K+j) (loaded one
// step earlier), adds it into g_d's accumulator and into row i's dot; before
// that it issues the loads of chunk K-1 into xn[] (zero past a row's end when
// MASKN, so the multiply-adds need no masks).  MASKN is set only when chunk
// K-1 is the second-highest chunk T-2 of the quad (T = ceil(sl_0 / 32)):
// sl_0 > 32 (T-1) and sl_1 = sl_0 - 1 >= 32 (T-1), so rows 0 and 1 hold every
// column of that chunk and only rows 2 and 3 can end inside it.
template <int K, bool MASKN, int NC, typename ST, typename CT, bool D>
__device__ __forceinline__ void quad_step(Nm<CT, D> (&acc)[NC], Nm<CT, D> (&dot)[4], const Nm<CT, D> (&ar)[NC],
                                          const ST *const (&prow)[4], const int (&sl)[4], int lane,
                                          const Nm<CT, D> (&cf)[4], const CT (&xc)[4], CT (&xn)[4]) {
  if constexpr (K >= 1 && K - 1 < NC) {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      xn[i] = (!MASKN || i < 2 || 32 * (K - 1) + lane < sl[i]) ? ld_elem<ST, CT>(prow[i] - 32 * (K - 1)) : CT(0);
  }
  if constexpr (K < NC) {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      fma_col(acc[K], xc[i], cf[i]);
      fma_acc(dot[i], xc[i], ar[K]);
    }
  }
}
// masked loads of the top chunk K of a quad
template <int K, int NC, typename ST, typename CT>
__device__ __forceinline__ void quad_load(const ST *const (&prow)[4], const int (&sl)[4], int lane, CT (&x)[4]) {
  if constexpr (K < NC) {
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = (32 * K + lane < sl[i]) ? ld_elem<ST, CT>(prow[i] - 32 * K) : CT(0);
  }
}

// Sum of one column of the per-block partials over blocks b0, b0+step, ...
// in increasing order, eight independent loads in flight (L2, not L1: the
// partials were written by other blocks).
__device__ __forceinline__ double sum_blocks(const double *col, int ld2, int grid, int b0, int step) {
  double s = 0.0;
  int b = b0;
  for (; b + 7 * step < grid; b += 8 * step) {
    double v[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __ldcg(col + (size_t)(b + i * step) * ld2);
#pragma unroll
    for (int i = 0; i < 8; ++i) s += v[i];
  }
  for (; b < grid; b += step) s += __ldcg(col + (size_t)b * ld2);
  return s;
}

// Run by the last block of a pass: the fixed-order FP64 sum of every block's
// partials, written as K[a^{m-1}] (mode 0), K[a^{m-2}, v] (mode 1, the
// derivative part over m-1), or the dual objective F, its gradient and the
// gradient norm (mode 2; F = S/m + lambda/2 |a|^2 - <y, a>, grad = g + lambda a - y).
static __device__ void final_reduce(const FinalizeArgs &f, const double *part, int grid) {
  __shared__ double red[3][32];
  const int n = f.n, ld = n + 2, ld2 = 2 * ld;
  const int vec = (f.mode == 1) ? 1 : 0;
  const int nt = blockDim.x;
  // split the blocks over several threads per column (a power of two, <= 8)
  // when the columns are few
  int per = 1;
  while (per < 8 && 2 * per * (n + 1) <= nt) per <<= 1;
  const int cols = (n + 1);
  double ssq = 0.0, aa = 0.0, ya = 0.0;
  __shared__ double S_tot;
  for (int base = 0; base < cols; base += nt / per) {
    const int t = threadIdx.x;
    const int l = base + t / per, sub = t % per;
    const bool act = (t / per) < nt / per && l < cols;
    double s = act ? sum_blocks(part + vec * ld + l, ld2, grid, sub, per) : 0.0;
    // fixed-order tree combine of the per-thread sub-sums of a column
    for (int k = 1; k < per; k <<= 1) s += __shfl_down_sync(0xffffffffu, s, k, per);
    if (act && sub == 0) {
      if (l == n) {
        if (f.mode != 1) S_tot = s;
      } else if (f.mode == 2) {
        const double a = f.alpha[l], gr = s + f.lambda[0] * a - f.y[l];
        if (f.grad) f.grad[l] = gr;
        ssq += gr * gr;
        aa += a * a;
        ya += f.y[l] * a;
      } else {
        const double v = (f.mode == 1) ? s / (double)(f.m - 1) : s;
        if (f.out_dtype == TK_F64) reinterpret_cast<double *>(f.G)[l] = v;
        else reinterpret_cast<float *>(f.G)[l] = (float)v;
      }
    }
  }
  __syncthreads();
  if (f.mode == 0) {
    if (threadIdx.x == 0 && f.S) f.S[0] = S_tot;
    return;
  }
  if (f.mode == 1) return;
  // fixed-order block sums of |grad|^2, |a|^2, <y, a>
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
    aa += __shfl_xor_sync(0xffffffffu, aa, o);
    ya += __shfl_xor_sync(0xffffffffu, ya, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = ssq;
    red[1][wid] = aa;
    red[2][wid] = ya;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0, t1 = 0, t2 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t0 += red[0][w];
      t1 += red[1][w];
      t2 += red[2][w];
    }
    const double S = S_tot;
    if (f.S) f.S[0] = S;
    if (f.F) f.F[0] = S / f.m + 0.5 * f.lambda[0] * t1 - t2;
    if (f.gnorm) f.gnorm[0] = sqrt(t0);
  }
}

// Block-uniform check at kernel entry that the workspace header's plan key
// is the launch's own (m, n, pieces, range); on a mismatch the status word
// records TK_EINVAL at kSiteStalePlan and the caller returns before any load.
__device__ __forceinline__ bool plan_is_stale(int *status, int m, int n, int pieces, int64_t lo, int64_t hi) {
  __shared__ int s_stale;
  if (threadIdx.x == 0) {
    const volatile WsHeader *wh = reinterpret_cast<const volatile WsHeader *>(status);
    s_stale = !(wh->plan_m == m && wh->plan_n == n && wh->plan_pieces == pieces && wh->plan_lo == lo &&
                wh->plan_hi == hi);
    if (s_stale) {
      atomicExch(&reinterpret_cast<WsHeader *>(status)->status, TK_EINVAL);
      reinterpret_cast<WsHeader *>(status)->where = kSiteStalePlan;
    }
  }
  __syncthreads();
  return s_stale != 0;
}

template <typename ST, typename CT, bool D, int NC>
__global__ void __launch_bounds__(max_threads<CT, D, NC>(), 1) contract_kernel(KParams p) {
  using N = Nm<CT, D>;
  constexpr int ES = sizeof(ST);
  // blocks of several whole triangles and the cached step between triangles
  // (n <= 256, n <= 128 for FP64: at larger n the triangles of at most 32 rows
  // hold a negligible share of the entries, and both cost the wide instances
  // registers)
  constexpr bool kMultiTri = NC <= (sizeof(CT) == 8 ? 4 : 8);
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int wid = threadIdx.x >> 5;
  const int m = p.m;
  const int n = p.n;

  CT *a_s = reinterpret_cast<CT *>(smem);
  CT *v_s = a_s + n;
  unsigned char *wb = smem + p.vec_bytes + (size_t)wid * p.warp_bytes;
  WarpHdr *hdr = reinterpret_cast<WarpHdr *>(wb);
  RowInfo<CT> *rinfo = reinterpret_cast<RowInfo<CT> *>(wb + 256);
  CT *g_v = reinterpret_cast<CT *>(wb + warp_fixed_bytes<CT, D>());
  CT *g_d = g_v + n;
  const int gbytes = (int)((((D ? 2 : 1) * n * (int)sizeof(CT)) + 127) & ~127);
  unsigned char *bufs = wb + warp_fixed_bytes<CT, D>() + gbytes;
  const int NB = p.nbuf;

  // the plan region must hold the plan of this launch (a CUDA graph replayed
  // after a later call re-planned the region for another shape would read
  // pieces of another layout): compare the key the host wrote with the upload
  if (plan_is_stale(p.status, m, n, p.pieces, p.off_lo, p.off_hi)) return;

  // rows of a block that starts with a row of length L (rows shrink by one):
  // at most kRows, at most L, within `cap` entries
  short *rfit = reinterpret_cast<short *>(smem + p.vec_bytes - 2 * (n + 1) - 2);
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    a_s[i] = ld_vec<CT>(p.alpha, p.vec_dtype, i);
    if (D) v_s[i] = ld_vec<CT>(p.v, p.vec_dtype, i);
  }
  for (int L = threadIdx.x; L <= n; L += blockDim.x) {
    int r = min(kRows, L);
    while (r > 1 && r * L - (r * (r - 1)) / 2 > p.cap) --r;
    rfit[L] = (short)max(r, 1);
  }
  for (int i = lane; i < n; i += 32) {
    g_v[i] = CT(0);
    if (D) g_d[i] = CT(0);
  }
  if (lane == 0) {
    for (int s = 0; s < NB; ++s) mbar_init(&hdr->bar[s], 1);
    fence_barrier_init();
  }
  __syncthreads();

  auto alpha_at = [&](int i) -> N { return mk<CT, D>(a_s[i], D ? v_s[i] : CT(0)); };

  // ------------------------------------------------------------ pieces
  // Warps take cost-balanced pieces of the range (statically, warp w taking
  // pieces w, w+W, ..., or from a shared ticket).  The copy side of a warp
  // takes the next piece when it has issued every block of the current one
  // and tags each block with a descriptor; the compute side follows the
  // descriptors and never tracks positions.
  const int W = (int)gridDim.x * p.warps;
  const int wg = (int)blockIdx.x * p.warps + wid;
  int next_static = wg;
  auto grab = [&]() -> int {
    if (!p.dynamic) {
      const int t = next_static;
      next_static += W;
      return t < p.pieces ? t : -1;
    }
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(p.ticket, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0);
    return t < (unsigned long long)p.pieces ? (int)t : -1;
  };

  // copy side: piece, triangle cursor (Qp, cp), address of the next entry
  // and the entries left in the piece
  int32_t Qp[kMaxOrder];
  int cp = 0, piece_p = -1;
  const unsigned char *srcp = p.K;
  long long remp = 0;
  bool prod_done = false;
  const unsigned char *const tail_ptr = p.K + (p.bytes & ~int64_t(15));
  // blocks issued / consumed; buffer index and mbarrier phase of each side
  // advance with wrap-around (no division by the runtime buffer count)
  int j_issue = 0, j_cons = 0;
  int bi_issue = 0, bi_cons = 0;
  uint32_t ph_cons = 0;
  bool failed = false;

  // issue the bulk copy of the next block at the copy cursor
  auto issue_next = [&]() {
    if (prod_done) return;
    while (remp <= 0) {
      piece_p = grab();
      if (piece_p < 0) {
        prod_done = true;
        return;
      }
      const WarpPlan &pl = p.plan[piece_p];
      remp = pl.end - pl.start;
      for (int j = 0; j < kMaxOrder; ++j) Qp[j] = pl.t[j];
      cp = pl.t[m - 2];
      srcp = p.K + (pl.start - p.off_lo) * ES;
    }
    const int L0 = n - cp;
    int nb = rfit[L0];
    int span = nb * L0 - ((nb * (nb - 1)) >> 1);
    while (nb > 1 && span > remp) {  // the piece ends inside this block (rare)
      --nb;
      span -= L0 - nb;
    }
    // A block that holds a whole triangle (it starts at the triangle's first
    // row and takes all its rows) also takes the whole triangles that follow,
    // while they fit the buffer and the piece (the many small triangles of
    // high orders then share one copy and one wait).
    const bool whole = kMultiTri && m > 2 && nb == L0 && cp == Qp[m - 3];
    remp -= span;
    cp += nb;
    if (cp == n && remp > 0) {
      if (m > 2 && next_sorted(m - 2, n, Qp)) cp = Qp[m - 3];
      else remp = 0;
    }
    int tot = span, ntri = 0;
    if (whole) {
      while (ntri < kDescMaxTri && remp > 0) {
        const int L = n - cp;  // cp is the first row of the next triangle
        const int ts = (L * (L + 1)) >> 1;
        if (L > kRows || tot + ts > p.cap || ts > remp) break;
        tot += ts;
        remp -= ts;
        ++ntri;
        cp = n;
        if (remp > 0) {
          if (next_sorted(m - 2, n, Qp)) cp = Qp[m - 3];
          else remp = 0;
        }
      }
    }
    const uint32_t lead = (uint32_t)reinterpret_cast<uintptr_t>(srcp) & 15u;
    const unsigned char *b0 = srcp - lead;
    const unsigned char *e1 = srcp + (int64_t)tot * ES;
    uint32_t bytes = (lead + (uint32_t)(tot * ES) + 15u) & ~15u;
    const int bi = bi_issue;
    unsigned char *dst = bufs + (size_t)bi * p.buf_bytes;
    if (e1 > tail_ptr) {
      // the block reaches past the array's last 16-byte boundary (the last
      // block of the range): the bytes from there are copied by hand
      bytes = (uint32_t)(tail_ptr - b0);
      const int nt = (int)(e1 - tail_ptr);
      if (lane < nt) dst[bytes + lane] = tail_ptr[lane];
      __syncwarp();
    }
    if (lane == 0) {
      hdr->desc[bi] = make_int2(piece_p, nb | (int)((lead / ES) << 6) | (remp <= 0 ? kDescLast : 0) |
                                             (ntri << kDescTriShift));
      if (bytes) {
        fence_proxy_async();
        mbar_expect_tx(&hdr->bar[bi], bytes);
        bulk_g2s(dst, b0, bytes, &hdr->bar[bi]);
      } else {
        mbar_arrive(&hdr->bar[bi]);  // nothing to copy: complete the phase
      }
    }
    srcp = e1;
    ++j_issue;
    bi_issue = (bi_issue + 1 == NB) ? 0 : bi_issue + 1;
  };

  // ------------------------------------------------------------ accumulators
  N acc[NC];
  N ar[NC];
#pragma unroll
  for (int k = 0; k < NC; ++k) {
    acc[k] = mk<CT, D>(CT(0), CT(0));
    const int e = 32 * k + lane;
    ar[k] = (e < n) ? alpha_at(n - 1 - e) : mk<CT, D>(CT(0), CT(0));
  }
  double S_v = 0.0, S_d = 0.0;

  // triangle state
  int32_t Q[kMaxOrder];
  int c = 0, piece_c = -1;
  int b = -1;   // last value of Q (-1: m = 2, no first row)
  int kb = 0;   // multiplicity of b in Q
  CT Mprime = CT(2), Mf = CT(2), inv_first = CT(0.5);
  N AQ = mk<CT, D>(CT(1), CT(0));
  N cA = AQ, cAf = AQ;
  N Trest = mk<CT, D>(CT(0), CT(0)), Tfirst = Trest;
  const CT inv_m = CT(1) / CT(m);
  // Prefix cache for the step between consecutive triangles (P, b) -> (P, b+1)
  // of one (m-3)-prefix P = (Q_0..Q_{m-4}) (multi-triangle instances): when b
  // is unique in Q and b < n-1, b+1 is unique in the next triangle too, so M',
  // M_f and 1/(cnt_Q(b)+2) stay, A_Q = A_P a_{b+1}, and lane l < m-2 keeps its
  // prefix value, its count and B_{Q,l} without the factor a_b.  Every product
  // is formed in the order of the full set-up, so both give the same roundings.
  N AP = mk<CT, D>(CT(1), CT(0));  // product of a over Q_0..Q_{m-4}
  N BP_l = AP;                     // lane l < m-3: that product without position l
  int q_l = 0, cnt_l = 0;          // lane l < m-2: Q_l and cnt_Q(Q_l) (0 unless first of its run)

  auto setup_triangle = [&]() {
    AQ = mk<CT, D>(CT(1), CT(0));
    AP = AQ;
    // M' = m! / prod_v cnt_Q(v)!: divide m! by the position of each entry in
    // its run of equal values (every partial quotient is a multinomial
    // coefficient, so each division is exact)
    uint64_t mp = 1;
    for (int i = 2; i <= m; ++i) mp *= (uint64_t)i;
    int run = 0;
    for (int j = 0; j < m - 2; ++j) {
      AQ = AQ * alpha_at(Q[j]);
      if (j == m - 4) AP = AQ;
      run = (j > 0 && Q[j] == Q[j - 1]) ? run + 1 : 1;
      if (run > 1) mp = exact_div_small(mp, run);
    }
    // the last run is the one of b = Q[m-3]: its length is cnt_Q(b)
    b = (m > 2) ? Q[m - 3] : -1;
    kb = (m > 2) ? run : 0;
    Mprime = CT(mp);
    Mf = CT(exact_div_small(mp, kb + 1));  // M' / (cnt_Q(b) + 1), an integer
    inv_first = kInvSmall<CT>[kb + 2];      // 1 / (cnt_Q(b) + 2), cnt_Q(b) <= m - 2
    cA = scale(Mprime * inv_m, AQ);
    cAf = scale(Mf * inv_m, AQ);
    if constexpr (kMultiTri) {
      if (lane < m - 2) {
        q_l = Q[lane];
        int cnt = 0;
        N B = mk<CT, D>(CT(1), CT(0));
        for (int j = 0; j < m - 2; ++j) {
          cnt += (Q[j] == q_l);
          if (j != lane && j < m - 3) B = B * alpha_at(Q[j]);
        }
        cnt_l = (lane == 0 || Q[lane] != Q[lane - 1]) ? cnt : 0;
        BP_l = B;
      }
    }
  };

  // the next triangle (P, b+1) when b is unique in Q and below n-1
  auto step_triangle = [&]() {
    b += 1;
    Q[m - 3] = b;
    AQ = AP * alpha_at(b);
    cA = scale(Mprime * inv_m, AQ);
    cAf = scale(Mf * inv_m, AQ);
    if (lane == m - 3) q_l = b;
  };

  auto flush_triangle = [&]() {
    __syncwarp();
    N Tr = warp_sum(Trest);
    N Tf = warp_sum(Tfirst);
    N T = Tr + Tf;
    N SQ = AQ * T;
    if (D) S_d += (double)SQ.d;
    else S_v += (double)SQ.v;
    if constexpr (kMultiTri) {
      if (lane < m - 2 && cnt_l > 0) {
        const N B = (lane < m - 3) ? BP_l * alpha_at(b) : AP;
        N add = scale(CT(cnt_l) * inv_m, B * ((q_l == b) ? Tr : T));
        if (D) g_d[q_l] += add.d;
        else g_v[q_l] += add.v;
      }
    } else if (lane < m - 2 && (lane == 0 || Q[lane] != Q[lane - 1])) {
      const int l = Q[lane];
      int cnt = 0;
      N B = mk<CT, D>(CT(1), CT(0));
      for (int j = 0; j < m - 2; ++j) {
        cnt += (Q[j] == l);
        if (j != lane) B = B * alpha_at(Q[j]);
      }
      N add = scale(CT(cnt) * inv_m, B * ((l == b) ? Tr : T));
      if (D) g_d[l] += add.d;
      else g_v[l] += add.v;
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < NC; ++k) {
      const int e = 32 * k + lane;
      if (e < n) {
        if (D) g_d[n - 1 - e] += acc[k].d;
        else g_v[n - 1 - e] += acc[k].v;
      }
      acc[k] = mk<CT, D>(CT(0), CT(0));
    }
    __syncwarp();
    Trest = mk<CT, D>(CT(0), CT(0));
    Tfirst = Trest;
  };

  for (int s = 0; s < NB - 1; ++s) issue_next();
  bool open = false;

  while (j_cons < j_issue && !failed) {
    // ---------------------------------------------------- wait for this block
    const int bi = bi_cons;
    const uint32_t parity = ph_cons;
    __syncwarp();
    const int2 dsc = hdr->desc[bi];
    int nb = dsc.y & 63;
    int ntri = (dsc.y >> kDescTriShift) & kDescMaxTri;  // whole triangles after the first nb rows
    if (dsc.x != piece_c) {
      // this block starts a new piece: restart the compute cursor there
      if (open) flush_triangle();
      const WarpPlan &pl = p.plan[dsc.x];
      for (int j = 0; j < kMaxOrder; ++j) Q[j] = pl.t[j];
      c = pl.t[m - 2];
      piece_c = dsc.x;
      setup_triangle();
      open = true;
    }
    const unsigned char *buf = bufs + (size_t)bi * p.buf_bytes;
    if (!__all_sync(0xffffffffu, mbar_wait_bounded(&hdr->bar[bi], parity))) {
      if (lane == 0) {
        atomicExch(&reinterpret_cast<WsHeader *>(p.status)->status, TK_ETIMEOUT);
        reinterpret_cast<WsHeader *>(p.status)->where = kSiteContractWait;
      }
      failed = true;
      break;
    }
    ++j_cons;
    if (++bi_cons == NB) {
      bi_cons = 0;
      ph_cons ^= 1u;
    }
    // the previous block's buffer is free again: keep NBUF-1 copies in flight
    issue_next();

    // ---------------------------------------------------- rows of the block
    // nb rows of the current triangle, then (ntri > 0) each following whole
    // triangle in turn, at consecutive positions of the buffer
    const ST *bp = reinterpret_cast<const ST *>(buf) + ((dsc.y >> 6) & 15);
    bool stop = false;
    for (;;) {
      const int L0 = n - c;
      __syncwarp();
      // lane i holds row i: its head, alpha and coefficients
      const bool live = lane < nb;
      const int ci = min(c + lane, n - 1);
      const N ac = alpha_at(ci);
      const bool first = ci == b;
      const N coef = first ? cAf : cA;
      const int rowend = live ? (L0 - 1) + lane * L0 - ((lane * (lane + 1)) >> 1) : L0 - 1;
      const int rsl = live ? L0 - lane - 1 : 0;
      const CT hv = ld_elem<ST, CT>(bp + (rowend - rsl));
      {
        // rows past the block's end read row 0's (finite) entries with a zero
        // coefficient, so the unmasked chunks stay harmless
        const N cfi = live ? coef * ac : mk<CT, D>(CT(0), CT(0));
        RowInfo<CT> rw;
        rw.cf_v = cfi.v;
        rw.cf_d = cfi.d;
        rw.rowend = rowend;
        rw.sl = rsl;
        rinfo[lane] = rw;
      }
      __syncwarp();
      N s = mk<CT, D>(CT(0), CT(0));  // the dot of row `lane`
      for (int r = 0; r < nb; r += 4) {
        // four rows at a time: their lengths differ by at most 3, so the chunk
        // count of the longest serves all four; only its top two chunks can run
        // past a row's end and need masks
        N cf[4], dot[4];
        int sl[4];
        const ST *prow[4];
        CT xa[4], xb[4];
  #pragma unroll
        for (int i = 0; i < 4; ++i) {
          const RowInfo<CT> rw = rinfo[r + i];
          cf[i] = mk<CT, D>(rw.cf_v, rw.cf_d);
          sl[i] = rw.sl;
          prow[i] = bp + (rw.rowend - lane);
          dot[i] = mk<CT, D>(CT(0), CT(0));
        }
        // enter at the top chunk (two masked chunks), continue down the
        // unmasked chain to chunk 0
        switch ((sl[0] + 31) >> 5) {
          case 1: quad_load<0, NC>(prow, sl, lane, xa); quad_step<0, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto chunks_done;
          case 2: quad_load<1, NC>(prow, sl, lane, xb); quad_step<1, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<0, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto chunks_done;
          case 3: quad_load<2, NC>(prow, sl, lane, xa); quad_step<2, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<1, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_0;
          case 4: quad_load<3, NC>(prow, sl, lane, xb); quad_step<3, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<2, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_1;
          case 5: quad_load<4, NC>(prow, sl, lane, xa); quad_step<4, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<3, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_2;
          case 6: quad_load<5, NC>(prow, sl, lane, xb); quad_step<5, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<4, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_3;
          case 7: quad_load<6, NC>(prow, sl, lane, xa); quad_step<6, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<5, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_4;
          case 8: quad_load<7, NC>(prow, sl, lane, xb); quad_step<7, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<6, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_5;
          case 9: quad_load<8, NC>(prow, sl, lane, xa); quad_step<8, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<7, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_6;
          case 10: quad_load<9, NC>(prow, sl, lane, xb); quad_step<9, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<8, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_7;
          case 11: quad_load<10, NC>(prow, sl, lane, xa); quad_step<10, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<9, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_8;
          case 12: quad_load<11, NC>(prow, sl, lane, xb); quad_step<11, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<10, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_9;
          case 13: quad_load<12, NC>(prow, sl, lane, xa); quad_step<12, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<11, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_10;
          case 14: quad_load<13, NC>(prow, sl, lane, xb); quad_step<13, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<12, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_11;
          case 15: quad_load<14, NC>(prow, sl, lane, xa); quad_step<14, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<13, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_12;
          case 16: quad_load<15, NC>(prow, sl, lane, xb); quad_step<15, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<14, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_13;
          case 17: quad_load<16, NC>(prow, sl, lane, xa); quad_step<16, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<15, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_14;
          case 18: quad_load<17, NC>(prow, sl, lane, xb); quad_step<17, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<16, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_15;
          case 19: quad_load<18, NC>(prow, sl, lane, xa); quad_step<18, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<17, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_16;
          case 20: quad_load<19, NC>(prow, sl, lane, xb); quad_step<19, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<18, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_17;
          case 21: quad_load<20, NC>(prow, sl, lane, xa); quad_step<20, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<19, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_18;
          case 22: quad_load<21, NC>(prow, sl, lane, xb); quad_step<21, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<20, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_19;
          case 23: quad_load<22, NC>(prow, sl, lane, xa); quad_step<22, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<21, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_20;
          case 24: quad_load<23, NC>(prow, sl, lane, xb); quad_step<23, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<22, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_21;
          case 25: quad_load<24, NC>(prow, sl, lane, xa); quad_step<24, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<23, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_22;
          case 26: quad_load<25, NC>(prow, sl, lane, xb); quad_step<25, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<24, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_23;
          case 27: quad_load<26, NC>(prow, sl, lane, xa); quad_step<26, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<25, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_24;
          case 28: quad_load<27, NC>(prow, sl, lane, xb); quad_step<27, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<26, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_25;
          case 29: quad_load<28, NC>(prow, sl, lane, xa); quad_step<28, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<27, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_26;
          case 30: quad_load<29, NC>(prow, sl, lane, xb); quad_step<29, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<28, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_27;
          case 31: quad_load<30, NC>(prow, sl, lane, xa); quad_step<30, true>(acc, dot, ar, prow, sl, lane, cf, xa, xb); quad_step<29, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa); goto full_28;
          case 32: quad_load<31, NC>(prow, sl, lane, xb); quad_step<31, true>(acc, dot, ar, prow, sl, lane, cf, xb, xa); quad_step<30, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb); goto full_29;
          default: goto chunks_done;
        }
      full_29: quad_step<29, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_28: quad_step<28, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_27: quad_step<27, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_26: quad_step<26, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_25: quad_step<25, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_24: quad_step<24, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_23: quad_step<23, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_22: quad_step<22, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_21: quad_step<21, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_20: quad_step<20, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_19: quad_step<19, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_18: quad_step<18, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_17: quad_step<17, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_16: quad_step<16, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_15: quad_step<15, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_14: quad_step<14, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_13: quad_step<13, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_12: quad_step<12, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_11: quad_step<11, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_10: quad_step<10, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_9: quad_step<9, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_8: quad_step<8, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_7: quad_step<7, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_6: quad_step<6, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_5: quad_step<5, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_4: quad_step<4, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_3: quad_step<3, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_2: quad_step<2, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      full_1: quad_step<1, false>(acc, dot, ar, prow, sl, lane, cf, xb, xa);
      full_0: quad_step<0, false>(acc, dot, ar, prow, sl, lane, cf, xa, xb);
      chunks_done:;
        {
          // butterfly over the lanes: after it lane l holds the dot of row
          // r + 2 (l >> 4 & 1) + (l >> 3 & 1); row r + i then moves to lane r + i
          const bool hi = (lane & 16) != 0, b8 = (lane & 8) != 0;
          const N k0 = (hi ? dot[2] : dot[0]) + shfl_xor(hi ? dot[0] : dot[2], 16);
          const N k1 = (hi ? dot[3] : dot[1]) + shfl_xor(hi ? dot[1] : dot[3], 16);
          N k = (b8 ? k1 : k0) + shfl_xor(b8 ? k0 : k1, 8);
          k = k + shfl_xor(k, 4);
          k = k + shfl_xor(k, 2);
          k = k + shfl_xor(k, 1);
          k = shfl_idx(k, ((lane & 2) << 3) | ((lane & 1) << 3));
          if ((lane & ~3) == r) s = k;
        }
      }

      // ---------------------------------------------------- row epilogue
      if (live) {
        const CT cnt = first ? CT(kb + 1) : CT(1);
        const N Rf = s + scale(hv * (first ? inv_first : CT(0.5)), ac);
        const N gadd = coef * (scale(hv, ac) + scale(cnt, s));
        if (D) g_d[ci] += gadd.d;
        else g_v[ci] += gadd.v;
        const N tadd = scale(first ? Mf : Mprime, ac * Rf);
        if (first) Tfirst = Tfirst + tadd;
        else Trest = Trest + tadd;
      }

      // ---------------------------------------------------- advance
      c += nb;
      if (c == n) {
        flush_triangle();
        open = false;
        // the block's last triangle may end its piece; the next piece then
        // restarts the cursor from its plan record
        if (ntri > 0 || !(dsc.y & kDescLast)) {
          if (kMultiTri && m > 2 && kb == 1 && b < n - 1) {
            step_triangle();
            c = b;
            open = true;
          } else if (m > 2 && next_sorted(m - 2, n, Q)) {
            c = Q[m - 3];
            setup_triangle();
            open = true;
          } else {
            stop = true;
            break;
          }
        }
      }
      if (!kMultiTri || ntri == 0) break;
      --ntri;
      bp += nb * L0 - ((nb * (nb - 1)) >> 1);
      nb = n - c;  // the next triangle, whole
    }
    if (stop) break;
  }
  if (open) flush_triangle();
  // drain copies still in flight before the block can exit
  while (j_cons < j_issue) {
    mbar_wait_bounded(&hdr->bar[bi_cons], ph_cons);
    ++j_cons;
    if (++bi_cons == NB) {
      bi_cons = 0;
      ph_cons ^= 1u;
    }
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
      const CT *gw = reinterpret_cast<const CT *>(smem + p.vec_bytes + (size_t)ww * p.warp_bytes +
                                                  warp_fixed_bytes<CT, D>());
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

  // ------------------------------------------------------------ last block sums all blocks
  __threadfence();
  __syncthreads();
  __shared__ int s_last;
  if (threadIdx.x == 0) s_last = (atomicAdd(p.done, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  final_reduce(p.fin, p.part, gridDim.x);
}

// ------------------------------------------------------------------ launch
template <typename ST, typename CT, bool D, int NC>
inline int launch_nc(const KParams &kp, int grid, int threads, size_t smem, cudaStream_t st) {
  auto kern = contract_kernel<ST, CT, D, NC>;
  if (threads > max_threads<CT, D, NC>())
    return fail(TK_EINVAL, "contract: %d threads exceed the kernel's bound", threads);
  // raise the kernel's dynamic shared-memory limit once per device (and when
  // a launch needs more): the attribute call is then absent from later calls,
  // which a stream capture may record
  static int limit_set[64] = {0};
  int dev = 0;
  TK_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64 || limit_set[dev] < (int)smem) {
    TK_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (dev >= 0 && dev < 64) limit_set[dev] = (int)smem;
  }
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
