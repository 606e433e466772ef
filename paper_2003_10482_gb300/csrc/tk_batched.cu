// Batched packed contraction: K[a_b^{m-1}] and K[a_b^m] (or, with directions,
// K[a_b^{m-2}, v_b]) for up to thousands of dual vectors in one launch -- the
// lambda path x cross-validation folds of a batched dual solve.  The sums and
// the triangle/row/entry decomposition are those of the single-vector kernel
// (tk_contract_impl.cuh); the mapping onto the GPU differs:
//
//   * a block owns a group of 32*VPL vectors (lane <-> vector, VPL per lane)
//     and one slice of the packed range (pieces s, s+S, s+2S, ... of the
//     cost-balanced cut); the blocks of all groups walk their slices in the
//     same order at the same pace, so a row block read from HBM by one group
//     is served from L2 to the others;
//   * row blocks are staged once per block by one cp.async.bulk copy and the
//     16 warps split the columns (warp w takes e = n-1-d = w, w+16, ...): each
//     entry is a broadcast shared load feeding 2*VPL FMAs per thread, and each
//     thread keeps the g_d accumulators of its columns for its vectors in
//     registers;
//   * the row dots are reduced across warps through shared memory four rows
//     at a time; the warp that owns row c's own column applies that row's
//     epilogue (its g_c term goes into that warp's accumulator);
//   * accumulators are flushed to a per-block FP64 partial every few thousand
//     rows (bounded FP32 summation depth); a second kernel sums the partials
//     of the slices in a fixed order.
#include <algorithm>

#include "tk_contract_impl.cuh"

namespace tk {

constexpr int kBW = 16;  // warps per block
constexpr int kBT = 512;

struct BParams {
  int m, n;
  const unsigned char *K;
  int64_t off_lo, off_hi, bytes;
  const void *A;
  const void *V;
  int vec_dtype;
  int64_t B;
  int groups, slices;
  const WarpPlan *plan;
  int pieces;
  double *gpart;  // [block][2][n+2][32*VPL]
  int *status;
  int nbuf, buf_bytes, cap;
  int flush_rows;
  int vec_bytes;  // bytes of the staged vectors (a, v), 128-aligned
};

template <typename CT, bool D, int VPL>
struct BShared {
  static constexpr int BL = 32 * VPL;              // vectors per block
  static constexpr int nv = D ? 2 : 1;
  static constexpr int red_floats = kBW * 16 * BL * nv;     // row dots of a block, per warp
  static constexpr int tsm_floats = 2 * kBW * BL * nv;      // rest / first per warp
  static constexpr int ttot_floats = 2 * BL * nv;
};

// one 16-column step of a quad: warp w takes column e = w + 16K of four rows.
// The bases are already shifted by w (pw[i] = row end - w, acw = alpha at
// column w, slw[i] = entries after the head - w), so each access is a fixed
// displacement from a per-quad register.
template <int K, int NCOL, int VPL, typename ST, bool D>
__device__ __forceinline__ void bquad(Nm<float, D> (&acc)[NCOL][VPL], Nm<float, D> (&dot)[4][VPL],
                                      const float *acw, const float *vcw, const ST *const (&pw)[4],
                                      const int (&slw)[4], const Nm<float, D> (&cf)[4][VPL]) {
  if constexpr (K < NCOL) {
    constexpr int BL = 32 * VPL;
    Nm<float, D> al[VPL];
    if constexpr (VPL == 2) {
      const float2 a2 = *reinterpret_cast<const float2 *>(acw - kBW * K * BL);
      al[0].v = a2.x;
      al[1].v = a2.y;
      if (D) {
        const float2 v2 = *reinterpret_cast<const float2 *>(vcw - kBW * K * BL);
        al[0].d = v2.x;
        al[1].d = v2.y;
      } else {
        al[0].d = al[1].d = 0.f;
      }
    } else {
      al[0].v = acw[-kBW * K * BL];
      al[0].d = D ? vcw[-kBW * K * BL] : 0.f;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (kBW * K < slw[i]) {
        const float x = ld_elem<ST, float>(pw[i] - kBW * K);
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
          fma_acc(acc[K][v], x, cf[i][v]);
          fma_acc(dot[i][v], x, al[v]);
        }
      }
    }
  }
}

template <int K, int NCOL, int VPL, bool D>
__device__ __forceinline__ void badd(Nm<float, D> (&acc)[NCOL][VPL], int v, Nm<float, D> x) {
  if constexpr (K < NCOL) acc[K][v] = acc[K][v] + x;
}

// acc[k][v] += x for a runtime k (jump table)
template <int NCOL, int VPL, bool D>
__device__ __forceinline__ void badd_dyn(Nm<float, D> (&acc)[NCOL][VPL], int k, int v, Nm<float, D> x) {
  switch (k) {
#define TK_BADD(K) \
  case K: badd<K, NCOL, VPL, D>(acc, v, x); break;
    TK_BADD(0) TK_BADD(1) TK_BADD(2) TK_BADD(3) TK_BADD(4) TK_BADD(5) TK_BADD(6) TK_BADD(7)
    TK_BADD(8) TK_BADD(9) TK_BADD(10) TK_BADD(11) TK_BADD(12) TK_BADD(13) TK_BADD(14) TK_BADD(15)
    TK_BADD(16) TK_BADD(17) TK_BADD(18) TK_BADD(19) TK_BADD(20) TK_BADD(21) TK_BADD(22) TK_BADD(23)
    TK_BADD(24) TK_BADD(25) TK_BADD(26) TK_BADD(27) TK_BADD(28) TK_BADD(29) TK_BADD(30) TK_BADD(31)
    TK_BADD(32) TK_BADD(33) TK_BADD(34) TK_BADD(35) TK_BADD(36) TK_BADD(37) TK_BADD(38) TK_BADD(39)
    TK_BADD(40) TK_BADD(41) TK_BADD(42) TK_BADD(43) TK_BADD(44) TK_BADD(45) TK_BADD(46) TK_BADD(47)
#undef TK_BADD
    default: break;
  }
}

template <typename ST, bool D, int VPL, int NCOL>
__global__ void __launch_bounds__(kBT, 1) batched_kernel(BParams p) {
  using N = Nm<float, D>;
  using SH = BShared<float, D, VPL>;
  constexpr int BL = SH::BL;
  constexpr int ES = sizeof(ST);
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31;
  const int w = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  const int g = blockIdx.x / p.slices;
  const int sidx = blockIdx.x % p.slices;
  if (plan_is_stale(p.status, m, n, p.pieces, p.off_lo, p.off_hi)) return;

  float *a_s = reinterpret_cast<float *>(smem);  // [n][BL] (value), then [n][BL] (direction)
  float *v_s = a_s + (size_t)n * BL;
  float *red = reinterpret_cast<float *>(smem + p.vec_bytes);   // [kBW][16][BL] x nv
  float *tsm = red + SH::red_floats;                             // [2: rest, first][kBW][BL] x nv
  float *ttot = tsm + SH::tsm_floats;                            // [2: rest, all][BL] x nv
  double *ssm = reinterpret_cast<double *>(ttot + SH::ttot_floats);  // [BL] x nv
  uint64_t *bar = reinterpret_cast<uint64_t *>(ssm + BL * SH::nv);
  int *desc_nb = reinterpret_cast<int *>(bar + 8);
  int *desc_pc = desc_nb + 8;
  const int bufs_off = (int)(((reinterpret_cast<unsigned char *>(desc_pc + 8) - smem) + 127) & ~127);
  unsigned char *bufs = smem + bufs_off;
  const int NB = p.nbuf;

  // stage this group's vectors: a_s[d][bl] for d < n
  for (int i = threadIdx.x; i < n * BL; i += blockDim.x) {
    const int d = i / BL, bl = i % BL;
    const int64_t b = (int64_t)g * BL + bl;
    float av = 0.f, vv = 0.f;
    if (b < p.B) {
      av = ld_vec<float>(p.A, p.vec_dtype, (int)(b * n + d));
      if (D) vv = ld_vec<float>(p.V, p.vec_dtype, (int)(b * n + d));
    }
    a_s[i] = av;
    if (D) v_s[i] = vv;
  }
  for (int i = threadIdx.x; i < SH::tsm_floats; i += blockDim.x) tsm[i] = 0.f;
  for (int i = threadIdx.x; i < BL * SH::nv; i += blockDim.x) ssm[i] = 0.0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NB; ++s) mbar_init(&bar[s], 1);
    fence_barrier_init();
  }
  // this block's partial region, zeroed
  double *gp = p.gpart + (size_t)blockIdx.x * 2 * (n + 2) * BL;
  for (int i = threadIdx.x; i < 2 * (n + 2) * BL; i += blockDim.x) gp[i] = 0.0;
  __syncthreads();

  auto alpha_at = [&](int d, int bl) -> N { return mk<float, D>(a_s[d * BL + bl], D ? v_s[d * BL + bl] : 0.f); };

  // per-thread column state
  N acc[NCOL][VPL];
#pragma unroll
  for (int k = 0; k < NCOL; ++k) {
    const int e = w + kBW * k;
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      acc[k][v] = mk<float, D>(0.f, 0.f);
      (void)e;
    }
  }
  auto flush_acc = [&]() {
#pragma unroll
    for (int k = 0; k < NCOL; ++k) {
      const int e = w + kBW * k;
      if (e < n) {
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
          const size_t o = (size_t)(n - 1 - e) * BL + lane * VPL + v;
          gp[o] += (double)acc[k][v].v;
          if (D) gp[(size_t)(n + 2) * BL + o] += (double)acc[k][v].d;
        }
      }
#pragma unroll
      for (int v = 0; v < VPL; ++v) acc[k][v] = mk<float, D>(0.f, 0.f);
    }
  };

  // ------------------------------------------------------------ pieces (static, this slice)
  int next_piece = sidx;
  auto grab = [&]() -> int {
    const int t = next_piece;
    next_piece += p.slices;
    return t < p.pieces ? t : -1;
  };
  int32_t Q[kMaxOrder], Qp[kMaxOrder];
  int c = 0, cp = 0;
  int64_t pos = 0, end = 0, posp = 0, endp = 0;
  int piece_p = grab();
  if (piece_p >= 0) {
    const WarpPlan &pl = p.plan[piece_p];
    for (int j = 0; j < kMaxOrder; ++j) Qp[j] = pl.t[j];
    cp = pl.t[m - 2];
    posp = pl.start;
    endp = pl.end;
  }
  bool prod_done = piece_p < 0;
  int piece_c = -1;
  const int64_t tail_lo = p.bytes & ~int64_t(15);
  // blocks issued / consumed; buffer index and mbarrier phase of each side
  // advance with wrap-around (no division by the runtime buffer count)
  int j_issue = 0, j_cons = 0;
  int bi_issue = 0, bi_cons = 0;
  uint32_t ph_cons = 0;

  // the copy side runs on every thread (uniform state), thread 0 issues
  auto issue_next = [&]() {
    while (!prod_done && posp >= endp) {
      piece_p = grab();
      if (piece_p < 0) {
        prod_done = true;
        return;
      }
      const WarpPlan &pl = p.plan[piece_p];
      for (int j = 0; j < kMaxOrder; ++j) Qp[j] = pl.t[j];
      cp = pl.t[m - 2];
      posp = pl.start;
      endp = pl.end;
    }
    if (prod_done) return;
    const int nb = block_rows(n, cp, posp, endp, p.cap);
    const int L0 = n - cp;
    const int64_t pend = posp + (int64_t)(nb * L0 - (nb * (nb - 1)) / 2);
    const int bi = bi_issue;
    const int64_t b0 = ((posp - p.off_lo) * ES) & ~int64_t(15);
    const int64_t b1 = min((((pend - p.off_lo) * ES) + 15) & ~int64_t(15), tail_lo);
    if (threadIdx.x == 0) {
      desc_nb[bi] = nb;
      desc_pc[bi] = piece_p;
      if (b1 > b0) {
        fence_proxy_async();
        mbar_expect_tx(&bar[bi], (uint32_t)(b1 - b0));
        bulk_g2s(bufs + (size_t)bi * p.buf_bytes, p.K + b0, (uint32_t)(b1 - b0), &bar[bi]);
      }
    }
    cp += nb;
    posp = pend;
    if (cp == n && posp < endp) {
      if (m > 2 && next_sorted(m - 2, n, Qp)) cp = Qp[m - 3];
    }
    ++j_issue;
    bi_issue = (bi_issue + 1 == NB) ? 0 : bi_issue + 1;
  };

  // ------------------------------------------------------------ triangle state (per vector)
  int b = -1, kb = 0;
  float Mprime = 2.f, Mf = 2.f, inv_first = 0.5f;
  N AQ[VPL], cA[VPL], cAf[VPL];
  const float inv_m = 1.f / (float)m;
  auto setup_triangle = [&]() {
    int fact_m = 1;
    for (int i = 2; i <= m; ++i) fact_m *= i;
    int den = 1, run = 0;
    for (int j = 0; j < m - 2; ++j) {
      run = (j > 0 && Q[j] == Q[j - 1]) ? run + 1 : 1;
      den *= run;
    }
    b = (m > 2) ? Q[m - 3] : -1;
    kb = 0;
    for (int j = 0; j < m - 2; ++j) kb += (Q[j] == b);
    Mprime = (float)(fact_m / den);
    Mf = Mprime / (float)(kb + 1);
    inv_first = 1.f / (float)(kb + 2);
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      N a = mk<float, D>(1.f, 0.f);
      for (int j = 0; j < m - 2; ++j) a = a * alpha_at(Q[j], lane * VPL + v);
      AQ[v] = a;
      cA[v] = scale(Mprime * inv_m, a);
      cAf[v] = scale(Mf * inv_m, a);
    }
  };
  // end of a triangle's rows in this block: S and the Q-index terms
  auto flush_triangle = [&]() {
    __syncthreads();  // every epilogue of the triangle has written tsm
    if (w < VPL) {
      // vector bl = lane*VPL + w is this thread's vector w
      const int bl = lane * VPL + w;
      N tr = mk<float, D>(0.f, 0.f), tf = tr;
      for (int ww = 0; ww < kBW; ++ww) {
        tr.v += tsm[(0 * kBW + ww) * BL + bl];
        tf.v += tsm[(1 * kBW + ww) * BL + bl];
        if (D) {
          tr.d += tsm[SH::tsm_floats / 2 + (0 * kBW + ww) * BL + bl];
          tf.d += tsm[SH::tsm_floats / 2 + (1 * kBW + ww) * BL + bl];
        }
      }
      const N T = tr + tf;
      ttot[bl] = tr.v;
      ttot[BL + bl] = T.v;
      if (D) {
        ttot[SH::ttot_floats / 2 + bl] = tr.d;
        ttot[SH::ttot_floats / 2 + BL + bl] = T.d;
      }
      // S += A_Q T (this thread's vector bl is AQ[w] of lane)
      const N sq = AQ[w] * T;
      ssm[bl] += (double)sq.v;
      if (D) ssm[BL + bl] += (double)sq.d;
    }
    __syncthreads();
    // Q-index terms: the warp owning column l adds them
    for (int j = 0; j < m - 2; ++j) {
      if (j > 0 && Q[j] == Q[j - 1]) continue;
      const int l = Q[j];
      const int e = n - 1 - l;
      if ((e % kBW) != w) continue;
      int cnt = 0;
      for (int jj = 0; jj < m - 2; ++jj) cnt += (Q[jj] == l);
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const int bl = lane * VPL + v;
        N B = mk<float, D>(1.f, 0.f);
        bool skipped = false;
        for (int jj = 0; jj < m - 2; ++jj) {
          if (!skipped && Q[jj] == l) {
            skipped = true;
            continue;
          }
          B = B * alpha_at(Q[jj], bl);
        }
        const int off = (l == b) ? 0 : BL;
        const N T = mk<float, D>(ttot[off + bl], D ? ttot[SH::ttot_floats / 2 + off + bl] : 0.f);
        badd_dyn<NCOL, VPL, D>(acc, e / kBW, v, scale((float)cnt * inv_m, B * T));
      }
    }
    // clear this warp's T slots for the next triangle
#pragma unroll
    for (int v = 0; v < VPL; ++v) {
      const int bl = lane * VPL + v;
      tsm[(0 * kBW + w) * BL + bl] = 0.f;
      tsm[(1 * kBW + w) * BL + bl] = 0.f;
      if (D) {
        tsm[SH::tsm_floats / 2 + (0 * kBW + w) * BL + bl] = 0.f;
        tsm[SH::tsm_floats / 2 + (1 * kBW + w) * BL + bl] = 0.f;
      }
    }
  };

  for (int s = 0; s < NB - 1; ++s) issue_next();
  __syncthreads();  // block descriptors written by thread 0 are visible
  bool open = false;
  int rows_since_flush = 0;

  while (j_cons < j_issue) {
    const int bi = bi_cons;
    const uint32_t parity = ph_cons;
    const int nb = desc_nb[bi];
    const int piece = desc_pc[bi];
    if (piece != piece_c) {
      if (open) flush_triangle();
      const WarpPlan &pl = p.plan[piece];
      for (int j = 0; j < kMaxOrder; ++j) Q[j] = pl.t[j];
      c = pl.t[m - 2];
      pos = pl.start;
      end = pl.end;
      piece_c = piece;
      setup_triangle();
      open = true;
    }
    const int L0 = n - c;
    const int64_t pend = pos + (int64_t)(nb * L0 - (nb * (nb - 1)) / 2);
    const int64_t rb0 = (pos - p.off_lo) * ES;
    const int64_t b0 = rb0 & ~int64_t(15);
    const int64_t rb1 = (pend - p.off_lo) * ES;
    const int64_t b1 = min((rb1 + 15) & ~int64_t(15), tail_lo);
    unsigned char *buf = bufs + (size_t)bi * p.buf_bytes;
    if (b1 > b0) {
      if (!mbar_wait_bounded(&bar[bi], parity)) {
        if (lane == 0) {
          atomicExch(&reinterpret_cast<WsHeader *>(p.status)->status, TK_ETIMEOUT);
          reinterpret_cast<WsHeader *>(p.status)->where = kSiteBatchedWait;
        }
      }
    }
    if (rb1 > tail_lo && threadIdx.x < 16) {
      const int64_t nt = rb1 - max(tail_lo, b0);
      if (threadIdx.x < nt) {
        const int64_t src = max(tail_lo, b0) + threadIdx.x;
        buf[src - b0] = p.K[src];
      }
    }
    ++j_cons;
    if (++bi_cons == NB) {
      bi_cons = 0;
      ph_cons ^= 1u;
    }
    __syncthreads();  // tail bytes visible; the previous block's buffer is free
    issue_next();

    const ST *bp = reinterpret_cast<const ST *>(buf) + (int)((rb0 - b0) / ES);
    int rowend = L0 - 1;
    const float *a_col = a_s + (size_t)(n - 1) * BL + lane * VPL;
    const float *v_col = v_s + (size_t)(n - 1) * BL + lane * VPL;
    for (int r = 0; r < nb; r += 4) {
      N cf[4][VPL], dot[4][VPL];
      int sl[4];
      const ST *prow[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int ri = r + i;
        const bool live = ri < nb;
        sl[i] = live ? L0 - ri - 1 : 0;
        prow[i] = bp + (live ? rowend : L0 - 1);
        rowend += live ? L0 - ri - 1 : 0;
        const int cr = min(c + ri, n - 1);
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
          cf[i][v] = live ? ((cr == b) ? cAf[v] : cA[v]) * alpha_at(cr, lane * VPL + v) : mk<float, D>(0.f, 0.f);
          dot[i][v] = mk<float, D>(0.f, 0.f);
        }
      }
      const int nk = (sl[0] > w) ? (sl[0] - w + kBW - 1) / kBW : 0;
      const ST *pw[4];
      int slw[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        pw[i] = prow[i] - w;
        slw[i] = sl[i] - w;
      }
      const float *acw = a_col - w * BL;
      const float *vcw = v_col - w * BL;
      switch (nk) {
#define TK_BQ(K) \
  case (K) + 1: bquad<K, NCOL, VPL, ST, D>(acc, dot, acw, vcw, pw, slw, cf); [[fallthrough]];
        TK_BQ(47) TK_BQ(46) TK_BQ(45) TK_BQ(44) TK_BQ(43) TK_BQ(42) TK_BQ(41) TK_BQ(40)
        TK_BQ(39) TK_BQ(38) TK_BQ(37) TK_BQ(36) TK_BQ(35) TK_BQ(34) TK_BQ(33) TK_BQ(32)
        TK_BQ(31) TK_BQ(30) TK_BQ(29) TK_BQ(28) TK_BQ(27) TK_BQ(26) TK_BQ(25) TK_BQ(24)
        TK_BQ(23) TK_BQ(22) TK_BQ(21) TK_BQ(20) TK_BQ(19) TK_BQ(18) TK_BQ(17) TK_BQ(16)
        TK_BQ(15) TK_BQ(14) TK_BQ(13) TK_BQ(12) TK_BQ(11) TK_BQ(10) TK_BQ(9) TK_BQ(8)
        TK_BQ(7) TK_BQ(6) TK_BQ(5) TK_BQ(4) TK_BQ(3) TK_BQ(2) TK_BQ(1) TK_BQ(0)
#undef TK_BQ
        default: break;
      }
      // this warp's partial dots of the quad's rows
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int v = 0; v < VPL; ++v) {
          const size_t o = (((size_t)w * 16 + r + i) * BL) * SH::nv + lane * VPL + v;
          red[o] = dot[i][v].v;
          if (D) red[o + BL] = dot[i][v].d;
        }
    }
    __syncthreads();
    // epilogue of each row of the block, by the warp owning the row's own column
    for (int r = 0; r < nb; ++r) {
      const int cr = c + r;
      const int e = n - 1 - cr;
      if ((e % kBW) != w) continue;
      const int head = r * L0 - (r * (r - 1)) / 2;
      const float h = ld_elem<ST, float>(bp + head);
      const bool first = (cr == b);
      const float cnt = first ? (float)(kb + 1) : 1.f;
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const int bl = lane * VPL + v;
        N R = mk<float, D>(0.f, 0.f);
        for (int ww = 0; ww < kBW; ++ww) {
          const size_t o = (((size_t)ww * 16 + r) * BL) * SH::nv + bl;
          R.v += red[o];
          if (D) R.d += red[o + BL];
        }
        const N ac = alpha_at(cr, bl);
        const N Rf = R + scale(h * (first ? inv_first : 0.5f), ac);
        const N gadd = (first ? cAf[v] : cA[v]) * (scale(h, ac) + scale(cnt, R));
        badd_dyn<NCOL, VPL, D>(acc, e / kBW, v, gadd);
        const N tadd = scale(first ? Mf : Mprime, ac * Rf);
        const int slot = ((first ? 1 : 0) * kBW + w) * BL + bl;
        tsm[slot] += tadd.v;
        if (D) tsm[SH::tsm_floats / 2 + slot] += tadd.d;
      }
    }

    c += nb;
    pos = pend;
    rows_since_flush += nb;
    if (c == n) {
      flush_triangle();
      open = false;
      if (pos < end) {
        if (m > 2 && next_sorted(m - 2, n, Q)) {
          c = Q[m - 3];
          setup_triangle();
          open = true;
        }
      }
    }
    if (rows_since_flush >= p.flush_rows) {
      flush_acc();
      rows_since_flush = 0;
    }
  }
  if (open) flush_triangle();
  flush_acc();
  __syncthreads();
  if (threadIdx.x < BL) {
    gp[(size_t)n * BL + threadIdx.x] = ssm[threadIdx.x];
    if (D) gp[(size_t)(n + 2) * BL + (size_t)n * BL + threadIdx.x] = ssm[BL + threadIdx.x];
  }
}

// G[b][d] (and S[b]) = sum over the slices of the block partials, fixed order
__global__ void batched_reduce(int m, int n, int64_t B, int BL, int slices, const double *gpart, int dual,
                               int out_dtype, void *G, double *S, const int *status, int pieces, int64_t lo,
                               int64_t hi) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t b = blockIdx.y;
  if (d > n || (d == n && (dual || !S))) return;
  // the main pass did nothing when its plan key did not match: write nothing
  const volatile WsHeader *wh = reinterpret_cast<const volatile WsHeader *>(status);
  if (!(wh->plan_m == m && wh->plan_n == n && wh->plan_pieces == pieces && wh->plan_lo == lo && wh->plan_hi == hi))
    return;
  const int g = (int)(b / BL), bl = (int)(b % BL);
  const size_t stride = (size_t)2 * (n + 2) * BL;
  const size_t off = (size_t)(dual ? (n + 2) * BL : 0) + (size_t)d * BL + bl;
  double s = 0.0;
  for (int k = 0; k < slices; ++k) s += gpart[(size_t)(g * slices + k) * stride + off];
  if (d == n) {
    S[b] = s;
    return;
  }
  if (dual) s /= (double)(m - 1);
  if (out_dtype == TK_F64) reinterpret_cast<double *>(G)[b * n + d] = s;
  else reinterpret_cast<float *>(G)[b * n + d] = (float)s;
}

template <typename ST, bool D, int VPL, int NCOL>
static int launch_b(const BParams &bp, int grid, size_t smem, cudaStream_t st) {
  auto kern = batched_kernel<ST, D, VPL, NCOL>;
  TK_CUDA_CHECK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, kBT, smem, st>>>(bp);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

template <typename ST, bool D, int VPL>
static int launch_ncol(const BParams &bp, int ncol, int grid, size_t smem, cudaStream_t st) {
  if (ncol <= 8) return launch_b<ST, D, VPL, 8>(bp, grid, smem, st);
  if (ncol <= 12) return launch_b<ST, D, VPL, 12>(bp, grid, smem, st);
  if (ncol <= 16) return launch_b<ST, D, VPL, 16>(bp, grid, smem, st);
  if (ncol <= 20) return launch_b<ST, D, VPL, 20>(bp, grid, smem, st);
  if constexpr (VPL == 1) {
    if (ncol <= 24) return launch_b<ST, D, VPL, 24>(bp, grid, smem, st);
    if (ncol <= 32) return launch_b<ST, D, VPL, 32>(bp, grid, smem, st);
    if (!D && ncol <= 40) return launch_b<ST, D, VPL, 40>(bp, grid, smem, st);
  }
  return fail(TK_EUNSUPPORTED, "batched contraction: n too large");
}

// vectors per lane and column slots per thread for (n, dual)
static bool batched_shape(int n, bool dual, int *vpl, int *ncol) {
  const int nc = (n + kBW - 1) / kBW;
  if (!dual && nc <= 20) {
    *vpl = 2;
    *ncol = nc;
    return true;
  }
  if (nc <= (dual ? 20 : 40)) {
    *vpl = 1;
    *ncol = nc;
    return true;
  }
  return false;
}

// plan records: 16 pieces per slice, slices <= slice_mult (<= 2) * SMs
static size_t batched_plan_bytes(int sms) { return (size_t)16 * 2 * sms * sizeof(WarpPlan); }

size_t batched_workspace_bytes(int n, int64_t B, int sms) {
  // header, plan (16 pieces per slice, at most two slices per SM), partials
  const int BL = 32;  // the smallest group gives the most blocks
  const int64_t groups = (B + BL - 1) / BL;
  const int64_t blocks = std::max<int64_t>(groups, (int64_t)sms) * 2;
  return sizeof(WsHeader) + batched_plan_bytes(sms) + (size_t)blocks * 2 * (n + 2) * 64 * sizeof(double);
}

tk_batched_config g_batched_cfg = {0, 0, 0, 0, 0, 0};

int64_t batched_min_batch(bool dual) {
  return g_batched_cfg.min_batch > 0 ? g_batched_cfg.min_batch : (dual ? 16 : 28);
}

static size_t batched_smem(int n, bool dual, int vpl, int nbuf, int buf_bytes) {
  const int BL = 32 * vpl, nv = dual ? 2 : 1;
  const size_t vec_bytes = ((size_t)nv * n * BL * 4 + 127) & ~size_t(127);
  const size_t fixed = (size_t)(kBW * 16 * BL * nv + 2 * kBW * BL * nv + 2 * BL * nv) * 4 + (size_t)BL * nv * 8 +
                       64 + 64 + 128;
  return vec_bytes + fixed + (size_t)nbuf * buf_bytes;
}

bool batched_resolve(int n, int storage, bool dual, int64_t B, int sms, int smem_optin, tk_batched_config *out) {
  const tk_batched_config &o = g_batched_cfg;
  *out = tk_batched_config{0, 0, 0, 0, (int)batched_min_batch(dual), 0};
  if (storage == TK_F64) return false;
  int vpl = 0, ncol = 0;
  if (!batched_shape(n, dual, &vpl, &ncol)) return false;
  if (o.vpl == 1) vpl = 1;  // vpl 2 only where the shape allows it
  const int es = dtype_size(storage);
  const int min_buf = (n * es + 32 + 127) & ~127;
  int buf = o.block_bytes > 0 ? o.block_bytes : std::max(8192 + 128, min_buf);
  if (buf < min_buf) return false;
  const int nbuf = o.nbuf > 0 ? o.nbuf : 3;
  const int BL = 32 * vpl;
  const int64_t groups = (B + BL - 1) / BL;
  if (groups > (int64_t)sms * 2) return false;
  if (batched_smem(n, dual, vpl, nbuf, buf) > (size_t)smem_optin - 1024) return false;
  out->vpl = vpl;
  out->block_bytes = buf;
  out->nbuf = nbuf;
  out->slice_mult = o.slice_mult > 0 ? o.slice_mult : 1;
  return true;
}

int contract_batched(const BatchedArgs &a, cudaStream_t st) {
  const bool dual = a.V != nullptr;
  if (a.storage == TK_F64) return fail(TK_EUNSUPPORTED, "batched kernel stores FP32/BF16");
  DevInfo di;
  int rc = dev_info(&di);
  if (rc != TK_OK) return rc;
  tk_batched_config cfg;
  if (!batched_resolve(a.n, a.storage, dual, a.B, di.sms, di.smem_optin, &cfg))
    return fail(TK_EUNSUPPORTED, "batched kernel does not cover this shape or configuration");
  int vpl = 0, ncol = 0;
  batched_shape(a.n, dual, &vpl, &ncol);
  vpl = cfg.vpl;
  const int BL = 32 * vpl;
  const int groups = (int)((a.B + BL - 1) / BL);
  const int slices = std::max(1, cfg.slice_mult * di.sms / groups);
  const int grid = groups * slices;
  const int es = dtype_size(a.storage);
  const int nv = dual ? 2 : 1;
  BParams bp;
  bp.m = a.m;
  bp.n = a.n;
  bp.K = reinterpret_cast<const unsigned char *>(a.K);
  bp.off_lo = a.off_lo;
  bp.off_hi = a.off_hi;
  bp.bytes = (a.off_hi - a.off_lo) * es;
  bp.A = a.A;
  bp.V = a.V;
  bp.vec_dtype = a.vec_dtype;
  bp.B = a.B;
  bp.groups = groups;
  bp.slices = slices;
  bp.pieces = 16 * slices;
  bp.nbuf = cfg.nbuf;
  bp.buf_bytes = cfg.block_bytes;
  bp.cap = (cfg.block_bytes - 32) / es;
  bp.flush_rows = 2048;
  bp.vec_bytes = (int)(((size_t)nv * a.n * BL * 4 + 127) & ~size_t(127));
  const size_t smem = batched_smem(a.n, dual, vpl, bp.nbuf, bp.buf_bytes);
  unsigned char *ws = reinterpret_cast<unsigned char *>(a.work);
  const size_t plan_bytes = batched_plan_bytes(di.sms);
  if ((size_t)bp.pieces * sizeof(WarpPlan) > plan_bytes)
    return fail(TK_EINVAL, "batched plan of %d pieces exceeds its workspace region", bp.pieces);
  const size_t part_bytes = (size_t)grid * 2 * (a.n + 2) * BL * sizeof(double);
  if (sizeof(WsHeader) + plan_bytes + part_bytes > a.work_bytes) return fail(TK_ENOMEM, "batched workspace too small");
  WarpPlan *plan = reinterpret_cast<WarpPlan *>(ws + sizeof(WsHeader));
  bp.plan = plan;
  bp.gpart = reinterpret_cast<double *>(ws + sizeof(WsHeader) + plan_bytes);
  bp.status = reinterpret_cast<int *>(ws);
  rc = plan_to_device(a.m, a.n, a.off_lo, a.off_hi, bp.pieces, 256, 1024, a.work, st);
  if (rc != TK_OK) return rc;
  if (a.storage == TK_F32) {
    rc = dual ? launch_ncol<float, true, 1>(bp, ncol, grid, smem, st)
              : (vpl == 2 ? launch_ncol<float, false, 2>(bp, ncol, grid, smem, st)
                          : launch_ncol<float, false, 1>(bp, ncol, grid, smem, st));
  } else {
    rc = dual ? launch_ncol<__nv_bfloat16, true, 1>(bp, ncol, grid, smem, st)
              : (vpl == 2 ? launch_ncol<__nv_bfloat16, false, 2>(bp, ncol, grid, smem, st)
                          : launch_ncol<__nv_bfloat16, false, 1>(bp, ncol, grid, smem, st));
  }
  if (rc != TK_OK) return rc;
  dim3 rg((unsigned)((a.n + 1 + 127) / 128), (unsigned)a.B);
  batched_reduce<<<rg, 128, 0, st>>>(a.m, a.n, a.B, BL, slices, bp.gpart, dual ? 1 : 0, a.vec_dtype, a.G, a.S,
                                     bp.status, bp.pieces, a.off_lo, a.off_hi);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

}  // namespace tk
