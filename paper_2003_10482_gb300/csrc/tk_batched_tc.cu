// Batched packed contraction on the 5th-generation tensor cores: K[a_b^{m-1}]
// and K[a_b^m] for B dual vectors in one launch (r = m-1), the passes of a
// batched dual solve over a lambda path x cross-validation folds (Section 4,
// eq. dual_tensor_kernel, for many a at once).
//
// What is computed is the contraction of the single-vector and SIMT batched
// kernels; the per-triangle decomposition the tensor cores take is in
// tk_tc_math.h: for every triangle Q the weighted symmetric row dots
// Rf_c = sum_d S_Q[c][d] f_d a_d of all vectors form one product
//   R (vectors x rows) = A (vectors x d) . S~_Q^T (d x rows),
// and an epilogue turns R into the g and S contributions.
//
// GB300 mapping.  A block (416 threads, one per SM: it holds all 512 columns
// of tensor memory) owns a slice of 128 vectors -- tensor-memory lane i is
// vector i of the slice -- and a contiguous range of jobs; a job is up to 96
// rows of one triangle (rows c in [cs, cs + 96), cs a multiple of 16).  The
// block is a warp-specialised pipeline connected by mbarriers:
//   * warps 4-11 walk the jobs chunk by 32-wide chunk of the column index d:
//     they gather the chunk of S~_Q's rows from the packed triangle -- entry
//     (c, d) from row min(c, d), lanes running along whichever index is
//     contiguous in memory -- weight column b, split it into TF32 hi/lo and
//     store both in the K-major 128-byte-swizzled layout of one of 3 ring
//     stages; their first thread also starts the cp.async.bulk of the slice's
//     vectors for the chunk (pre-split into TF32 hi and lo and pre-swizzled:
//     a 32 KB image written once per pass) into the same stage;
//   * one thread of warp 12 waits for a stage, issues 4 k-steps x 3
//     tcgen05.mma (hi.hi + hi.lo + lo.hi; M = 128 vectors, N = the job's
//     rows, K = 8) into one of two alternating job accumulators and commits
//     the stage back to the gatherers, and the accumulator to the epilogue at
//     the job's end;
//   * warps 0-3 read the accumulator (tcgen05.ld), hand it back, add
//     A_Q (M'/m) Rf_c into the block's g accumulator -- 128 x n FP32 values in
//     tensor memory, column c, each thread its own lane -- and carry the
//     triangle's quadratic-form sum; the triangle's last job adds its S and
//     prefix-value terms.  Every 128 jobs the g accumulator is added into the
//     block's FP64 partial (bounded FP32 summation depth); a second kernel
//     sums the partials in a fixed order.
#include <cuda_bf16.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tk_tc_math.h"
#include "tk_umma.cuh"

namespace tk {

constexpr int kTcEpiWarps = 4;       // warps 0-3: epilogue, thread i <-> tensor-memory lane i <-> vector i
constexpr int kTcGatherWarps = 8;    // warps 4-11: gather the rows of S~_Q into the stage ring
constexpr int kTcGatherThreads = 32 * kTcGatherWarps;
constexpr int kTcThreads = 32 * (kTcEpiWarps + kTcGatherWarps + 1);  // + warp 12: issues the MMAs
constexpr int kTcSlice = 128;        // vectors per block (M of the MMA)
constexpr int kTcMaxN = 320;         // g accumulator columns left beside the two job accumulators
constexpr int kTcFlushJobs = 128;    // jobs between FP64 flushes of the g accumulator
constexpr uint32_t kTcAccCols = 96;  // tensor-memory columns: [0, 96) and [96, 192) the two job accumulators,
constexpr uint32_t kTcAColsG = 192;  // [192, 192 + n16) the g accumulator
constexpr int kTcStages = 3;         // ring of stages, each: vectors' chunk (hi, lo) + rows' chunk (hi, lo)
constexpr int kTcAPart = 16384;      // 128 vectors x 32 values x 4 bytes
constexpr int kTcAStage = 2 * kTcAPart;
constexpr int kTcBPart = tc::kRowsPerJob * 128;  // one part (hi or lo) of a row chunk
constexpr int kTcStageBytes = kTcAStage + 2 * kTcBPart;

struct TcJob {
  int32_t tri;
  int16_t cs;     // first row of the job (a multiple of 16)
  int16_t npad;   // rows, rounded up to 16 (N of the MMA)
  int16_t kc0;    // first 32-column chunk (floor(max(b, 0) / 32))
  int16_t flags;  // 1: first job of its triangle, 2: last
  int32_t pad;
};
static_assert(sizeof(TcJob) == 16, "job record");

struct TcTri {
  int64_t base;           // packed offset of the triangle's first entry (b, b)
  int32_t b;              // last prefix value (-1 for m = 2)
  int16_t kb;             // cnt_Q(b)
  int16_t nq;             // m - 2
  int32_t mprime;         // m! / prod_v cnt_Q(v)!
  uint16_t q[kMaxOrder - 2];
};
static_assert(sizeof(TcTri) == 32, "triangle record");

struct TcParams {
  int m, n, n16, nkc;   // order, points, n rounded up to 16, 32-column chunks
  const unsigned char *K;
  const TcJob *jobs;
  const TcTri *tris;
  const int *range;     // P + 1 job bounds
  int P, slices, Bpad;
  const float *img;     // [slice][chunk][hi, lo][128 x 32 swizzled]
  const float *at;      // n x Bpad, a[b][d] at [d][b]
  double *gpart;        // [block][n16][128]
  double *spart;        // [block][128]
  int *status;
};

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15, %16};" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])),
      "r"(__float_as_uint(v[11])), "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])),
      "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

template <typename ST>
__device__ __forceinline__ float ld_entry(const unsigned char *K, int64_t off) {
  return ld_elem<ST, float>(reinterpret_cast<const ST *>(K) + off);
}

// Gather rows [cs, cs + npad) x columns [d0, d0 + 32) of S~_Q into the
// swizzled hi/lo tiles.  A thread takes 4 consecutive columns of a row (one
// 16-byte chunk of the tile) in each 32-row sub-block.  Sub-blocks wholly
// below the diagonal put the lanes along the rows (entry (c, d) with d < c
// sits in stored row d, consecutive c contiguous); the others along the
// columns (8 lanes per row, consecutive d contiguous).  The in-triangle
// offset (r - bb)(2n - bb - r + 1)/2 + (s - r), r = min(c, d), s = max(c, d),
// fits 32 bits (n <= 320).  All loads are issued before the first is used.
template <typename ST>
__device__ __forceinline__ void stage_rows(const TcParams &p, const TcTri &tri, int cs, int npad, int d0,
                                           unsigned char *bhi, unsigned char *blo, int t) {
  constexpr int kSub = tc::kRowsPerJob / 32;
  const int n = p.n, b = tri.b, bb = b < 0 ? 0 : b;
  const int span = 2 * n - bb + 1;
  const ST *__restrict__ Kt = reinterpret_cast<const ST *>(p.K) + tri.base;
  float x[kSub][4];
#pragma unroll
  for (int sb = 0; sb < kSub; ++sb) {
    const int jb = 32 * sb;
    const bool lower = d0 + 31 < cs + jb;   // every column below every row of the sub-block
    const bool upper = d0 >= cs + jb + 31;  // every column at or above every row
    const int j = lower ? jb + (t & 31) : jb + (t >> 3);
    const int k4 = lower ? 4 * (t >> 5) : 4 * (t & 7);
    const int c = cs + j, d = d0 + k4;
    if (lower) {
      // entries (d + e, c) of stored rows d + e: row d + 1 starts n - d after row d
      int off = (((d - bb) * (span - d)) >> 1) + (c - d);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const bool ok = j < npad && d + e >= bb && c < n;
        x[sb][e] = ok ? ld_elem<ST, float>(Kt + off) : 0.f;
        off += n - d - e - 1;
      }
    } else if (upper) {
      // entries (c, d + e), consecutive in stored row c
      const int off = (((c - bb) * (span - c)) >> 1) + (d - c);
      const bool okr = j < npad && c >= bb;
#pragma unroll
      for (int e = 0; e < 4; ++e) x[sb][e] = (okr && d + e < n) ? ld_elem<ST, float>(Kt + off + e) : 0.f;
    } else {
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int de = d + e;
        const int r = min(c, de), s2 = max(c, de);
        const bool ok = j < npad && r >= bb && s2 < n;
        const int off = (((r - bb) * (span - r)) >> 1) + (s2 - r);
        x[sb][e] = ok ? ld_elem<ST, float>(Kt + off) : 0.f;
      }
    }
  }
  const float fb = kInvSmall<float>[tri.kb + 1];
  const bool has_b = b >= d0 && b < d0 + 32;
#pragma unroll
  for (int sb = 0; sb < kSub; ++sb) {
    const int jb = 32 * sb;
    if (jb >= npad) break;
    const bool lower = d0 + 31 < cs + jb;
    const int j = lower ? jb + (t & 31) : jb + (t >> 3);
    const int k4 = lower ? 4 * (t >> 5) : 4 * (t & 7);
    if (j >= npad) continue;
    float h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float v = x[sb][e];
      if (has_b && d0 + k4 + e == b) v *= fb;
      umma::split_tf32(v, h[e], l[e]);
    }
    const uint32_t so = umma::sw128_offset((uint32_t)j, (uint32_t)k4);
    *reinterpret_cast<float4 *>(bhi + so) = make_float4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<float4 *>(blo + so) = make_float4(l[0], l[1], l[2], l[3]);
  }
}

// Bounded wait on an mbarrier phase; once any wait of the block has run out
// every later wait returns false at once, so all roles leave their loops.
__device__ __forceinline__ bool tc_wait(uint64_t *bar, uint32_t parity, volatile int *bad) {
  if (*bad) return false;
  if (mbar_wait_bounded(bar, parity)) return true;
  *bad = 1;
  return false;
}

template <typename ST>
__global__ void __launch_bounds__(kTcThreads, 1) tc_batched_kernel(TcParams p) {
  extern __shared__ unsigned char tc_smem_raw[];
  // ring: full (gathered rows written: 256 arrivals), afull (vectors' chunk
  // landed: the bulk copy's bytes), empty (the MMAs that read the stage are
  // done: a commit); job accumulators: accf (a job's MMAs are done: a
  // commit), acce (the epilogue has read the accumulator: 128 arrivals)
  __shared__ uint64_t bar_full[kTcStages], bar_afull[kTcStages], bar_empty[kTcStages], bar_accf[2], bar_acce[2];
  __shared__ uint32_t tbase;
  __shared__ int s_bad;
  if (plan_is_stale(p.status, p.m, p.n, p.P, -2, -2)) return;
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) &
                                                        ~uintptr_t(1023));
  const int tid = threadIdx.x, w = tid >> 5;
  const int m = p.m, n = p.n;
  const int slice = blockIdx.x / p.P, part = blockIdx.x % p.P;
  const int j_lo = p.range[part], j_hi = p.range[part + 1];
  if (w == 0) {
    umma::tmem_alloc(&tbase, 512);
    umma::tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kTcStages; ++s) {
      mbar_init(&bar_full[s], kTcGatherThreads);
      mbar_init(&bar_afull[s], 1);
      mbar_init(&bar_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bar_accf[b], 1);
      mbar_init(&bar_acce[b], 32 * kTcEpiWarps);
    }
    fence_barrier_init();
    s_bad = 0;
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  volatile int *bad = &s_bad;

  if (w < kTcEpiWarps) {
    // ---------------------------------------------------------------- epilogue
    const int vl = tid;  // vector of the slice = tensor-memory lane
    const int beta = slice * kTcSlice + vl;
    const uint32_t tl = tbase + ((uint32_t)(32 * w) << 16);
    const uint32_t tG = tl + kTcAColsG;
    const float zero16[16] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int c0 = 0; c0 < p.n16; c0 += 16) tmem_st16(tG + c0, zero16);
    tmem_wait_st();
    double *gp = p.gpart + (size_t)blockIdx.x * p.n16 * kTcSlice;
    for (int c = 0; c < n; ++c) gp[(size_t)c * kTcSlice + vl] = 0.0;
    const float *atb = p.at + beta;  // a[beta][d] at atb[d * Bpad]
    const float inv_m = 1.f / (float)m;
    double S64 = 0.0;
    float Sacc = 0.f, P1 = 0.f, Rfb = 0.f;
    int since_flush = 0;
    auto flush = [&]() {
      for (int c0 = 0; c0 < p.n16; c0 += 16) {
        float g[16];
        double old[16];
        umma::tmem_ld16(tG + c0, g);
#pragma unroll
        for (int i = 0; i < 16; ++i) old[i] = c0 + i < n ? gp[(size_t)(c0 + i) * kTcSlice + vl] : 0.0;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (c0 + i < n) gp[(size_t)(c0 + i) * kTcSlice + vl] = old[i] + (double)g[i];
        tmem_st16(tG + c0, zero16);
      }
      tmem_wait_st();
      S64 += (double)Sacc;
      Sacc = 0.f;
    };
    int jl = 0;
    for (int jx = j_lo; jx < j_hi; ++jx, ++jl) {
      const TcJob job = p.jobs[jx];
      const TcTri tri = p.tris[job.tri];
      const int b = tri.b, cs = job.cs, npad = job.npad;
      const int buf = jl & 1;
      float AQ = 1.f;
      for (int j = 0; j < tri.nq; ++j) AQ *= atb[(size_t)tri.q[j] * p.Bpad];
      const float mprime = (float)tri.mprime;
      const float coef = AQ * mprime * inv_m;
      if (!tc_wait(&bar_accf[buf], (uint32_t)(jl >> 1) & 1u, bad)) break;
      umma::fence_after_sync();
      const uint32_t tR = tl + (uint32_t)buf * kTcAccCols;
      for (int j0 = 0; j0 < npad; j0 += 16) {
        float av[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = cs + j0 + i;
          av[i] = (c > b && c < n) ? atb[(size_t)c * p.Bpad] : 0.f;
        }
        uint32_t ur[16], ug[16];
        umma::tmem_ld16_async(tR + j0, ur);
        umma::tmem_ld16_async(tG + cs + j0, ug);
        umma::tmem_wait_ld();
        float g[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float r = __uint_as_float(ur[i]);
          g[i] = __uint_as_float(ug[i]) + coef * r;
          P1 += av[i] * r;
          if (cs + j0 + i == b) Rfb = r;
        }
        tmem_st16(tG + cs + j0, g);
      }
      tmem_wait_st();
      umma::fence_before_sync();
      mbar_arrive(&bar_acce[buf]);  // this accumulator may take the job after next
      if (job.flags & 2) {
        const float hb = b >= 0 ? ld_entry<ST>(p.K, tri.base) : 0.f;
        const float ab = b >= 0 ? atb[(size_t)b * p.Bpad] : 0.f;
        float T, Tr;
        tc::finish_triangle<float>(b, tri.kb, mprime, P1, Rfb, hb, ab, &T, &Tr);
        Sacc += AQ * T;
        // prefix-value terms: g_l += (cnt_Q(l)/m) B_{Q,l} (l == b ? T_rest : T)
        for (int j = 0; j < tri.nq; ++j) {
          if (j > 0 && tri.q[j] == tri.q[j - 1]) continue;
          const int l = tri.q[j];
          int cnt = 0;
          float Bl = 1.f;
          bool skipped = false;
          for (int jj = 0; jj < tri.nq; ++jj) {
            if (tri.q[jj] == l) {
              ++cnt;
              if (!skipped) {
                skipped = true;
                continue;
              }
            }
            Bl *= atb[(size_t)tri.q[jj] * p.Bpad];
          }
          const float add = (float)cnt * inv_m * Bl * (l == b ? Tr : T);
          float g[16];
          const int l0 = l & ~15;
          umma::tmem_ld16(tG + l0, g);
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (i == (l & 15)) g[i] += add;
          tmem_st16(tG + l0, g);
          tmem_wait_st();
        }
        P1 = 0.f;
        Rfb = 0.f;
      }
      if (++since_flush == kTcFlushJobs) {
        flush();
        since_flush = 0;
      }
    }
    flush();
    p.spart[(size_t)blockIdx.x * kTcSlice + vl] = S64;
  } else if (w < kTcEpiWarps + kTcGatherWarps) {
    // ---------------------------------------------------------------- gather
    const int gt = tid - 32 * kTcEpiWarps;
    uint32_t gc = 0;
    for (int jx = j_lo; jx < j_hi; ++jx) {
      const TcJob job = p.jobs[jx];
      const TcTri tri = p.tris[job.tri];
      bool ok = true;
      for (int kc = job.kc0; kc < p.nkc; ++kc, ++gc) {
        const int s = (int)(gc % kTcStages);
        const uint32_t use = gc / kTcStages;
        if (use > 0 && !tc_wait(&bar_empty[s], (use - 1) & 1u, bad)) {
          ok = false;
          break;
        }
        unsigned char *st = sm + s * kTcStageBytes;
        if (gt == 0) {
          mbar_expect_tx(&bar_afull[s], kTcAStage);
          bulk_g2s(st, p.img + ((size_t)slice * p.nkc + kc) * (kTcAStage / 4), kTcAStage, &bar_afull[s]);
        }
        stage_rows<ST>(p, tri, job.cs, job.npad, 32 * kc, st + kTcAStage, st + kTcAStage + kTcBPart, gt);
        fence_proxy_async();  // the rows written above become visible to the tensor cores
        mbar_arrive(&bar_full[s]);
      }
      if (!ok) break;
    }
  } else if ((tid & 31) == 0) {
    // ---------------------------------------------------------------- MMA issue
    uint32_t gc = 0;
    int jl = 0;
    const uint32_t idesc_base = umma::idesc_tf32(kTcSlice, 16) & ~(0x3Fu << 17);
    for (int jx = j_lo; jx < j_hi; ++jx, ++jl) {
      const TcJob job = p.jobs[jx];
      const int buf = jl & 1;
      if (jl >= 2 && !tc_wait(&bar_acce[buf], (uint32_t)((jl >> 1) - 1) & 1u, bad)) break;
      umma::fence_after_sync();
      const uint32_t tR = tbase + (uint32_t)buf * kTcAccCols;
      const uint32_t idesc = idesc_base | ((uint32_t)(job.npad >> 3) << 17);
      bool ok = true;
      for (int kc = job.kc0; kc < p.nkc; ++kc, ++gc) {
        const int s = (int)(gc % kTcStages);
        const uint32_t par = (gc / kTcStages) & 1u;
        if (!tc_wait(&bar_full[s], par, bad) || !tc_wait(&bar_afull[s], par, bad)) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        const uint32_t a0 = saddr(sm + s * kTcStageBytes), b0 = a0 + kTcAStage;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t ah = umma::desc_sw128(a0 + 32 * ks), al = umma::desc_sw128(a0 + kTcAPart + 32 * ks);
          const uint64_t bh = umma::desc_sw128(b0 + 32 * ks), bl = umma::desc_sw128(b0 + kTcBPart + 32 * ks);
          umma::mma_tf32(tR, ah, bh, idesc, (kc > job.kc0 || ks > 0) ? 1u : 0u);
          umma::mma_tf32(tR, ah, bl, idesc, 1u);
          umma::mma_tf32(tR, al, bh, idesc, 1u);
        }
        umma::mma_commit(&bar_empty[s]);
      }
      umma::mma_commit(&bar_accf[buf]);  // the epilogue may read this job's accumulator
      if (!ok) break;
    }
    // nothing may still write tensor memory when it is released
    if (jl > 0) mbar_wait_bounded(&bar_accf[(jl - 1) & 1], (uint32_t)((jl - 1) >> 1) & 1u);
  }
  umma::fence_before_sync();
  __syncthreads();
  if (w == 0) umma::tmem_dealloc(tbase, 512);
  if (tid == 0 && s_bad) {
    atomicExch(&reinterpret_cast<WsHeader *>(p.status)->status, TK_ETIMEOUT);
    reinterpret_cast<WsHeader *>(p.status)->where = kSiteTcWait;
  }
}

// The vectors' image: per slice and 32-column chunk the TF32 hi and lo parts
// in the swizzled layout the MMA reads, and a transposed FP32 copy.
__global__ void tc_prep_vectors(int n, int nkc, int64_t B, int Bpad, int vec_dtype, const void *A, float *img,
                                float *at) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // over Bpad x (32 nkc)
  const int cols = 32 * nkc;
  if (i >= (int64_t)Bpad * cols) return;
  const int beta = (int)(i / cols), d = (int)(i % cols);
  float x = 0.f;
  if (beta < B && d < n)
    x = vec_dtype == TK_F64 ? (float)reinterpret_cast<const double *>(A)[(size_t)beta * n + d]
                            : reinterpret_cast<const float *>(A)[(size_t)beta * n + d];
  float hi, lo;
  umma::split_tf32(x, hi, lo);
  const int slice = beta / kTcSlice, row = beta % kTcSlice, kc = d / 32, k = d % 32;
  float *blk = img + ((size_t)slice * nkc + kc) * (kTcAStage / 4);
  const uint32_t so = umma::sw128_offset((uint32_t)row, (uint32_t)k) / 4;
  blk[so] = hi;
  blk[4096 + so] = lo;
  if (d < n) at[(size_t)d * Bpad + beta] = x;
}

// G[b][c] and S[b]: the blocks' partials of b's slice, summed in a fixed order.
__global__ void tc_reduce(int m, int n, int n16, int64_t B, int P, const double *gpart, const double *spart,
                          int out_dtype, void *G, double *S, const int *status) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t b = blockIdx.y;
  if (c > n || (c == n && !S)) return;
  const volatile WsHeader *wh = reinterpret_cast<const volatile WsHeader *>(status);
  if (!(wh->plan_m == m && wh->plan_n == n && wh->plan_pieces == P && wh->plan_lo == -2 && wh->plan_hi == -2))
    return;
  const int slice = (int)(b / kTcSlice), bl = (int)(b % kTcSlice);
  double s = 0.0;
  if (c == n) {
    for (int k = 0; k < P; ++k) s += spart[(size_t)(slice * P + k) * kTcSlice + bl];
    S[b] = s;
    return;
  }
  for (int k = 0; k < P; ++k) s += gpart[((size_t)(slice * P + k) * n16 + c) * kTcSlice + bl];
  if (out_dtype == TK_F64) reinterpret_cast<double *>(G)[b * n + c] = s;
  else reinterpret_cast<float *>(G)[b * n + c] = (float)s;
}

// ------------------------------------------------------------------ host
struct TcPlan {
  std::vector<TcTri> tris;
  std::vector<TcJob> jobs;
  std::vector<int> range;  // P + 1
};

static void build_tc_plan(int m, int n, int P, TcPlan *out) {
  out->tris.clear();
  out->jobs.clear();
  const int nkc = (n + 31) / 32;
  int32_t Q[kMaxOrder] = {0};
  int64_t base = 0;
  uint64_t mfact = 1;
  for (int i = 2; i <= m; ++i) mfact *= (uint64_t)i;
  std::vector<int64_t> cost;
  for (;;) {
    TcTri t;
    memset(&t, 0, sizeof(t));
    t.base = base;
    uint64_t mp = mfact;
    int run = 0;
    for (int j = 0; j < m - 2; ++j) {
      run = (j > 0 && Q[j] == Q[j - 1]) ? run + 1 : 1;
      if (run > 1) mp = exact_div_small(mp, run);
      t.q[j] = (uint16_t)Q[j];
    }
    t.b = m > 2 ? Q[m - 3] : -1;
    t.kb = (int16_t)(m > 2 ? run : 0);
    t.nq = (int16_t)(m - 2);
    t.mprime = (int32_t)mp;
    const int bb = t.b < 0 ? 0 : t.b;
    const int cs0 = bb & ~15;
    for (int cs = cs0; cs < n; cs += tc::kRowsPerJob) {
      TcJob jb;
      memset(&jb, 0, sizeof(jb));
      jb.tri = (int32_t)out->tris.size();
      jb.cs = (int16_t)cs;
      const int rows = std::min(tc::kRowsPerJob, n - cs);
      jb.npad = (int16_t)((rows + 15) & ~15);
      jb.kc0 = (int16_t)(bb >> 5);
      jb.flags = (int16_t)((cs == cs0 ? 1 : 0) | (cs + tc::kRowsPerJob >= n ? 2 : 0));
      out->jobs.push_back(jb);
      cost.push_back((int64_t)jb.npad * 32 * (nkc - jb.kc0) + 2048 + 16 * jb.npad);
    }
    out->tris.push_back(t);
    const int L = n - bb;
    base += (int64_t)L * (L + 1) / 2;
    if (m <= 2 || !next_sorted(m - 2, n, Q)) break;
  }
  // cut into P ranges of near-equal cost, only between triangles (a
  // triangle's jobs carry its quadratic-form sum from one to the next)
  int64_t total = 0;
  for (int64_t c : cost) total += c;
  out->range.assign(P + 1, 0);
  int64_t acc = 0;
  int k = 1;
  for (size_t j = 0; j < cost.size() && k < P; ++j) {
    acc += cost[j];
    const bool boundary = j + 1 == cost.size() || (out->jobs[j + 1].flags & 1);
    while (boundary && k < P && acc * P >= total * k) out->range[k++] = (int)(j + 1);
  }
  for (; k < P; ++k) out->range[k] = (int)cost.size();
  out->range[P] = (int)cost.size();
}

struct TcKey {
  int m, n, P;
  bool operator<(const TcKey &o) const { return std::tie(m, n, P) < std::tie(o.m, o.n, o.P); }
};
static std::mutex g_tcmu;
static std::map<TcKey, TcPlan> g_tcplans;
static std::map<std::pair<int, const void *>, TcKey> g_tcup;

void forget_tc_plan(void *work) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(g_tcmu);
  g_tcup.erase({dev, work});
}

static const TcPlan &tc_plan_for(int m, int n, int P) {
  TcKey k{m, n, P};
  auto it = g_tcplans.find(k);
  if (it == g_tcplans.end()) {
    if (g_tcplans.size() > 8) g_tcplans.clear();
    TcPlan pl;
    build_tc_plan(m, n, P, &pl);
    it = g_tcplans.emplace(k, std::move(pl)).first;
  }
  return it->second;
}

// grid shape: slices of 128 vectors, P blocks (job ranges) per slice
static void tc_shape(int64_t B, int sms, int *slices, int *P) {
  *slices = (int)((B + kTcSlice - 1) / kTcSlice);
  *P = std::max(1, sms / *slices);
}

struct TcLayout {
  size_t jobs, tris, range, img, at, gpart, spart, total;
};
static TcLayout tc_layout(int n, int64_t B, int sms, size_t njobs, size_t ntris) {
  auto al = [](size_t x) { return (x + 1023) & ~size_t(1023); };
  int slices = 0, P = 0;
  tc_shape(B, sms, &slices, &P);
  const int nkc = (n + 31) / 32, n16 = (n + 15) & ~15;
  const int Bpad = slices * kTcSlice, grid = slices * P;
  TcLayout L;
  size_t off = al(sizeof(WsHeader));
  L.jobs = off;
  off = al(off + njobs * sizeof(TcJob));
  L.tris = off;
  off = al(off + ntris * sizeof(TcTri));
  L.range = off;
  off = al(off + (size_t)(P + 1) * sizeof(int));
  L.img = off;
  off = al(off + (size_t)slices * nkc * kTcAStage);
  L.at = off;
  off = al(off + (size_t)n * Bpad * sizeof(float));
  L.gpart = off;
  off = al(off + (size_t)grid * n16 * kTcSlice * sizeof(double));
  L.spart = off;
  off = al(off + (size_t)grid * kTcSlice * sizeof(double));
  L.total = off;
  return L;
}

// Number of jobs and triangles of (m, n) without building the plan.
static void tc_counts(int m, int n, size_t *njobs, size_t *ntris) {
  // triangles with last prefix value b: C(b + m - 3, m - 3); each has
  // ceil((n - cs0) / 96) jobs, cs0 = floor16(b)
  size_t nj = 0, nt = 0;
  if (m == 2) {
    *ntris = 1;
    *njobs = (size_t)((n + tc::kRowsPerJob - 1) / tc::kRowsPerJob);
    return;
  }
  for (int b = 0; b < n; ++b) {
    const int64_t cnt = multiset(b + 1, m - 3);  // sorted (m-3)-tuples over [0, b]
    const int cs0 = b & ~15;
    nt += (size_t)cnt;
    nj += (size_t)cnt * (size_t)((n - cs0 + tc::kRowsPerJob - 1) / tc::kRowsPerJob);
  }
  *njobs = nj;
  *ntris = nt;
}

bool tc_covers(int m, int n, int storage, bool dual, int64_t B, int64_t off_lo, int64_t off_hi) {
  const int mode = g_batched_cfg.tensor_cores;
  if (mode < 0 || dual || storage == TK_F64) return false;
  if (off_lo != 0 || off_hi != multiset(n, m)) return false;  // whole tensor only
  if (n > kTcMaxN || m > kMaxOrder) return false;
  // where it was measured to win (GB300, m = 4, n = 300, FP32 and BF16: 2.7x
  // the SIMT batched kernel at B = 128, 3.3x at B = 512)
  if (mode == 0 && !(m >= 3 && m <= 4 && n >= 64 && B >= 64)) return false;
  return true;
}

size_t tc_workspace_bytes(int m, int n, int64_t B, int sms) {
  size_t nj = 0, nt = 0;
  tc_counts(m, n, &nj, &nt);
  return tc_layout(n, B, sms, nj, nt).total;
}

int contract_batched_tc(const BatchedArgs &a, cudaStream_t st) {
  DevInfo di;
  int rc = dev_info(&di);
  if (rc != TK_OK) return rc;
  int major = 0, dev = 0;
  TK_CUDA_CHECK(cudaGetDevice(&dev));
  TK_CUDA_CHECK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  if (major != 10) return fail(TK_EUNSUPPORTED, "tensor-core batched contraction needs compute capability 10.x");
  const int m = a.m, n = a.n;
  int slices = 0, P = 0;
  tc_shape(a.B, di.sms, &slices, &P);
  const int nkc = (n + 31) / 32, n16 = (n + 15) & ~15, Bpad = slices * kTcSlice, grid = slices * P;
  const size_t smem = 1024 + (size_t)kTcStages * kTcStageBytes;
  if (smem > (size_t)di.smem_optin) return fail(TK_EUNSUPPORTED, "tensor-core batched kernel: shared memory");
  unsigned char *ws = reinterpret_cast<unsigned char *>(a.work);
  size_t njobs = 0, ntris = 0;
  tc_counts(m, n, &njobs, &ntris);
  const TcLayout L = tc_layout(n, a.B, di.sms, njobs, ntris);
  if (a.work_bytes < L.total) return fail(TK_ENOMEM, "workspace %zu < %zu bytes (tensor-core batched pass)",
                                          a.work_bytes, L.total);
  bool uploaded = false;
  {
  std::lock_guard<std::mutex> lk(g_tcmu);
  TcKey key{m, n, P};
  auto up = g_tcup.find({dev, a.work});
  if (up == g_tcup.end() || up->second < key || key < up->second) {
    const TcPlan &pl = tc_plan_for(m, n, P);
    if (pl.jobs.size() != njobs || pl.tris.size() != ntris)
      return fail(TK_EINVAL, "tensor-core plan: %zu jobs / %zu triangles, layout sized for %zu / %zu",
                  pl.jobs.size(), pl.tris.size(), njobs, ntris);
    TK_CUDA_CHECK(cudaMemcpyAsync(ws + L.jobs, pl.jobs.data(), pl.jobs.size() * sizeof(TcJob),
                                  cudaMemcpyHostToDevice, st));
    TK_CUDA_CHECK(cudaMemcpyAsync(ws + L.tris, pl.tris.data(), pl.tris.size() * sizeof(TcTri),
                                  cudaMemcpyHostToDevice, st));
    TK_CUDA_CHECK(cudaMemcpyAsync(ws + L.range, pl.range.data(), pl.range.size() * sizeof(int),
                                  cudaMemcpyHostToDevice, st));
    const WsHeader h = plan_key(m, n, -2, -2, P);
    TK_CUDA_CHECK(cudaMemcpyAsync(ws + offsetof(WsHeader, plan_m),
                                  reinterpret_cast<const unsigned char *>(&h) + offsetof(WsHeader, plan_m),
                                  offsetof(WsHeader, pad) - offsetof(WsHeader, plan_m), cudaMemcpyHostToDevice, st));
    TK_CUDA_CHECK(cudaStreamSynchronize(st));  // the host plan lives in a cache that may be rebuilt
    g_tcup[{dev, a.work}] = key;
    uploaded = true;
  }
  }
  if (uploaded) {  // the other kernels' plan regions overlap this one
    forget_plan(a.work);
    forget_hessian_plan(a.work);
  }
  TcParams p;
  p.m = m;
  p.n = n;
  p.n16 = n16;
  p.nkc = nkc;
  p.K = reinterpret_cast<const unsigned char *>(a.K);
  p.jobs = reinterpret_cast<const TcJob *>(ws + L.jobs);
  p.tris = reinterpret_cast<const TcTri *>(ws + L.tris);
  p.range = reinterpret_cast<const int *>(ws + L.range);
  p.P = P;
  p.slices = slices;
  p.Bpad = Bpad;
  p.img = reinterpret_cast<const float *>(ws + L.img);
  p.at = reinterpret_cast<const float *>(ws + L.at);
  p.gpart = reinterpret_cast<double *>(ws + L.gpart);
  p.spart = reinterpret_cast<double *>(ws + L.spart);
  p.status = reinterpret_cast<int *>(ws);
  {
    const int64_t total = (int64_t)Bpad * 32 * nkc;
    tc_prep_vectors<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(n, nkc, a.B, Bpad, a.vec_dtype, a.A,
                                                                     reinterpret_cast<float *>(ws + L.img),
                                                                     reinterpret_cast<float *>(ws + L.at));
    TK_CUDA_CHECK(cudaGetLastError());
  }
  if (a.storage == TK_F32) {
    TK_CUDA_CHECK(cudaFuncSetAttribute(tc_batched_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    tc_batched_kernel<float><<<grid, kTcThreads, smem, st>>>(p);
  } else {
    TK_CUDA_CHECK(cudaFuncSetAttribute(tc_batched_kernel<__nv_bfloat16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tc_batched_kernel<__nv_bfloat16><<<grid, kTcThreads, smem, st>>>(p);
  }
  TK_CUDA_CHECK(cudaGetLastError());
  dim3 rg((unsigned)((n + 1 + 127) / 128), (unsigned)a.B);
  tc_reduce<<<rg, 128, 0, st>>>(m, n, n16, a.B, P, p.gpart, p.spart, a.vec_dtype, a.G, a.S, p.status);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

}  // namespace tk
