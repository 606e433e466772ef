// Packed build on the 5th-generation tensor cores (FP32 and BF16 storage).
//
// What is computed is the build of tk_build.cu (Section 4 tensor kernel,
// Section 5 storage): for a triangle Q with last value b the entries
// (Q, c, d), b <= c <= d < n, are the upper triangle of the weighted Gram
// matrix G^Q = X_{[b:n]} diag(w_Q) X_{[b:n]}^T, w_Q[k] = prod_{q in Q} x_{q,k},
// passed through the feature map.
//
// GB300 mapping.  The triangles with last value b (multiset(b+1, m-3) of them)
// share their rows and columns [b, n), L = n - b.  A task is one MMA tile of
// 128 rows: for L <= 128 the rows of floor(128/L) consecutive such triangles
// stacked (columns [b, n)); for L > 128 one triangle's 128-row block c in
// [b + 128 rt, ...) against the 128-column block d in [b + 128 ct, ...),
// ct >= rt.  Tasks are enumerated per b and strided over a persistent grid of
// one block per SM.  The block is a warp-specialised pipeline connected by
// mbarriers:
//   * warps 4-11 build, per 32-feature chunk, both operands from X in FP64 --
//     A[r][k] = x_{c_r,k} prod_{q in Q_r} x_{q,k} for row r's triangle Q_r and
//     row c_r, B[j][k] = x_{d_j,k} -- with each triangle's weight row formed
//     once per chunk (rounded to FP32), lanes along the features (coalesced
//     loads, all of a warp's rows issued before use), round them to FP32,
//     split them into TF32 hi and lo and store them in the K-major
//     128-byte-swizzled layout of one of 3 ring stages;
//   * one thread of warp 12 issues 4 k-steps of tcgen05.mma kind::tf32
//     (M = 128 rows, N = the tile's columns, K = 8): hi.hi into one tensor-
//     memory accumulator, hi.lo + lo.hi into a second (the large products
//     summed apart from the small ones), two such pairs alternating between
//     tasks;
//   * warps 0-3 (thread i <-> tensor-memory lane i <-> row i of the tile) add
//     the two accumulators, apply the feature map and write row i's entries
//     d >= c to its triangle's packed offsets.
#include <cuda_bf16.h>

#include "tk_umma.cuh"

namespace tk {

constexpr int kCT = 128;  // tile rows and (at most) columns
constexpr int kCEpiWarps = 4, kCGatherWarps = 8;
constexpr int kCGatherThreads = 32 * kCGatherWarps;
constexpr int kCThreads = 32 * (kCEpiWarps + kCGatherWarps + 1);
constexpr int kCStages = 3;
constexpr int kCPart = kCT * 128;  // 128 rows x 32 FP32 values
constexpr int kCStageBytes = 4 * kCPart;  // A hi, A lo, B hi, B lo

// Set by a tensor-core build whose bounded wait ran out (read by tk_build_status).
__device__ int g_tc_build_status;

struct CParams {
  int m, n, d, nkc;
  const double *X;
  int feat, degree;
  void *K;  // entry off_lo
  int64_t off_lo, off_hi;
  int64_t total_tasks;
};

struct CTask {
  int b, L;          // last prefix value, rows/columns of its triangles
  int stacked;       // 1: floor(128/L) whole triangles stacked, 0: one 128 x 128 block of one triangle
  int64_t qi0;       // index (among the triangles with last value b) of the task's first triangle
  int ntri;          // triangles in the task
  int rt, ct;        // row / column block (L > 128)
  int npad;          // columns, rounded up to 16 (N of the MMA)
};

__host__ __device__ __forceinline__ int64_t c_count(int m, int n, int b) {
  const int64_t cb = (m == 2) ? 1 : multiset(b + 1, m - 3);
  const int L = n - b;
  if (L <= kCT) {
    const int k = kCT / L;
    return (cb + k - 1) / k;
  }
  const int64_t lt = (L + kCT - 1) / kCT;
  return cb * (lt * (lt + 1) / 2);
}

// Task t -> its triangle group or block.
__host__ __device__ __forceinline__ CTask c_decode(const CParams &p, const int64_t *pre, int64_t t) {
  CTask r;
  const int m = p.m, n = p.n;
  const int ngroups = (m == 2) ? 1 : n;
  int lo = 0, hi = ngroups - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  const int b = (m == 2) ? 0 : lo;
  const int64_t cb = (m == 2) ? 1 : multiset(b + 1, m - 3);
  const int L = n - b;
  const int64_t local = t - pre[lo];
  r.b = b;
  r.L = L;
  if (L <= kCT) {
    const int k = kCT / L;
    r.stacked = 1;
    r.qi0 = local * k;
    r.ntri = (int)(cb - r.qi0 < k ? cb - r.qi0 : k);
    r.rt = r.ct = 0;
    r.npad = (L + 15) & ~15;
  } else {
    const int lt = (L + kCT - 1) / kCT;
    const int64_t T = (int64_t)lt * (lt + 1) / 2;
    r.stacked = 0;
    r.qi0 = local / T;
    r.ntri = 1;
    int tp = (int)(local - r.qi0 * T), rt = 0;
    while (tp >= lt - rt) {
      tp -= lt - rt;
      ++rt;
    }
    r.rt = rt;
    r.ct = rt + tp;
    const int cols = min(kCT, L - kCT * r.ct);
    r.npad = (cols + 15) & ~15;
  }
  return r;
}

// Row r of a task: its triangle (prefix Q, packed base of (Q, b, b)) and row c.
struct CRow {
  bool valid;
  int c;
  int32_t q[kMaxOrder];
  int64_t base;
};
__host__ __device__ __forceinline__ CRow c_row(const CParams &p, const CTask &t, int r) {
  CRow w;
  const int m = p.m, n = p.n, b = t.b;
  int64_t qi;
  if (t.stacked) {
    const int j = r / t.L;
    w.valid = j < t.ntri;
    qi = t.qi0 + (w.valid ? j : 0);
    w.c = b + r - j * t.L;
  } else {
    w.c = b + kCT * t.rt + r;
    w.valid = w.c < n;
    qi = t.qi0;
  }
  int32_t tup[kMaxOrder];
  if (m >= 3) {
    if (m > 3) unrank(m - 3, b + 1, qi, tup);
    tup[m - 3] = b;
  }
  tup[m - 2] = b;
  tup[m - 1] = b;
  for (int j = 0; j < m - 2; ++j) w.q[j] = tup[j];
  w.base = (m == 2) ? 0 : rank(m, n, tup);
  return w;
}

__host__ __device__ __forceinline__ int c_col0(const CTask &t) { return t.b + (t.stacked ? 0 : kCT * t.ct); }

template <typename ST>
__device__ __forceinline__ void c_store(void *K, int64_t idx, float v);
template <>
__device__ __forceinline__ void c_store<float>(void *K, int64_t idx, float v) {
  reinterpret_cast<float *>(K)[idx] = v;
}
template <>
__device__ __forceinline__ void c_store<__nv_bfloat16>(void *K, int64_t idx, float v) {
  reinterpret_cast<__nv_bfloat16 *>(K)[idx] = __float2bfloat16_rn(v);
}

__device__ __forceinline__ float c_feat(float v, int feat, int degree) {
  if (feat == TK_FEAT_POLY) {
    float r = 1.f;
    for (int i = 0; i < degree; ++i) r *= v;
    return r;
  }
  if (feat == TK_FEAT_EXP) return expf(v);
  return v;
}

__device__ __forceinline__ bool c_wait(uint64_t *bar, uint32_t parity, volatile int *bad) {
  if (*bad) return false;
  if (mbar_wait_bounded(bar, parity)) return true;
  *bad = 1;
  return false;
}

// Whether any entry of the task lies in [off_lo, off_hi).
__host__ __device__ __forceinline__ bool c_live(const CParams &p, const CTask &t) {
  const CRow f = c_row(p, t, 0);
  const CRow l = c_row(p, t, t.stacked ? (t.ntri - 1) * t.L : 0);
  const int64_t L = t.L;
  return !(l.base + L * (L + 1) / 2 <= p.off_lo || f.base >= p.off_hi);
}

template <typename ST>
__global__ void __launch_bounds__(kCThreads, 1) tc_build_kernel(CParams p) {
  extern __shared__ unsigned char cb_smem_raw[];
  __shared__ uint64_t bar_full[kCStages], bar_empty[kCStages], bar_accf[2], bar_acce[2];
  __shared__ uint32_t tbase;
  __shared__ int s_bad;
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(cb_smem_raw) + 1023) &
                                                        ~uintptr_t(1023));
  int64_t *pre = reinterpret_cast<int64_t *>(sm + kCStages * kCStageBytes);  // [n + 1]
  float *wtab = reinterpret_cast<float *>(pre + (TK_MAX_POINTS + 1));        // [128 triangles][32 features]
  int32_t *qtab = reinterpret_cast<int32_t *>(wtab + kCT * 32);               // [128 triangles][kMaxOrder]

  const int tid = threadIdx.x, w = tid >> 5;
  const int m = p.m, n = p.n;
  const int ngroups = (m == 2) ? 1 : n;
  for (int b = tid; b < ngroups; b += blockDim.x) pre[b + 1] = c_count(m, n, b);
  if (w == 0) {
    umma::tmem_alloc(&tbase, 512);
    umma::tmem_relinquish();
  }
  if (tid == 0) {
    for (int s = 0; s < kCStages; ++s) {
      mbar_init(&bar_full[s], kCGatherThreads);
      mbar_init(&bar_empty[s], 1);
    }
    for (int b2 = 0; b2 < 2; ++b2) {
      mbar_init(&bar_accf[b2], 1);
      mbar_init(&bar_acce[b2], 32 * kCEpiWarps);
    }
    fence_barrier_init();
    s_bad = 0;
  }
  __syncthreads();
  if (tid == 0) {
    pre[0] = 0;
    for (int b = 1; b <= ngroups; ++b) pre[b] += pre[b - 1];
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  volatile int *bad = &s_bad;

  if (w < kCEpiWarps) {
    // ---------------------------------------------------------------- epilogue
    const uint32_t tl = tbase + ((uint32_t)(32 * w) << 16);
    int jl = 0;
    for (int64_t t = blockIdx.x; t < p.total_tasks; t += gridDim.x) {
      const CTask tsk = c_decode(p, pre, t);
      if (!c_live(p, tsk)) continue;
      const CRow row = c_row(p, tsk, tid);
      const int buf = jl & 1;
      if (!c_wait(&bar_accf[buf], (uint32_t)(jl >> 1) & 1u, bad)) break;
      umma::fence_after_sync();
      const int c = row.c, b = tsk.b, d0 = c_col0(tsk);
      const int64_t rowoff = row.base + (int64_t)(c - b) * (2 * n - b - c + 1) / 2 - c;
      const uint32_t tb = tl + (uint32_t)buf * 256u, ts = tb + 128u;
      for (int j0 = 0; j0 < tsk.npad; j0 += 16) {
        uint32_t ub[16], us[16];
        umma::tmem_ld16_async(tb + j0, ub);
        umma::tmem_ld16_async(ts + j0, us);
        umma::tmem_wait_ld();
        if (!row.valid) continue;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int dd = d0 + j0 + i;
          if (dd < c || dd >= n) continue;
          const int64_t off = rowoff + dd;
          if (off < p.off_lo || off >= p.off_hi) continue;
          const float v = __uint_as_float(ub[i]) + __uint_as_float(us[i]);
          c_store<ST>(p.K, off - p.off_lo, c_feat(v, p.feat, p.degree));
        }
      }
      umma::fence_before_sync();
      mbar_arrive(&bar_acce[buf]);
      ++jl;
    }
  } else if (w < kCEpiWarps + kCGatherWarps) {
    // ---------------------------------------------------------------- operands
    // per task the prefixes of its triangles go into a table; per chunk each
    // triangle's weight row w_Q[k] = prod_{q in Q} x_{q,k} is formed once, then
    // warp gw builds rows 16 gw .. 16 gw + 15 of both operands, lanes along
    // the chunk's 32 features, all row loads issued before the first is used.
    // (No early exit: the gathering warps meet at named barriers, so a wait
    // that ran out only skips its stage and the loops run to the end.)
    const int gt = tid - 32 * kCEpiWarps, gw = gt >> 5, lane = tid & 31;
    uint32_t gc = 0;
    for (int64_t t = blockIdx.x; t < p.total_tasks; t += gridDim.x) {
      const CTask tsk = c_decode(p, pre, t);
      if (!c_live(p, tsk)) continue;
      // the previous task's last chunk has been read by every gathering warp
      asm volatile("bar.sync 1, %0;" ::"n"(kCGatherThreads) : "memory");
      if (gt < tsk.ntri) {
        const CRow first = c_row(p, tsk, tsk.stacked ? gt * tsk.L : 0);
        for (int j = 0; j < m - 2; ++j) qtab[gt * kMaxOrder + j] = first.q[j];
      }
      int rc[16];
      bool rv[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int r = 16 * gw + i;
        if (tsk.stacked) {
          const int j = r / tsk.L;
          rv[i] = j < tsk.ntri;
          rc[i] = tsk.b + r - j * tsk.L;
        } else {
          rc[i] = tsk.b + kCT * tsk.rt + r;
          rv[i] = rc[i] < n;
        }
      }
      const int d0 = c_col0(tsk);
      for (int kc = 0; kc < p.nkc; ++kc, ++gc) {
        const int s = (int)(gc % kCStages);
        const uint32_t use = gc / kCStages;
        const int k = 32 * kc + lane;
        const bool kok = k < p.d;
        // the weight rows of the task's triangles for this chunk
        asm volatile("bar.sync 1, %0;" ::"n"(kCGatherThreads) : "memory");
        for (int j = gw; j < tsk.ntri; j += kCGatherWarps) {
          double wv = kok ? 1.0 : 0.0;
          if (kok)
            for (int jj = 0; jj < m - 2; ++jj) wv *= p.X[(size_t)qtab[j * kMaxOrder + jj] * p.d + k];
          wtab[j * 32 + lane] = (float)wv;
        }
        double xa[16], xb[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int r = 16 * gw + i, dd = d0 + r;
          xa[i] = (rv[i] && kok) ? p.X[(size_t)rc[i] * p.d + k] : 0.0;
          xb[i] = (r < tsk.npad && dd < n && kok) ? p.X[(size_t)dd * p.d + k] : 0.0;
        }
        asm volatile("bar.sync 1, %0;" ::"n"(kCGatherThreads) : "memory");  // weight rows in place
        if (use > 0 && !c_wait(&bar_empty[s], (use - 1) & 1u, bad)) continue;
        unsigned char *st = sm + s * kCStageBytes;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int r = 16 * gw + i;
          const int j = tsk.stacked ? r / tsk.L : 0;
          const double a = rv[i] ? xa[i] * wtab[(j < tsk.ntri ? j : 0) * 32 + lane] : 0.0;
          float h, l;
          umma::split_tf32((float)a, h, l);
          const uint32_t so = umma::sw128_offset((uint32_t)r, (uint32_t)lane);
          *reinterpret_cast<float *>(st + so) = h;
          *reinterpret_cast<float *>(st + kCPart + so) = l;
          umma::split_tf32((float)xb[i], h, l);
          *reinterpret_cast<float *>(st + 2 * kCPart + so) = h;
          *reinterpret_cast<float *>(st + 3 * kCPart + so) = l;
        }
        fence_proxy_async();  // the operands written above become visible to the tensor cores
        mbar_arrive(&bar_full[s]);
      }
    }
  } else if ((tid & 31) == 0) {
    // ---------------------------------------------------------------- MMA issue
    uint32_t gc = 0;
    int jl = 0;
    const uint32_t idesc_base = umma::idesc_tf32(kCT, 16) & ~(0x3Fu << 17);
    bool ok = true;
    for (int64_t t = blockIdx.x; t < p.total_tasks && ok; t += gridDim.x) {
      const CTask tsk = c_decode(p, pre, t);
      if (!c_live(p, tsk)) continue;
      const int buf = jl & 1;
      if (jl >= 2 && !c_wait(&bar_acce[buf], (uint32_t)((jl >> 1) - 1) & 1u, bad)) break;
      umma::fence_after_sync();
      const uint32_t idesc = idesc_base | ((uint32_t)(tsk.npad >> 3) << 17);
      const uint32_t tb = tbase + (uint32_t)buf * 256u, ts = tb + 128u;
      for (int kc = 0; kc < p.nkc; ++kc, ++gc) {
        const int s = (int)(gc % kCStages);
        if (!c_wait(&bar_full[s], (gc / kCStages) & 1u, bad)) {
          ok = false;
          break;
        }
        umma::fence_after_sync();
        const uint32_t a0 = saddr(sm + s * kCStageBytes), b0 = a0 + 2 * kCPart;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
          const uint64_t ah = umma::desc_sw128(a0 + 32 * ks), al = umma::desc_sw128(a0 + kCPart + 32 * ks);
          const uint64_t bh = umma::desc_sw128(b0 + 32 * ks), bl = umma::desc_sw128(b0 + kCPart + 32 * ks);
          const uint32_t acc = (kc > 0 || ks > 0) ? 1u : 0u;
          umma::mma_tf32(tb, ah, bh, idesc, acc);
          umma::mma_tf32(ts, ah, bl, idesc, acc);
          umma::mma_tf32(ts, al, bh, idesc, 1u);
        }
        umma::mma_commit(&bar_empty[s]);
      }
      umma::mma_commit(&bar_accf[buf]);
      ++jl;
    }
    // nothing may still write tensor memory when it is released
    if (jl > 0) mbar_wait_bounded(&bar_accf[(jl - 1) & 1], (uint32_t)((jl - 1) >> 1) & 1u);
  }
  umma::fence_before_sync();
  __syncthreads();
  if (w == 0) umma::tmem_dealloc(tbase, 512);
  if (tid == 0 && s_bad) atomicExch(&g_tc_build_status, TK_ETIMEOUT);
}

size_t tc_build_smem() {
  return 1024 + (size_t)kCStages * kCStageBytes + (size_t)(TK_MAX_POINTS + 1) * sizeof(int64_t) +
         (size_t)kCT * 32 * sizeof(float) + (size_t)kCT * kMaxOrder * sizeof(int32_t);
}

int build_tc(int m, int n, int d, const double *X, int feat, int degree, int storage, int64_t off_lo,
             int64_t off_hi, void *K, cudaStream_t st) {
  DevInfo di;
  int rc = dev_info(&di);
  if (rc != TK_OK) return rc;
  const size_t smem = tc_build_smem();
  if (smem > (size_t)di.smem_optin) return fail(TK_EUNSUPPORTED, "tensor-core build: shared memory");
  CParams p;
  p.m = m;
  p.n = n;
  p.d = d;
  p.nkc = (d + 31) / 32;
  p.X = X;
  p.feat = feat;
  p.degree = degree;
  p.K = K;
  p.off_lo = off_lo;
  p.off_hi = off_hi;
  int64_t total = 0;
  for (int b = 0; b < ((m == 2) ? 1 : n); ++b) total += c_count(m, n, b);
  p.total_tasks = total;
  if (total == 0) return TK_OK;
  const int grid = (int)std::min<int64_t>(total, di.sms);
  if (storage == TK_F32) {
    TK_CUDA_CHECK(cudaFuncSetAttribute(tc_build_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    tc_build_kernel<float><<<grid, kCThreads, smem, st>>>(p);
  } else {
    TK_CUDA_CHECK(cudaFuncSetAttribute(tc_build_kernel<__nv_bfloat16>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tc_build_kernel<__nv_bfloat16><<<grid, kCThreads, smem, st>>>(p);
  }
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

int build_tc_status(cudaStream_t st) {
  int h = 0;
  TK_CUDA_CHECK(cudaMemcpyFromSymbolAsync(&h, g_tc_build_status, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
  TK_CUDA_CHECK(cudaStreamSynchronize(st));
  if (h != TK_OK) {
    const int zero = 0;
    TK_CUDA_CHECK(cudaMemcpyToSymbolAsync(g_tc_build_status, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, st));
    TK_CUDA_CHECK(cudaStreamSynchronize(st));
  }
  return h;
}

}  // namespace tk
