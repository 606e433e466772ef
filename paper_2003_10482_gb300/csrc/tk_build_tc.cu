// Packed build on the 5th-generation tensor cores (FP32 and BF16 storage).
//
// What is computed is the build of tk_build.cu (Section 4 tensor kernel,
// Section 5 storage): for a triangle Q with last value b the entries
// (Q, c, d), b <= c <= d < n, are the upper triangle of the weighted Gram
// matrix G^Q = X_{[b:n]} diag(w_Q) X_{[b:n]}^T, w_Q[k] = prod_{q in Q} x_{q,k},
// passed through the feature map.
//
// GB300 mapping.  A task is one 128 x 128 tile (rows c, columns d >= c) of
// one triangle on a fixed grid of 128-row tiles; tasks are enumerated per b
// (multiset(b+1, m-3) triangles, each with T(nt - b/128) tile pairs) and
// strided over a persistent grid of one block per SM.  The block is a
// warp-specialised pipeline connected by mbarriers:
//   * warps 4-11 build, per 32-feature chunk, both operands from X in FP64 --
//     A[c][k] = w_Q[k] x_{c,k} and B[d][k] = x_{d,k} -- round them to FP32,
//     split them into TF32 hi and lo and store them in the K-major
//     128-byte-swizzled layout of one of 3 ring stages;
//   * one thread of warp 12 issues 4 k-steps of tcgen05.mma kind::tf32
//     (M = 128 rows, N = the tile's columns, K = 8): hi.hi into one tensor-
//     memory accumulator, hi.lo + lo.hi into a second (the large products
//     summed apart from the small ones), two such pairs alternating between
//     tasks;
//   * warps 0-3 (thread i <-> tensor-memory lane i <-> row c0 + i) add the
//     two accumulators, apply the feature map and write each row's entries
//     d >= c to their packed offsets.
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
  int m, n, d, nt, nkc;
  const double *X;
  int feat, degree;
  void *K;  // entry off_lo
  int64_t off_lo, off_hi;
  int64_t total_tasks;
};

struct CTask {
  int b, bb, rt, ct;
  int32_t q[kMaxOrder];
  int64_t base;
  bool live;
};

__host__ __device__ __forceinline__ int64_t c_tiles(int nt, int b) {
  const int k = nt - b / kCT;
  return (int64_t)k * (k + 1) / 2;
}

// Task t -> triangle (its prefix, b, packed base) and tile pair (rt, ct).
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
  const int rt0 = b / kCT, k = p.nt - rt0;
  const int64_t T = (int64_t)k * (k + 1) / 2;
  const int64_t local = t - pre[lo];
  const int64_t qi = local / T;
  int tp = (int)(local - qi * T);
  int rt = rt0;
  while (tp >= p.nt - rt) {
    tp -= p.nt - rt;
    ++rt;
  }
  r.b = b;
  r.bb = b;
  r.rt = rt;
  r.ct = rt + tp;
  int32_t tup[kMaxOrder];
  if (m >= 3) {
    if (m > 3) unrank(m - 3, b + 1, qi, tup);
    tup[m - 3] = b;
  }
  tup[m - 2] = b;
  tup[m - 1] = b;
  for (int j = 0; j < m - 2; ++j) r.q[j] = tup[j];
  r.base = (m == 2) ? 0 : rank(m, n, tup);
  const int64_t L = n - b;
  r.live = !(r.base + L * (L + 1) / 2 <= p.off_lo || r.base >= p.off_hi);
  return r;
}

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

// 16 consecutive values of row `row` (features k0 .. k0+15 of X's row `xr`,
// times w[0..15] when w is given) as TF32 hi/lo in the swizzled tile.
__device__ __forceinline__ void c_row16(const CParams &p, int xr, bool valid, int k0, const double *w, int row, int kin,
                                        unsigned char *thi, unsigned char *tlo) {
  float h[16], l[16];
  const double *xrow = p.X + (size_t)xr * p.d;
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int k = k0 + i;
    double x = (valid && k < p.d) ? xrow[k] : 0.0;
    if (w) x *= w[i];
    umma::split_tf32((float)x, h[i], l[i]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const uint32_t so = umma::sw128_offset((uint32_t)row, (uint32_t)(kin + 4 * j));
    *reinterpret_cast<float4 *>(thi + so) = make_float4(h[4 * j], h[4 * j + 1], h[4 * j + 2], h[4 * j + 3]);
    *reinterpret_cast<float4 *>(tlo + so) = make_float4(l[4 * j], l[4 * j + 1], l[4 * j + 2], l[4 * j + 3]);
  }
}

template <typename ST>
__global__ void __launch_bounds__(kCThreads, 1) tc_build_kernel(CParams p) {
  extern __shared__ unsigned char cb_smem_raw[];
  __shared__ uint64_t bar_full[kCStages], bar_empty[kCStages], bar_accf[2], bar_acce[2];
  __shared__ uint32_t tbase;
  __shared__ int s_bad;
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(cb_smem_raw) + 1023) &
                                                        ~uintptr_t(1023));
  int64_t *pre = reinterpret_cast<int64_t *>(sm + kCStages * kCStageBytes);      // [n + 1]
  double *wbuf = reinterpret_cast<double *>(pre + (TK_MAX_POINTS + 1));          // [stages][32]
  const int tid = threadIdx.x, w = tid >> 5;
  const int m = p.m, n = p.n;
  const int ngroups = (m == 2) ? 1 : n;
  for (int b = tid; b < ngroups; b += blockDim.x)
    pre[b + 1] = (m == 2 ? 1 : multiset(b + 1, m - 3)) * c_tiles(p.nt, b);
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
      if (!tsk.live) continue;
      const int buf = jl & 1;
      if (!c_wait(&bar_accf[buf], (uint32_t)(jl >> 1) & 1u, bad)) break;
      umma::fence_after_sync();
      const int c = kCT * tsk.rt + tid, d0 = kCT * tsk.ct;
      const int npad = min(kCT, ((n - d0) + 15) & ~15);
      const bool row_ok = c >= tsk.bb && c < n;
      const int64_t rowoff = tsk.base + (int64_t)(c - tsk.bb) * (2 * n - tsk.bb - c + 1) / 2 - c;
      const uint32_t tb = tl + (uint32_t)buf * 256u, ts = tb + 128u;
      for (int j0 = 0; j0 < npad; j0 += 16) {
        uint32_t ub[16], us[16];
        umma::tmem_ld16_async(tb + j0, ub);
        umma::tmem_ld16_async(ts + j0, us);
        umma::tmem_wait_ld();
        if (!row_ok) continue;
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
    const int gt = tid - 32 * kCEpiWarps;
    const int row = gt >> 1, kin = 16 * (gt & 1);
    uint32_t gc = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < p.total_tasks && ok; t += gridDim.x) {
      const CTask tsk = c_decode(p, pre, t);
      if (!tsk.live) continue;
      const int c = kCT * tsk.rt + row, dd = kCT * tsk.ct + row;
      for (int kc = 0; kc < p.nkc; ++kc, ++gc) {
        const int s = (int)(gc % kCStages);
        const uint32_t use = gc / kCStages;
        if (use > 0 && !c_wait(&bar_empty[s], (use - 1) & 1u, bad)) {
          ok = false;
          break;
        }
        double *ws = wbuf + 32 * s;
        if (gt < 32) {
          const int k = 32 * kc + gt;
          double wv = 0.0;
          if (k < p.d) {
            wv = 1.0;
            for (int j = 0; j < m - 2; ++j) wv *= p.X[(size_t)tsk.q[j] * p.d + k];
          }
          ws[gt] = wv;
        }
        asm volatile("bar.sync 1, %0;" ::"n"(kCGatherThreads) : "memory");  // the chunk's weights are in place
        unsigned char *st = sm + s * kCStageBytes;
        c_row16(p, c, c < n, 32 * kc + kin, ws + kin, row, kin, st, st + kCPart);
        c_row16(p, dd, dd < n, 32 * kc + kin, nullptr, row, kin, st + 2 * kCPart, st + 3 * kCPart);
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
      if (!tsk.live) continue;
      const int buf = jl & 1;
      if (jl >= 2 && !c_wait(&bar_acce[buf], (uint32_t)((jl >> 1) - 1) & 1u, bad)) break;
      umma::fence_after_sync();
      const int d0 = kCT * tsk.ct;
      const int npad = min(kCT, ((n - d0) + 15) & ~15);
      const uint32_t idesc = idesc_base | ((uint32_t)(npad >> 3) << 17);
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
         (size_t)kCStages * 32 * sizeof(double);
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
  p.nt = (n + kCT - 1) / kCT;
  p.nkc = (d + 31) / 32;
  p.X = X;
  p.feat = feat;
  p.degree = degree;
  p.K = K;
  p.off_lo = off_lo;
  p.off_hi = off_hi;
  int64_t total = 0;
  for (int b = 0; b < ((m == 2) ? 1 : n); ++b) {
    const int k = p.nt - b / kCT;
    total += (m == 2 ? 1 : multiset(b + 1, m - 3)) * ((int64_t)k * (k + 1) / 2);
  }
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
