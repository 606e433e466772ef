// Packed build of the order-m tensor kernel (Section 4), stored in the
// sorted-tuple order of Section 5.
//
// For a triangle Q = (i_1..i_{m-2}) with last value b, the entries (Q, c, d),
// b <= c <= d < n, form the upper triangle of the weighted Gram matrix
//   G^Q = X_{[b:n]} diag(w_Q) X_{[b:n]}^T,   w_Q[k] = prod_{q in Q} x_{q,k},
// i.e. K_{Qcd} = sum_k w_Q[k] x_{c,k} x_{d,k}.  Each block computes one 64 x 64
// tile of one such triangle as a small GEMM (16 x 16 threads, 4 x 4 outputs
// each, features staged 16 at a time in shared memory) and writes the entries
// with c <= d to their packed offsets
//   off(Q, c, d) = base(Q) + (c - b)(2n - b - c + 1)/2 + (d - c).
// Tasks are (triangle, tile pair) in layout order, grouped by b: the number
// of triangles whose last index is b is multiset(b+1, m-3), each with
// T(n-b) = nb(nb+1)/2 tile pairs (nb = ceil((n-b)/64)).  A persistent grid
// strides over the tasks; each block builds the per-b prefix table of task
// counts in shared memory once.
#include <cuda_bf16.h>

#include <algorithm>

#include "tk_internal.h"

namespace tk {

constexpr int kTM = 64;  // tile rows (c) and columns (d)
constexpr int kKT = 16;  // features per stage

struct BParams {
  int m, n, d;
  const double *X;
  int feat, degree;
  void *K;  // entry off_lo
  int64_t off_lo, off_hi;
  int64_t total_tasks;
};

__device__ __forceinline__ int tiles_for(int L) {
  const int nb = (L + kTM - 1) / kTM;
  return nb * (nb + 1) / 2;
}

__device__ __forceinline__ float fmx(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return __fma_rn(a, b, c); }

template <typename CT>
__device__ __forceinline__ CT feat_apply(CT v, int feat, int degree) {
  if (feat == TK_FEAT_POLY) {
    CT r = CT(1);
    for (int i = 0; i < degree; ++i) r *= v;
    return r;
  }
  if (feat == TK_FEAT_EXP) return exp(v);
  return v;
}

template <typename ST, typename CT>
__device__ __forceinline__ void store_entry(void *K, int64_t idx, CT v);
template <>
__device__ __forceinline__ void store_entry<double, double>(void *K, int64_t idx, double v) {
  reinterpret_cast<double *>(K)[idx] = v;
}
template <>
__device__ __forceinline__ void store_entry<float, float>(void *K, int64_t idx, float v) {
  reinterpret_cast<float *>(K)[idx] = v;
}
template <>
__device__ __forceinline__ void store_entry<__nv_bfloat16, float>(void *K, int64_t idx, float v) {
  reinterpret_cast<__nv_bfloat16 *>(K)[idx] = __float2bfloat16_rn(v);
}

template <typename ST, typename CT>
__global__ void __launch_bounds__(256) build_kernel(BParams p) {
  __shared__ int64_t pre[TK_MAX_POINTS + 1];
  __shared__ __align__(16) CT Ys[kKT][kTM];
  __shared__ __align__(16) CT Xs[kKT][kTM];
  __shared__ CT ws[kKT];
  const int tid = threadIdx.x;
  const int m = p.m, n = p.n, d = p.d;
  const int ngroups = (m == 2) ? 1 : n;

  // per-b task counts, then an exclusive prefix sum (one thread; n <= 1024)
  for (int b = tid; b < ngroups; b += blockDim.x) {
    if (m == 2) pre[b + 1] = tiles_for(n);
    else pre[b + 1] = multiset(b + 1, m - 3) * (int64_t)tiles_for(n - b);
  }
  __syncthreads();
  if (tid == 0) {
    pre[0] = 0;
    for (int b = 1; b <= ngroups; ++b) pre[b] += pre[b - 1];
  }
  __syncthreads();

  const int ty = tid >> 4, tx = tid & 15;
  int32_t tup[kMaxOrder];

  for (int64_t t = blockIdx.x; t < p.total_tasks; t += gridDim.x) {
    // locate the group b: largest b with pre[b] <= t
    int lo = 0, hi = ngroups - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (pre[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const int b = (m == 2) ? 0 : lo;
    const int L = n - b;
    const int nb = (L + kTM - 1) / kTM;
    const int T = nb * (nb + 1) / 2;
    const int64_t local = t - pre[lo];
    const int64_t qi = local / T;
    int tp = (int)(local - qi * T);
    int rb = 0;
    while (tp >= nb - rb) {
      tp -= nb - rb;
      ++rb;
    }
    const int cb = rb + tp;

    // triangle Q = (prefix of m-3 values in [0, b], b); base offset of (Q, b, b)
    if (m >= 3) {
      if (m > 3) unrank(m - 3, b + 1, qi, tup);
      tup[m - 3] = b;
    }
    tup[m - 2] = b;
    tup[m - 1] = b;
    const int64_t base = (m == 2) ? 0 : rank(m, n, tup);
    const int64_t tri_size = (int64_t)L * (L + 1) / 2;
    if (base + tri_size <= p.off_lo || base >= p.off_hi) continue;  // outside the range

    const int c0 = b + rb * kTM;
    const int d0 = b + cb * kTM;
    CT acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[i][j] = CT(0);

    for (int k0 = 0; k0 < d; k0 += kKT) {
      __syncthreads();
      if (tid < kKT) {
        const int k = k0 + tid;
        CT w = CT(1);
        if (k < d)
          for (int j = 0; j < m - 2; ++j) w *= (CT)p.X[(int64_t)tup[j] * d + k];
        ws[tid] = (k < d) ? w : CT(0);
      }
      __syncthreads();
      // 64 rows x 16 features for each of Ys and Xs: 1024 values, 4 per thread
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int e = tid + 256 * r;
        const int row = e >> 4, kk = e & 15;
        const int k = k0 + kk;
        const int c = c0 + row, dd = d0 + row;
        const CT xc = (c < n && k < d) ? (CT)p.X[(int64_t)c * d + k] : CT(0);
        const CT xd = (dd < n && k < d) ? (CT)p.X[(int64_t)dd * d + k] : CT(0);
        Ys[kk][row] = xc * ws[kk];
        Xs[kk][row] = xd;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < kKT; ++kk) {
        CT a[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          a[i] = Ys[kk][ty * 4 + i];
          bv[i] = Xs[kk][tx * 4 + i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fmx(a[i], bv[j], acc[i][j]);
      }
    }

    // packed stores of the upper-triangle entries
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int c = c0 + ty * 4 + i;
      if (c >= n) continue;
      const int64_t rowoff = base + (int64_t)(c - b) * (2 * n - b - c + 1) / 2 - c;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int dd = d0 + tx * 4 + j;
        if (dd < c || dd >= n) continue;
        const int64_t off = rowoff + dd;
        if (off < p.off_lo || off >= p.off_hi) continue;
        store_entry<ST, CT>(p.K, off - p.off_lo, feat_apply(acc[i][j], p.feat, p.degree));
      }
    }
  }
}

template <typename ST, typename CT>
static int launch_build(const BParams &bp, cudaStream_t st) {
  DevInfo di;
  int rc = dev_info(&di);
  if (rc != TK_OK) return rc;
  int64_t blocks = std::min<int64_t>(bp.total_tasks, (int64_t)di.sms * 4);
  if (blocks < 1) return TK_OK;
  build_kernel<ST, CT><<<(int)blocks, 256, 0, st>>>(bp);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

int g_build_tc_mode = 0;

}  // namespace tk

using namespace tk;

extern "C" int tk_build_set_config(int tensor_cores) {
  if (tensor_cores < -1 || tensor_cores > 1) return fail(TK_EINVAL, "tensor_cores must be -1, 0 or 1");
  g_build_tc_mode = tensor_cores;
  return TK_OK;
}

extern "C" int tk_build_status(void *stream) { return build_tc_status(reinterpret_cast<cudaStream_t>(stream)); }

static bool build_takes_tc(int64_t d, int storage) {
  // the tensor-core build is opt-in: on GB300 it measured slower than the SIMT
  // build (m = 4: n = 200, d = 20,000: 501 vs 443 ms; n = 400, d = 100: 56 vs
  // 29 ms), bound by its operand-building warps rather than the tensor cores
  (void)d;
  if (storage == TK_F64 || g_build_tc_mode <= 0) return false;
  int dev = 0, major = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return false;
  return major == 10;
}

extern "C" int tk_build_path(int64_t d, int storage) { return build_takes_tc(d, storage) ? 1 : 0; }

extern "C" int tk_build_packed_range(int m, int64_t n, int64_t d, const double *X, int feat, int degree,
                                     int storage, int64_t off_lo, int64_t off_hi, void *K, void *stream) {
  if (m < 2 || m > TK_MAX_ORDER) return fail(TK_EINVAL, "order m=%d outside [2, %d]", m, TK_MAX_ORDER);
  if (n < 1 || d < 1) return fail(TK_EINVAL, "n and d must be >= 1");
  if (n > TK_MAX_POINTS) return fail(TK_EUNSUPPORTED, "n=%lld exceeds %d", (long long)n, TK_MAX_POINTS);
  if (storage < TK_F64 || storage > TK_BF16) return fail(TK_EINVAL, "bad storage dtype %d", storage);
  if (feat < TK_FEAT_LINEAR || feat > TK_FEAT_EXP) return fail(TK_EINVAL, "bad feature map %d", feat);
  if (feat == TK_FEAT_POLY && degree < 1) return fail(TK_EINVAL, "polynomial degree must be >= 1");
  const int64_t N = tk_packed_size(m, n);
  if (N < 0) return fail(TK_EOVERFLOW, "C(n+m-1, m) overflows");
  if (off_lo < 0 || off_hi > N || off_lo > off_hi) return fail(TK_EINVAL, "range outside [0, N]");
  if (off_hi == off_lo) return TK_OK;
  if (!X || !K) return fail(TK_EINVAL, "NULL X or K");
  BParams bp;
  bp.m = m;
  bp.n = (int)n;
  bp.d = (int)d;
  bp.X = X;
  bp.feat = feat;
  bp.degree = degree;
  bp.K = K;
  bp.off_lo = off_lo;
  bp.off_hi = off_hi;
  int64_t total = 0;
  if (m == 2) {
    const int nb = (int)((n + kTM - 1) / kTM);
    total = (int64_t)nb * (nb + 1) / 2;
  } else {
    for (int64_t b = 0; b < n; ++b) {
      const int64_t L = n - b, nb = (L + kTM - 1) / kTM;
      total += multiset(b + 1, m - 3) * (nb * (nb + 1) / 2);
    }
  }
  bp.total_tasks = total;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (build_takes_tc(d, storage)) {
    const int rc = build_tc(m, (int)n, (int)d, X, feat, degree, storage, off_lo, off_hi, K, st);
    if (rc != TK_EUNSUPPORTED) return rc;
  }
  if (storage == TK_F64) return launch_build<double, double>(bp, st);
  if (storage == TK_F32) return launch_build<float, float>(bp, st);
  return launch_build<__nv_bfloat16, float>(bp, st);
}

extern "C" int tk_build_packed(int m, int64_t n, int64_t d, const double *X, int feat, int degree, int storage,
                               void *K, void *stream) {
  const int64_t N = tk_packed_size(m, n);
  if (N < 0) return fail(TK_EOVERFLOW, "C(n+m-1, m) overflows or m, n invalid");
  return tk_build_packed_range(m, n, d, X, feat, degree, storage, 0, N, K, stream);
}
