// Primal recovery and prediction (Section 4, eqs. tensor_representer and
// tensor_1, linear tensor kernel) and the Nystrom-like subsampling of
// Section 6.1.
#include <math.h>

#include <algorithm>
#include <vector>

#include "tk_internal.h"

namespace tk {

// w[b][k] = sign(u)|u|^{m-1}, u = sum_i X[i][k] a[b][i]; one thread per (b, k),
// consecutive k coalesced
__global__ void k_primal(int m, int n, int d, const double *X, const double *A, double *W) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y;
  if (k >= d) return;
  const double *a = A + (size_t)b * n;
  double u = 0.0;
  for (int i = 0; i < n; ++i) u += X[(size_t)i * d + k] * a[i];
  double p = 1.0;
  const double au = fabs(u);
  for (int e = 0; e < m - 1; ++e) p *= au;
  W[(size_t)b * d + k] = (u < 0.0) ? -p : p;
}

// yhat[b][j] = <w_b, x_j>; one warp per (b, j), lanes over features
__global__ void k_predict(int t, int d, const double *Xt, int B, const double *W, double *Y) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (gw >= (int64_t)t * B) return;
  const int64_t b = gw / t, j = gw % t;
  const double *x = Xt + j * d;
  const double *w = W + b * d;
  double s = 0.0;
  for (int k = lane; k < d; k += 32) s += x[k] * w[k];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) Y[b * t + j] = s;
}

// Adaptive threshold of Section 6.3: keep feature j of problem b when
// |w_j| > 2 std(w), std the population standard deviation of the d weights.
// One block per problem; mean and variance in FP64 by a two-pass sum in a
// fixed order (thread-strided partials, then a fixed tree), so the decision
// is reproducible.
__global__ void __launch_bounds__(256) k_support(int d, const double *W, uint8_t *keep, int64_t *count) {
  __shared__ double sh[256];
  __shared__ int shc[256];
  const double *w = W + (size_t)blockIdx.x * d;
  auto block_sum = [&](double v) -> double {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
      if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
      __syncthreads();
    }
    const double t = sh[0];
    __syncthreads();
    return t;
  };
  double s = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) s += w[j];
  const double mean = block_sum(s) / d;
  double q = 0.0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const double e = w[j] - mean;
    q += e * e;
  }
  const double thr = 2.0 * sqrt(block_sum(q) / d);
  int c = 0;
  for (int j = threadIdx.x; j < d; j += blockDim.x) {
    const bool k = fabs(w[j]) > thr;
    keep[(size_t)blockIdx.x * d + j] = k ? 1 : 0;
    c += k;
  }
  shc[threadIdx.x] = c;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) shc[threadIdx.x] += shc[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0 && count) count[blockIdx.x] = shc[0];
}

// SplitMix64 step: add the golden-ratio increment, then the variant-13 mixer
static inline uint64_t splitmix64(uint64_t &st) {
  uint64_t z = (st += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace tk

using namespace tk;

extern "C" int tk_primal(int m, int64_t n, int64_t d, const double *X, int64_t B, const double *A, double *W,
                         void *stream) {
  if (m < 2 || n < 1 || d < 1 || B < 0) return fail(TK_EINVAL, "bad sizes");
  if (B == 0) return TK_OK;
  if (!X || !A || !W) return fail(TK_EINVAL, "NULL pointer");
  if (n > 2147483647ll || d > 2147483647ll || B > 65535) return fail(TK_EUNSUPPORTED, "sizes too large");
  dim3 grid((unsigned)((d + 127) / 128), (unsigned)B);
  k_primal<<<grid, 128, 0, reinterpret_cast<cudaStream_t>(stream)>>>(m, (int)n, (int)d, X, A, W);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

extern "C" int tk_predict(int64_t t, int64_t d, const double *Xt, int64_t B, const double *W, double *Y,
                          void *stream) {
  if (t < 0 || d < 1 || B < 0) return fail(TK_EINVAL, "bad sizes");
  if (t == 0 || B == 0) return TK_OK;
  if (!Xt || !W || !Y) return fail(TK_EINVAL, "NULL pointer");
  if (t > 2147483647ll || d > 2147483647ll || B > 2147483647ll) return fail(TK_EUNSUPPORTED, "sizes too large");
  const int64_t warps = t * B;
  const unsigned blocks = (unsigned)((warps * 32 + 255) / 256);
  k_predict<<<blocks, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>((int)t, (int)d, Xt, (int)B, W, Y);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

extern "C" int tk_nystrom_select(int64_t N, int64_t np, uint64_t seed, int64_t *out) {
  if (N < 0 || np < 0 || np > N) return fail(TK_EINVAL, "n_prime must lie in [0, N]");
  if (np > 0 && !out) return fail(TK_EINVAL, "NULL output");
  uint64_t st = seed;
  std::vector<int64_t> taken;
  taken.reserve((size_t)np);
  std::vector<int64_t> sorted;  // membership test on the taken set
  for (int64_t j = N - np; j < N; ++j) {
    const uint64_t range = (uint64_t)j + 1;
    const uint64_t limit = UINT64_MAX - (UINT64_MAX % range);
    uint64_t x;
    do {
      x = splitmix64(st);
    } while (x >= limit);
    const int64_t r = (int64_t)(x % range);
    const bool in = std::binary_search(sorted.begin(), sorted.end(), r);
    const int64_t pick = in ? j : r;
    taken.push_back(pick);
    sorted.insert(std::upper_bound(sorted.begin(), sorted.end(), pick), pick);
  }
  std::copy(sorted.begin(), sorted.end(), out);
  return TK_OK;
}

extern "C" int tk_support_threshold(int64_t d, int64_t B, const double *W, uint8_t *keep, int64_t *count,
                                    void *stream) {
  if (d < 1 || B < 0) return fail(TK_EINVAL, "bad sizes");
  if (B == 0) return TK_OK;
  if (!W || !keep) return fail(TK_EINVAL, "NULL pointer");
  if (d > 2147483647ll || B > 2147483647ll) return fail(TK_EUNSUPPORTED, "sizes too large");
  k_support<<<(unsigned)B, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>((int)d, W, keep, count);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}
