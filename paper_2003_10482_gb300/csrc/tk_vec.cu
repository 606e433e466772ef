// FP64 vector kernels of the dual solver (Section 4, eqs. dual_tensor_kernel
// and jq): objective and gradient assembly from reduced contractions.
#include "tk_internal.h"

namespace tk {

// one block per problem b; fixed-order block reductions in FP64
__global__ void __launch_bounds__(256) assemble_kernel(int m, int n, const double *G, const double *S,
                                                       const double *A, const double *y, const double *lambda,
                                                       double *F, double *grad, double *gnorm) {
  __shared__ double sh[3][8];
  const int b = blockIdx.x;
  const double lam = lambda[b];
  const double *g = G + (size_t)b * n;
  const double *a = A + (size_t)b * n;
  double ssq = 0.0, aa = 0.0, ya = 0.0;
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    const double gr = g[l] + lam * a[l] - y[l];
    if (grad) grad[(size_t)b * n + l] = gr;
    ssq += gr * gr;
    aa += a[l] * a[l];
    ya += y[l] * a[l];
  }
  for (int o = 16; o > 0; o >>= 1) {
    ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
    aa += __shfl_xor_sync(0xffffffffu, aa, o);
    ya += __shfl_xor_sync(0xffffffffu, ya, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sh[0][wid] = ssq;
    sh[1][wid] = aa;
    sh[2][wid] = ya;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t0 = 0, t1 = 0, t2 = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      t0 += sh[0][w];
      t1 += sh[1][w];
      t2 += sh[2][w];
    }
    F[b] = S[b] / m + 0.5 * lam * t1 - t2;
    if (gnorm) gnorm[b] = sqrt(t0);
  }
}

}  // namespace tk

using namespace tk;

extern "C" int tk_assemble_objective(int m, int64_t n, int64_t B, const double *G, const double *S,
                                     const double *A, const double *y, const double *lambda, double *F,
                                     double *grad, double *gnorm, void *stream) {
  if (m < 2 || n < 1 || B < 0) return fail(TK_EINVAL, "bad m, n or B");
  if (B == 0) return TK_OK;
  if (!G || !S || !A || !y || !lambda || !F) return fail(TK_EINVAL, "NULL pointer");
  if (B > 2147483647ll) return fail(TK_EINVAL, "B too large");
  assemble_kernel<<<(unsigned)B, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(m, (int)n, G, S, A, y, lambda, F,
                                                                                grad, gnorm);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}
