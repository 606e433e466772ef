// Newton steps with the full dual Hessian (Section 4, second derivative of
// eq. dual_tensor_kernel): H_b = (m-1) K[a_b^{m-2}] + lambda_b I restricted to
// the kept points of problem b, factorised H_b = L L^T by a blocked Cholesky
// in FP64, then p_b = -H_b^{-1} grad_b by two triangular solves.
//
// Matrices are stored row-major with leading dimension npad = ceil(n/32)*32;
// held-out points and the padding get identity rows and columns (their step
// is then -grad = 0).  The factorisation runs panel by panel (32 columns):
// the diagonal block is factorised by one block per problem, the panel below
// it solved by one block per 32-row block, and the trailing matrix updated by
// one block per 32 x 32 tile; each launch covers every problem of the batch
// (grid y), so one large problem or many small ones both fill the GPU.  A
// pivot that is not positive (a tensor rounded to FP32 or BF16 can make the
// form indefinite by more than lambda) marks the problem; the solver then
// falls back to the steepest-descent direction for it.
#include <math.h>

#include "tk_internal.h"

namespace tk {

constexpr int kNP = 32;

// H[b] = (m-1) Hk[b] + lambda_b I on kept points; identity elsewhere (npad x npad)
__global__ void k_form_newton(int m, int n, int npad, const int *idx, const double *Hk, const double *lambda,
                              const uint8_t *mask, double *H) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  const int j = blockIdx.z;
  if (c >= npad) return;
  const int b = idx[j];
  const bool kr = r < n && (!mask || mask[(size_t)b * n + r]);
  const bool kc = c < n && (!mask || mask[(size_t)b * n + c]);
  double v;
  if (kr && kc) v = (m - 1) * Hk[(size_t)b * n * n + (size_t)r * n + c] + (r == c ? lambda[b] : 0.0);
  else v = (r == c) ? 1.0 : 0.0;
  H[(size_t)j * npad * npad + (size_t)r * npad + c] = v;
}

// factorise diagonal block k of every problem in place (lower triangle)
__global__ void __launch_bounds__(kNP * kNP) k_potrf_diag(int npad, int k, double *H, int *bad) {
  __shared__ double A[kNP][kNP + 1];
  const int j = blockIdx.x;
  double *M = H + (size_t)j * npad * npad + (size_t)k * kNP * npad + k * kNP;
  const int r = threadIdx.x / kNP, c = threadIdx.x % kNP;
  A[r][c] = M[(size_t)r * npad + c];
  __syncthreads();
  for (int p = 0; p < kNP; ++p) {
    if (threadIdx.x == 0) {
      double d = A[p][p];
      if (!(d > 0.0) || !isfinite(d)) {
        bad[j] = 1;
        d = 1.0;
      }
      A[p][p] = sqrt(d);
    }
    __syncthreads();
    if (c == p && r > p) A[r][p] /= A[p][p];
    __syncthreads();
    if (r > p && c > p && c <= r) A[r][c] -= A[r][p] * A[c][p];
    __syncthreads();
  }
  M[(size_t)r * npad + c] = (c <= r) ? A[r][c] : 0.0;
}

// panel below diagonal block k: X L_kk^T = A_ik for every block row i > k
__global__ void __launch_bounds__(kNP * kNP) k_trsm_panel(int npad, int k, double *H) {
  __shared__ double L[kNP][kNP + 1];
  __shared__ double X[kNP][kNP + 1];
  const int i = k + 1 + blockIdx.x;
  const int j = blockIdx.y;
  double *Hb = H + (size_t)j * npad * npad;
  const int r = threadIdx.x / kNP, c = threadIdx.x % kNP;
  L[r][c] = Hb[(size_t)(k * kNP + r) * npad + k * kNP + c];
  X[r][c] = Hb[(size_t)(i * kNP + r) * npad + k * kNP + c];
  __syncthreads();
  // row r of X: forward substitution over the 32 columns (thread c == 0 of each row)
  if (c == 0) {
    for (int q = 0; q < kNP; ++q) {
      double s = X[r][q];
      for (int t = 0; t < q; ++t) s -= X[r][t] * L[q][t];
      X[r][q] = s / L[q][q];
    }
  }
  __syncthreads();
  Hb[(size_t)(i * kNP + r) * npad + k * kNP + c] = X[r][c];
}

// trailing update: A_il -= L_ik L_lk^T for k < l <= i
__global__ void __launch_bounds__(kNP * kNP) k_syrk_update(int npad, int k, int nb, double *H) {
  __shared__ double Li[kNP][kNP + 1];
  __shared__ double Ll[kNP][kNP + 1];
  // blockIdx.x enumerates the pairs (i, l), k < l <= i < nb
  int t = blockIdx.x, l = k + 1, i = 0;
  for (;; ++l) {
    const int cnt = nb - l;
    if (t < cnt) {
      i = l + t;
      break;
    }
    t -= cnt;
  }
  const int j = blockIdx.y;
  double *Hb = H + (size_t)j * npad * npad;
  const int r = threadIdx.x / kNP, c = threadIdx.x % kNP;
  Li[r][c] = Hb[(size_t)(i * kNP + r) * npad + k * kNP + c];
  Ll[r][c] = Hb[(size_t)(l * kNP + r) * npad + k * kNP + c];
  __syncthreads();
  double s = 0.0;
#pragma unroll 8
  for (int q = 0; q < kNP; ++q) s += Li[r][q] * Ll[c][q];
  Hb[(size_t)(i * kNP + r) * npad + l * kNP + c] -= s;
}

// p_b = -(L L^T)^{-1} g_b on kept points (zero elsewhere); one block per problem
__global__ void __launch_bounds__(256) k_chol_solve(int n, int npad, const int *idx, const double *Lf,
                                                    const double *grad, const uint8_t *mask, double *p,
                                                    double *scratch) {
  const int j = blockIdx.x;
  const int b = idx[j];
  const double *L = Lf + (size_t)j * npad * npad;
  double *y = scratch + (size_t)j * npad;
  for (int i = threadIdx.x; i < npad; i += blockDim.x) {
    const bool keep = i < n && (!mask || mask[(size_t)b * n + i]);
    y[i] = keep ? -grad[(size_t)b * n + i] : 0.0;
  }
  __syncthreads();
  // L y = -g, column-oriented: y_i final, then eliminate it from the rows below
  for (int i = 0; i < npad; ++i) {
    if (threadIdx.x == 0) y[i] /= L[(size_t)i * npad + i];
    __syncthreads();
    const double yi = y[i];
    for (int r = i + 1 + threadIdx.x; r < npad; r += blockDim.x) y[r] -= L[(size_t)r * npad + i] * yi;
    __syncthreads();
  }
  // L^T x = y: row i of L^T is column i of L
  for (int i = npad - 1; i >= 0; --i) {
    if (threadIdx.x == 0) y[i] /= L[(size_t)i * npad + i];
    __syncthreads();
    const double yi = y[i];
    for (int r = threadIdx.x; r < i; r += blockDim.x) y[r] -= L[(size_t)i * npad + r] * yi;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const bool keep = !mask || mask[(size_t)b * n + i];
    p[(size_t)b * n + i] = keep ? y[i] : 0.0;
  }
}

// From a Hessian pass at a: G = K[a^{m-1}] = K[a^{m-2}] a and S = K[a^m] = a.G
// (Euler's identity for the homogeneous form), then the dual objective of
// problem idx[j]: F = S/m + lambda/2 |a|^2 - <y, a>, grad = G + lambda a - y on
// kept points, gn2 = |grad|^2.  One block per problem, fixed-order sums.
__global__ void __launch_bounds__(256) k_objective_from_hessian(int m, int n, const int *idx, const double *Hk,
                                                                const double *A, const double *y,
                                                                const double *lambda, const uint8_t *mask,
                                                                double *F, double *grad, double *gn2) {
  __shared__ double sh[4][8];
  const int b = idx[blockIdx.x];
  const double *H = Hk + (size_t)b * n * n;
  const double *a = A + (size_t)b * n;
  const double lam = lambda[b];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double s_part = 0.0, aa = 0.0, ya = 0.0, gg = 0.0;
  for (int i = wid; i < n; i += 8) {
    double g = 0.0;
    for (int j = lane; j < n; j += 32) g += H[(size_t)i * n + j] * a[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
    if (lane == 0) {
      const bool keep = !mask || mask[(size_t)b * n + i];
      const double gr = keep ? g + lam * a[i] - y[i] : 0.0;
      grad[(size_t)b * n + i] = gr;
      s_part += a[i] * g;
      aa += a[i] * a[i];
      ya += y[i] * a[i];
      gg += gr * gr;
    }
  }
  if (lane == 0) {
    sh[0][wid] = s_part;
    sh[1][wid] = aa;
    sh[2][wid] = ya;
    sh[3][wid] = gg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, ta = 0.0, ty = 0.0, tg = 0.0;
    for (int w = 0; w < 8; ++w) {
      S += sh[0][w];
      ta += sh[1][w];
      ty += sh[2][w];
      tg += sh[3][w];
    }
    F[b] = S / m + 0.5 * lam * ta - ty;
    gn2[b] = tg;
  }
}

int objective_from_hessian(int m, int n, int nb, const int *idx_dev, const double *Hk, const double *A,
                           const double *y, const double *lambda, const uint8_t *mask, double *F, double *grad,
                           double *gn2, cudaStream_t st) {
  k_objective_from_hessian<<<nb, 256, 0, st>>>(m, n, idx_dev, Hk, A, y, lambda, mask, F, grad, gn2);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

// Hdst[b] = Hsrc[b] for the problems whose flag is set (n x n each)
__global__ void k_take_hessians(int64_t B, int n, const double *flag, const double *Hsrc, double *Hdst) {
  const size_t nn = (size_t)n * n;
  const int64_t b = blockIdx.y;
  if (flag[b] == 0.0) return;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += (size_t)gridDim.x * blockDim.x)
    Hdst[b * nn + i] = Hsrc[b * nn + i];
}

int take_hessians(int64_t B, int n, const double *flag_dev, const double *Hsrc, double *Hdst, cudaStream_t st) {
  k_take_hessians<<<dim3(64, (unsigned)B), 256, 0, st>>>(B, n, flag_dev, Hsrc, Hdst);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

size_t newton_ws_bytes(int n, int64_t nb) {
  const int npad = (n + kNP - 1) / kNP * kNP;
  return (size_t)nb * ((size_t)npad * npad + npad) * sizeof(double) + (size_t)nb * 2 * sizeof(int);
}

// Newton directions of the problems idx[0..nb-1]: Hk holds K[a_b^{m-2}] of
// every problem b (B x n x n, indexed by problem); buffers from `ws`
// (newton_ws_bytes(n, nb) bytes).
int newton_directions(int m, int n, int nb, const int *idx_dev, const double *Hk, const double *lambda,
                      const uint8_t *mask, const double *grad, double *p, void *ws, int *bad_host,
                      cudaStream_t st) {
  const int npad = (n + kNP - 1) / kNP * kNP;
  const int nbk = npad / kNP;
  unsigned char *w = reinterpret_cast<unsigned char *>(ws);
  double *H = reinterpret_cast<double *>(w);
  double *y = H + (size_t)nb * npad * npad;
  int *bad = reinterpret_cast<int *>(y + (size_t)nb * npad);
  TK_CUDA_CHECK(cudaMemsetAsync(bad, 0, (size_t)nb * sizeof(int), st));
  dim3 gf((unsigned)((npad + 127) / 128), (unsigned)npad, (unsigned)nb);
  k_form_newton<<<gf, 128, 0, st>>>(m, n, npad, idx_dev, Hk, lambda, mask, H);
  TK_CUDA_CHECK(cudaGetLastError());
  for (int k = 0; k < nbk; ++k) {
    k_potrf_diag<<<nb, kNP * kNP, 0, st>>>(npad, k, H, bad);
    const int below = nbk - k - 1;
    if (below > 0) {
      k_trsm_panel<<<dim3((unsigned)below, (unsigned)nb), kNP * kNP, 0, st>>>(npad, k, H);
      k_syrk_update<<<dim3((unsigned)(below * (below + 1) / 2), (unsigned)nb), kNP * kNP, 0, st>>>(npad, k, nbk, H);
    }
  }
  TK_CUDA_CHECK(cudaGetLastError());
  k_chol_solve<<<nb, 256, 0, st>>>(n, npad, idx_dev, H, grad, mask, p, y);
  TK_CUDA_CHECK(cudaGetLastError());
  TK_CUDA_CHECK(cudaMemcpyAsync(bad_host, bad, (size_t)nb * sizeof(int), cudaMemcpyDeviceToHost, st));
  TK_CUDA_CHECK(cudaStreamSynchronize(st));
  return TK_OK;
}

}  // namespace tk
