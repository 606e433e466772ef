// Dual solver (Section 4, eq. dual_tensor_kernel with lambda = 1/gamma) for B
// problems over one packed tensor.  The thesis does not state its algorithm;
// F is lambda-strongly convex, so the minimiser is unique and the method only
// changes the time to reach it.  Vector algebra is FP64 on the device; the
// host reads B scalars per step (dots, objective values) to drive the
// conjugate-gradient and Armijo decisions.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "tk_internal.h"

namespace tk {

// ------------------------------------------------------------------ kernels
__global__ void k_mask(int64_t B, int n, const uint8_t *mask, double *x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B * n && mask && !mask[i]) x[i] = 0.0;
}

template <int BS>
__device__ double block_sum_fixed(double v, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < BS / 32; ++w) t += sh[w];
  return t;  // valid on thread 0
}

// out[b] = <x_b, y_b>   (one block per problem, fixed order)
__global__ void __launch_bounds__(256) k_dots(int n, const double *x, const double *y, double *out) {
  __shared__ double sh[8];
  const int64_t b = blockIdx.x;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[b * n + i] * y[b * n + i];
  s = block_sum_fixed<256>(s, sh);
  if (threadIdx.x == 0) out[b] = s;
}

// z_b = ca_b x_b + cb_b y_b  (z may alias x or y)
__global__ void k_axpby(int64_t B, int n, const double *ca, const double *x, const double *cb, const double *y,
                        double *z) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * n) return;
  const int64_t b = i / n;
  z[i] = ca[b] * x[i] + cb[b] * y[i];
}

// dst_b = src_b where flag_b
__global__ void k_select(int64_t B, int n, const double *flag, const double *src, double *dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B * n && flag[i / n] != 0.0) dst[i] = src[i];
}

// F_b = S_b/m + lambda_b/2 |a_b|^2 - <y, a_b>; grad_b = (G_b + lambda_b a_b - y) on kept points;
// gn2_b = |grad_b|^2
__global__ void __launch_bounds__(256) k_assemble(int m, int n, const double *G, const double *S, const double *A,
                                                  const double *y, const double *lambda, const uint8_t *mask,
                                                  double *F, double *grad, double *gn2) {
  __shared__ double sh[8];
  const int64_t b = blockIdx.x;
  const double lam = lambda[b];
  double ssq = 0.0, aa = 0.0, ya = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t k = b * n + i;
    const double a = A[k];
    const bool keep = !mask || mask[k];
    const double gr = keep ? G[k] + lam * a - y[i] : 0.0;
    grad[k] = gr;
    ssq += gr * gr;
    aa += a * a;
    ya += y[i] * a;
  }
  const double t0 = block_sum_fixed<256>(ssq, sh);
  const double t1 = block_sum_fixed<256>(aa, sh);
  const double t2 = block_sum_fixed<256>(ya, sh);
  if (threadIdx.x == 0) {
    F[b] = S[b] / m + 0.5 * lam * t1 - t2;
    gn2[b] = t0;
  }
}

// Hd_b = ((m-1) G_b + lambda_b d_b) on kept points
__global__ void k_hvp_finish(int m, int64_t B, int n, const double *G, const double *d, const double *lambda,
                             const uint8_t *mask, double *Hd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= B * n) return;
  const bool keep = !mask || mask[i];
  Hd[i] = keep ? (m - 1) * G[i] + lambda[i / n] * d[i] : 0.0;
}

// ------------------------------------------------------------------ host
struct SolveWs {
  unsigned char *cws;  // contraction workspace
  size_t cws_bytes;
  double *G, *g, *p, *r, *d, *Hd, *at, *gt;  // B x n each
  double *S, *F, *Ft, *gn2, *gn2t, *sc, *ca, *cb;  // B each
};

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static size_t solve_layout(int64_t B, int64_t n, size_t cws_bytes, SolveWs *w, unsigned char *base) {
  size_t off = align256(cws_bytes);
  const size_t vec = align256((size_t)B * n * sizeof(double));
  const size_t sca = align256((size_t)B * sizeof(double));
  if (w) {
    w->cws = base;
    w->cws_bytes = cws_bytes;
    double **vs[] = {&w->G, &w->g, &w->p, &w->r, &w->d, &w->Hd, &w->at, &w->gt};
    for (double **v : vs) {
      *v = reinterpret_cast<double *>(base + off);
      off += vec;
    }
    double **ss[] = {&w->S, &w->F, &w->Ft, &w->gn2, &w->gn2t, &w->sc, &w->ca, &w->cb};
    for (double **v : ss) {
      *v = reinterpret_cast<double *>(base + off);
      off += sca;
    }
    return off;
  }
  return off + 8 * vec + 8 * sca;
}

static inline unsigned grid_for(int64_t cnt) { return (unsigned)((cnt + 255) / 256); }

struct Solver {
  const tk_problem *P;
  SolveWs w;
  cudaStream_t st;
  int64_t B;
  int n, m;
  std::vector<double> h_a, h_b;  // coefficient staging

  int objective(const double *A, double *F, double *grad, double *gn2) {
    int rc = tk_contract(m, n, P->storage_dtype, P->K, B, TK_F64, A, m - 1, nullptr, w.G, w.S, w.cws, w.cws_bytes, st);
    if (rc != TK_OK) return rc;
    k_assemble<<<(unsigned)B, 256, 0, st>>>(m, n, w.G, w.S, A, P->y, P->lambda, P->mask, F, grad, gn2);
    TK_CUDA_CHECK(cudaGetLastError());
    return TK_OK;
  }
  int hvp(const double *A, const double *d, double *Hd) {
    int rc = tk_contract(m, n, P->storage_dtype, P->K, B, TK_F64, A, m - 2, d, w.G, nullptr, w.cws, w.cws_bytes, st);
    if (rc != TK_OK) return rc;
    k_hvp_finish<<<grid_for(B * n), 256, 0, st>>>(m, B, n, w.G, d, P->lambda, P->mask, Hd);
    TK_CUDA_CHECK(cudaGetLastError());
    return TK_OK;
  }
  int dots(const double *x, const double *y, std::vector<double> &out) {
    k_dots<<<(unsigned)B, 256, 0, st>>>(n, x, y, w.sc);
    TK_CUDA_CHECK(cudaGetLastError());
    TK_CUDA_CHECK(cudaMemcpyAsync(out.data(), w.sc, B * sizeof(double), cudaMemcpyDeviceToHost, st));
    TK_CUDA_CHECK(cudaStreamSynchronize(st));
    return TK_OK;
  }
  int fetch(const double *dev, std::vector<double> &out) {
    TK_CUDA_CHECK(cudaMemcpyAsync(out.data(), dev, B * sizeof(double), cudaMemcpyDeviceToHost, st));
    TK_CUDA_CHECK(cudaStreamSynchronize(st));
    return TK_OK;
  }
  // z = a x + b y with per-problem coefficients
  int axpby(const std::vector<double> &a, const double *x, const std::vector<double> &b, const double *y, double *z) {
    TK_CUDA_CHECK(cudaMemcpyAsync(w.ca, a.data(), B * sizeof(double), cudaMemcpyHostToDevice, st));
    TK_CUDA_CHECK(cudaMemcpyAsync(w.cb, b.data(), B * sizeof(double), cudaMemcpyHostToDevice, st));
    k_axpby<<<grid_for(B * n), 256, 0, st>>>(B, n, w.ca, x, w.cb, y, z);
    TK_CUDA_CHECK(cudaGetLastError());
    return TK_OK;
  }
  int select(const std::vector<double> &flag, const double *src, double *dst) {
    TK_CUDA_CHECK(cudaMemcpyAsync(w.ca, flag.data(), B * sizeof(double), cudaMemcpyHostToDevice, st));
    k_select<<<grid_for(B * n), 256, 0, st>>>(B, n, w.ca, src, dst);
    TK_CUDA_CHECK(cudaGetLastError());
    return TK_OK;
  }
};

}  // namespace tk

using namespace tk;

extern "C" size_t tk_solve_workspace_size(const tk_problem *P) {
  if (!P) return 0;
  const size_t cws = tk_contract_workspace_size(P->m, P->n, P->B);
  if (cws == 0) return 0;
  return solve_layout(P->B, P->n, cws, nullptr, nullptr);
}

#define TK_TRY(x)                  \
  do {                             \
    int rc__ = (x);                \
    if (rc__ != TK_OK) return rc__; \
  } while (0)

extern "C" int tk_solve_dual(const tk_problem *P, const tk_solve_opts *O, double *A, tk_solve_report *R, void *work,
                             size_t work_bytes, void *stream) {
  if (!P || !O || !A || !R || !work) return fail(TK_EINVAL, "NULL argument");
  if (P->B < 1 || !P->K || !P->y || !P->lambda) return fail(TK_EINVAL, "bad problem");
  if (O->method != TK_NEWTON_CG && O->method != TK_GD_BT) return fail(TK_EINVAL, "unknown method %d", O->method);
  if (O->max_iter < 0 || O->tol_gradnorm < 0) return fail(TK_EINVAL, "bad options");
  const size_t need = tk_solve_workspace_size(P);
  if (need == 0) return TK_EINVAL;
  if (work_bytes < need) return fail(TK_ENOMEM, "workspace %zu < %zu bytes", work_bytes, need);
  Solver s;
  s.P = P;
  s.st = reinterpret_cast<cudaStream_t>(stream);
  s.B = P->B;
  s.n = (int)P->n;
  s.m = P->m;
  solve_layout(P->B, P->n, tk_contract_workspace_size(P->m, P->n, P->B), &s.w, reinterpret_cast<unsigned char *>(work));
  const int64_t B = s.B;
  const int n = s.n;
  const double c_arm = O->armijo_c > 0 ? O->armijo_c : 1e-4;
  const int max_cg = O->max_cg > 0 ? O->max_cg : std::max(1, std::min(n, 200));
  const double tol = O->tol_gradnorm;

  std::vector<double> F(B), gn2(B), Ft(B), gn2t(B), rr(B), rr_new(B), dHd(B), slope(B), t(B), gstep(B, 0.0);
  std::vector<double> one(B, 1.0), zero(B, 0.0), minus1(B, -1.0), ca(B), cb(B), flag(B);
  std::vector<int> status(B, TK_ENOTCONV), iters(B, 0), passes(B, 0);
  std::vector<char> active(B, 1), stalled(B, 0);

  if (P->mask) {
    k_mask<<<grid_for(B * n), 256, 0, s.st>>>(B, n, P->mask, A);
    TK_CUDA_CHECK(cudaGetLastError());
  }
  TK_TRY(s.objective(A, s.w.F, s.w.g, s.w.gn2));
  for (auto &x : passes) ++x;
  TK_TRY(s.fetch(s.w.F, F));
  TK_TRY(s.fetch(s.w.gn2, gn2));

  for (int it = 0; it < O->max_iter; ++it) {
    bool any = false;
    for (int64_t b = 0; b < B; ++b) {
      active[b] = !stalled[b] && sqrt(gn2[b]) > tol;
      if (!active[b] && !stalled[b]) status[b] = TK_OK;
      any |= active[b];
    }
    if (!any) break;
    for (int64_t b = 0; b < B; ++b) iters[b] += active[b];

    if (O->method == TK_NEWTON_CG) {
      // p = 0, r = -g, d = r
      TK_TRY(s.axpby(zero, s.w.g, zero, s.w.g, s.w.p));
      TK_TRY(s.axpby(minus1, s.w.g, zero, s.w.g, s.w.r));
      TK_TRY(s.axpby(one, s.w.r, zero, s.w.r, s.w.d));
      TK_TRY(s.dots(s.w.r, s.w.r, rr));
      std::vector<char> cg(B);
      std::vector<double> eta(B);
      for (int64_t b = 0; b < B; ++b) {
        cg[b] = active[b];
        eta[b] = std::min(0.5, sqrt(sqrt(gn2[b])));
      }
      for (int k = 0; k < max_cg; ++k) {
        TK_TRY(s.hvp(A, s.w.d, s.w.Hd));
        for (int64_t b = 0; b < B; ++b) passes[b] += cg[b];
        TK_TRY(s.dots(s.w.d, s.w.Hd, dHd));
        for (int64_t b = 0; b < B; ++b) {
          ca[b] = (cg[b] && dHd[b] > 0) ? rr[b] / dHd[b] : 0.0;
          if (cg[b] && !(dHd[b] > 0)) cg[b] = 0;  // (H is positive definite; guards rounding)
        }
        std::vector<double> nca(B);
        for (int64_t b = 0; b < B; ++b) nca[b] = -ca[b];
        TK_TRY(s.axpby(one, s.w.p, ca, s.w.d, s.w.p));
        TK_TRY(s.axpby(one, s.w.r, nca, s.w.Hd, s.w.r));
        TK_TRY(s.dots(s.w.r, s.w.r, rr_new));
        bool more = false;
        for (int64_t b = 0; b < B; ++b) {
          if (cg[b] && sqrt(rr_new[b]) <= eta[b] * sqrt(gn2[b])) cg[b] = 0;
          cb[b] = cg[b] ? rr_new[b] / rr[b] : 0.0;
          rr[b] = rr_new[b];
          more |= cg[b];
        }
        if (!more) break;
        TK_TRY(s.axpby(one, s.w.r, cb, s.w.d, s.w.d));
      }
      for (int64_t b = 0; b < B; ++b) t[b] = 1.0;
    } else {
      TK_TRY(s.axpby(minus1, s.w.g, zero, s.w.g, s.w.p));
      for (int64_t b = 0; b < B; ++b) t[b] = gstep[b] > 0 ? 2.0 * gstep[b] : 1.0 / std::max(1.0, sqrt(gn2[b]));
    }
    TK_TRY(s.dots(s.w.g, s.w.p, slope));
    for (int64_t b = 0; b < B; ++b) {
      if (active[b] && !(slope[b] < 0)) {
        // not a descent direction (rounding in the inner solve): fall back to -grad
        slope[b] = -gn2[b];
      }
    }
    // directions of problems whose slope was repaired: p = -g
    for (int64_t b = 0; b < B; ++b) flag[b] = (active[b] && slope[b] == -gn2[b] && O->method == TK_NEWTON_CG) ? 1.0 : 0.0;
    TK_TRY(s.axpby(minus1, s.w.g, zero, s.w.g, s.w.at));
    TK_TRY(s.select(flag, s.w.at, s.w.p));

    // Armijo backtracking, all problems in lockstep
    std::vector<char> ls(B);
    std::vector<double> accepted(B, 0.0);
    for (int64_t b = 0; b < B; ++b) ls[b] = active[b];
    for (int tries = 0; tries < 80; ++tries) {
      for (int64_t b = 0; b < B; ++b) {
        ca[b] = 1.0;
        cb[b] = ls[b] ? t[b] : 0.0;
      }
      TK_TRY(s.axpby(ca, A, cb, s.w.p, s.w.at));
      TK_TRY(s.objective(s.w.at, s.w.Ft, s.w.gt, s.w.gn2t));
      TK_TRY(s.fetch(s.w.Ft, Ft));
      TK_TRY(s.fetch(s.w.gn2t, gn2t));
      bool more = false;
      for (int64_t b = 0; b < B; ++b) {
        if (!ls[b]) continue;
        ++passes[b];
        // Armijo sufficient decrease; once the decrease is below the rounding
        // level of F itself, a smaller gradient norm decides instead
        const bool armijo = Ft[b] <= F[b] + c_arm * t[b] * slope[b];
        const bool in_noise = fabs(Ft[b] - F[b]) <= 1e-12 * std::max(1.0, fabs(F[b])) && gn2t[b] < gn2[b];
        if (armijo || in_noise) {
          ls[b] = 0;
          accepted[b] = 1.0;
        } else {
          t[b] *= 0.5;
          if (t[b] < 1e-30) {
            ls[b] = 0;
            stalled[b] = 1;
          } else {
            more = true;
          }
        }
      }
      if (!more) break;
    }
    for (int64_t b = 0; b < B; ++b)
      if (ls[b]) stalled[b] = 1;
    // take the accepted trial points (and their objective and gradient)
    TK_TRY(s.select(accepted, s.w.at, A));
    TK_TRY(s.select(accepted, s.w.gt, s.w.g));
    for (int64_t b = 0; b < B; ++b) {
      if (accepted[b] != 0.0) {
        F[b] = Ft[b];
        gn2[b] = gn2t[b];
        gstep[b] = t[b];
      }
    }
  }
  for (int64_t b = 0; b < B; ++b) {
    if (sqrt(gn2[b]) <= tol) status[b] = TK_OK;
    R[b].iters = iters[b];
    R[b].passes = passes[b];
    R[b].gradnorm = sqrt(gn2[b]);
    R[b].F = F[b];
    R[b].status = status[b];
  }
  TK_CUDA_CHECK(cudaStreamSynchronize(s.st));
  for (int64_t b = 0; b < B; ++b)
    if (R[b].status != TK_OK) return fail(TK_ENOTCONV, "problem %lld stopped at |grad F| = %.3e", (long long)b, R[b].gradnorm);
  return TK_OK;
}
