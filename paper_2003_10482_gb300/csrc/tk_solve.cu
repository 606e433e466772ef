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

size_t newton_ws_bytes(int n, int64_t nb);
int newton_directions(int m, int n, int nb, const int *idx_dev, const double *Hk, const double *lambda,
                      const uint8_t *mask, const double *grad, double *p, void *ws, int *bad_host,
                      cudaStream_t st);
int objective_from_hessian(int m, int n, int nb, const int *idx_dev, const double *Hk, const double *A,
                           const double *y, const double *lambda, const uint8_t *mask, double *F, double *grad,
                           double *gn2, cudaStream_t st);
int take_hessians(int64_t B, int n, const double *flag_dev, const double *Hsrc, double *Hdst, cudaStream_t st);

// problems whose Newton systems are formed and factorised together
constexpr int kNewtonChunk = 64;

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

// x_b = y for every problem b
__global__ void k_fill_y(int64_t B, int n, const double *y, double *x) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < B * n) x[i] = y[i % n];
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

// dst_j = src_{idx_j}  (gathers the rows of the problems in a pass)
__global__ void k_gather(int64_t nb, int n, const int *idx, const double *src, double *dst) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * n) return;
  const int64_t j = i / n;
  dst[i] = src[(int64_t)idx[j] * n + (i - j * n)];
}

// k_assemble for the compacted problems: row j of G and S belongs to problem idx_j
__global__ void __launch_bounds__(256) k_assemble_idx(int m, int n, const int *idx, const double *G,
                                                      const double *S, const double *A, const double *y,
                                                      const double *lambda, const uint8_t *mask, double *F,
                                                      double *grad, double *gn2) {
  __shared__ double sh[8];
  const int64_t j = blockIdx.x;
  const int64_t b = idx[j];
  const double lam = lambda[b];
  double ssq = 0.0, aa = 0.0, ya = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int64_t k = b * n + i;
    const double a = A[k];
    const bool keep = !mask || mask[k];
    const double gr = keep ? G[j * n + i] + lam * a - y[i] : 0.0;
    grad[k] = gr;
    ssq += gr * gr;
    aa += a * a;
    ya += y[i] * a;
  }
  const double t0 = block_sum_fixed<256>(ssq, sh);
  const double t1 = block_sum_fixed<256>(aa, sh);
  const double t2 = block_sum_fixed<256>(ya, sh);
  if (threadIdx.x == 0) {
    F[b] = S[j] / m + 0.5 * lam * t1 - t2;
    gn2[b] = t0;
  }
}

// k_hvp_finish for the compacted problems
__global__ void k_hvp_finish_idx(int m, int64_t nb, int n, const int *idx, const double *G, const double *d,
                                 const double *lambda, const uint8_t *mask, double *Hd) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * n) return;
  const int64_t j = i / n;
  const int64_t b = idx[j];
  const int64_t k = b * n + (i - j * n);
  const bool keep = !mask || mask[k];
  Hd[k] = keep ? (m - 1) * G[i] + lambda[b] * d[k] : 0.0;
}

// ------------------------------------------------------------------ host
struct SolveWs {
  unsigned char *cws;  // contraction workspace
  size_t cws_bytes;
  double *G, *g, *p, *r, *d, *Hd, *at, *gt, *Ac, *dc;  // B x n each (Ac, dc: compacted rows)
  double *S, *F, *Ft, *gn2, *gn2t, *sc, *ca, *cb;  // B each
  int *idx;                                         // B problem indices of a compacted pass
};

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static size_t solve_layout(int64_t B, int64_t n, size_t cws_bytes, SolveWs *w, unsigned char *base) {
  size_t off = align256(cws_bytes);
  const size_t vec = align256((size_t)B * n * sizeof(double));
  const size_t sca = align256((size_t)B * sizeof(double));
  if (w) {
    w->cws = base;
    w->cws_bytes = cws_bytes;
    double **vs[] = {&w->G, &w->g, &w->p, &w->r, &w->d, &w->Hd, &w->at, &w->gt, &w->Ac, &w->dc};
    for (double **v : vs) {
      *v = reinterpret_cast<double *>(base + off);
      off += vec;
    }
    double **ss[] = {&w->S, &w->F, &w->Ft, &w->gn2, &w->gn2t, &w->sc, &w->ca, &w->cb};
    for (double **v : ss) {
      *v = reinterpret_cast<double *>(base + off);
      off += sca;
    }
    w->idx = reinterpret_cast<int *>(base + off);
    off += align256((size_t)B * sizeof(int));
    return off;
  }
  return off + 10 * vec + 8 * sca + align256((size_t)B * sizeof(int));
}

static inline unsigned grid_for(int64_t cnt) { return (unsigned)((cnt + 255) / 256); }

struct Solver {
  const tk_problem *P;
  SolveWs w;
  cudaStream_t st;
  int64_t B;
  int n, m;
  std::vector<double> h_a, h_b;  // coefficient staging

  // the tensor the Hessian-vector passes read (the optional second copy)
  const void *hvp_tensor() const { return P->K_hvp ? P->K_hvp : P->K; }
  int hvp_storage() const { return P->K_hvp ? P->hvp_storage_dtype : P->storage_dtype; }

  // full-Hessian Newton: every objective evaluation is a Hessian pass at the
  // point (K[a^{m-1}] = K[a^{m-2}] a and K[a^m] = a . K[a^{m-1}]), whose
  // matrices land in hdst (B x n x n, by problem) for the next Newton system
  bool full = false;
  double *hdst = nullptr;
  unsigned char *hws = nullptr;
  size_t hws_bytes = 0;
  int *hidx = nullptr;  // device list of problems (B ints)
  int hess_objective(const std::vector<int> &list, const double *A, double *F, double *grad, double *gn2) {
    if (list.empty()) return TK_OK;
    for (int b : list) {
      int rc = tk_hessian(m, n, P->storage_dtype, P->K, A + (size_t)b * n, hdst + (size_t)b * n * n, hws, hws_bytes,
                          st);
      if (rc != TK_OK) return rc;
    }
    TK_CUDA_CHECK(cudaMemcpyAsync(hidx, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    return objective_from_hessian(m, n, (int)list.size(), hidx, hdst, A, P->y, P->lambda, P->mask, F, grad, gn2, st);
  }

  // Objective (or HVP) of the problems in `list` only: their rows are gathered,
  // contracted as one smaller batch and the results scattered back; rows of
  // the other problems in F / grad / gn2 (or Hd) are left as they are.
  int set_list(const std::vector<int> &list) {
    TK_CUDA_CHECK(cudaMemcpyAsync(w.idx, list.data(), list.size() * sizeof(int), cudaMemcpyHostToDevice, st));
    return TK_OK;
  }
  int objective_sub(const std::vector<int> &list, const double *A, double *F, double *grad, double *gn2) {
    if (full) return hess_objective(list, A, F, grad, gn2);
    const int64_t nb = (int64_t)list.size();
    if (nb == 0) return TK_OK;
    if (nb == B) return objective(A, F, grad, gn2);
    int rc = set_list(list);
    if (rc != TK_OK) return rc;
    k_gather<<<grid_for(nb * n), 256, 0, st>>>(nb, n, w.idx, A, w.Ac);
    TK_CUDA_CHECK(cudaGetLastError());
    rc = tk_contract(m, n, P->storage_dtype, P->K, nb, TK_F64, w.Ac, m - 1, nullptr, w.G, w.S, w.cws, w.cws_bytes, st);
    if (rc != TK_OK) return rc;
    k_assemble_idx<<<(unsigned)nb, 256, 0, st>>>(m, n, w.idx, w.G, w.S, A, P->y, P->lambda, P->mask, F, grad, gn2);
    TK_CUDA_CHECK(cudaGetLastError());
    return TK_OK;
  }
  int hvp_sub(const std::vector<int> &list, const double *A, const double *d, double *Hd) {
    const int64_t nb = (int64_t)list.size();
    if (nb == 0) return TK_OK;
    if (nb == B) return hvp(A, d, Hd);
    int rc = set_list(list);
    if (rc != TK_OK) return rc;
    k_gather<<<grid_for(nb * n), 256, 0, st>>>(nb, n, w.idx, A, w.Ac);
    k_gather<<<grid_for(nb * n), 256, 0, st>>>(nb, n, w.idx, d, w.dc);
    TK_CUDA_CHECK(cudaGetLastError());
    rc = tk_contract(m, n, hvp_storage(), hvp_tensor(), nb, TK_F64, w.Ac, m - 2, w.dc, w.G, nullptr, w.cws,
                     w.cws_bytes, st);
    if (rc != TK_OK) return rc;
    k_hvp_finish_idx<<<grid_for(nb * n), 256, 0, st>>>(m, nb, n, w.idx, w.G, d, P->lambda, P->mask, Hd);
    TK_CUDA_CHECK(cudaGetLastError());
    return TK_OK;
  }
  int objective(const double *A, double *F, double *grad, double *gn2) {
    if (full) {
      std::vector<int> all(B);
      for (int64_t b = 0; b < B; ++b) all[b] = (int)b;
      return hess_objective(all, A, F, grad, gn2);
    }
    int rc = tk_contract(m, n, P->storage_dtype, P->K, B, TK_F64, A, m - 1, nullptr, w.G, w.S, w.cws, w.cws_bytes, st);
    if (rc != TK_OK) return rc;
    k_assemble<<<(unsigned)B, 256, 0, st>>>(m, n, w.G, w.S, A, P->y, P->lambda, P->mask, F, grad, gn2);
    TK_CUDA_CHECK(cudaGetLastError());
    return TK_OK;
  }
  int hvp(const double *A, const double *d, double *Hd) {
    int rc = tk_contract(m, n, hvp_storage(), hvp_tensor(), B, TK_F64, A, m - 2, d, w.G, nullptr, w.cws,
                         w.cws_bytes, st);
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

// extra bytes of the full-Hessian Newton method, after the common layout:
// the Hessian pass's workspace, K[a^{m-2}] of every problem at its current
// point and at its trial point, the Newton matrices and factors of one chunk
// of problems, the device list of problems
struct FullLayout {
  size_t hws, hcur, htrial, nws, hidx, total;
};
static FullLayout full_layout(const tk_problem *P) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  FullLayout L{};
  const size_t hws = tk_hessian_workspace_size(P->m, P->n);
  if (hws == 0) return L;
  const size_t mats = al((size_t)P->B * P->n * P->n * sizeof(double));
  size_t off = 0;
  L.hws = off;
  off += al(hws);
  L.hcur = off;
  off += mats;
  L.htrial = off;
  off += mats;
  L.nws = off;
  off += al(newton_ws_bytes((int)P->n, std::min<int64_t>(P->B, kNewtonChunk)));
  L.hidx = off;
  off += al((size_t)P->B * sizeof(int));
  L.total = off;
  return L;
}

extern "C" size_t tk_solve_workspace_size_opts(const tk_problem *P, const tk_solve_opts *O) {
  const size_t base = tk_solve_workspace_size(P);
  if (base == 0 || !O) return base;
  if (O->method != TK_NEWTON_FULL) return base;
  const size_t extra = full_layout(P).total;
  return extra == 0 ? 0 : ((base + 255) & ~size_t(255)) + extra;
}

extern "C" int tk_dual_hvp(int m, int64_t n, int storage, const void *K, int64_t B, const double *A, const double *V,
                           const double *lambda, double *HV, void *work, size_t work_bytes, void *stream) {
  if (B < 0) return fail(TK_EINVAL, "B < 0");
  if (B == 0) return TK_OK;
  if (!lambda || !HV || !V) return fail(TK_EINVAL, "NULL pointer");
  // K[a^{m-2}, v] into HV, then HV = (m-1) HV + lambda v in place
  int rc = tk_contract(m, n, storage, K, B, TK_F64, A, m - 2, V, HV, nullptr, work, work_bytes, stream);
  if (rc != TK_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_hvp_finish<<<grid_for(B * n), 256, 0, st>>>(m, B, (int)n, HV, V, lambda, nullptr, HV);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

// Next trial step after a rejected one: the minimiser of the cubic that
// matches F and its slope along p at 0 and at t (Hermite interpolation; the
// form of Nocedal and Wright, Numerical Optimization, eq. 3.59), kept in
// [0.1 t, 0.5 t]; halving when the cubic gives no usable minimiser.  Along a
// Newton direction F is a polynomial of degree m in the step, which the cubic
// follows far more closely than halving does.
static double backtrack_step(double t, double f0, double g0, double f1, double g1) {
  const double d1 = g0 + g1 - 3.0 * (f1 - f0) / t;
  const double disc = d1 * d1 - g0 * g1;
  double tn = 0.5 * t;
  if (std::isfinite(disc) && disc >= 0.0 && std::isfinite(f1) && std::isfinite(g1)) {
    const double d2 = sqrt(disc);
    const double den = g1 - g0 + 2.0 * d2;
    if (den != 0.0) {
      const double c = t - t * (g1 + d2 - d1) / den;
      if (std::isfinite(c)) tn = c;
    }
  }
  return std::min(0.5 * t, std::max(0.1 * t, tn));
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
  if (P->K_hvp && (P->hvp_storage_dtype < TK_F64 || P->hvp_storage_dtype > TK_BF16))
    return fail(TK_EINVAL, "bad storage dtype %d of the Hessian-vector tensor", P->hvp_storage_dtype);
  if (O->method != TK_NEWTON_CG && O->method != TK_GD_BT && O->method != TK_NEWTON_FULL)
    return fail(TK_EINVAL, "unknown method %d", O->method);
  if (O->max_iter < 0 || O->tol_gradnorm < 0 || O->tol_rel_gap < 0) return fail(TK_EINVAL, "bad options");
  const size_t need = tk_solve_workspace_size_opts(P, O);
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
  const bool newton = O->method == TK_NEWTON_CG || O->method == TK_NEWTON_FULL;
  // full-Hessian Newton buffers (after the common layout)
  double *Hcur = nullptr, *Htrial = nullptr;
  unsigned char *nws = nullptr;
  if (O->method == TK_NEWTON_FULL) {
    unsigned char *base = reinterpret_cast<unsigned char *>(work) + ((tk_solve_workspace_size(P) + 255) & ~size_t(255));
    const FullLayout L = full_layout(P);
    // without a second tensor every evaluation is a Hessian pass over K (it
    // gives F and grad F too); with one, F and grad F come from contraction
    // passes over K and the Hessian of each new point from a pass over K_hvp
    s.full = P->K_hvp == nullptr;
    s.hws = base + L.hws;
    // this region's offset in the workspace depends on B: a plan recorded
    // here by an earlier call may have been overwritten since (by that call's
    // matrices at another B), so the pass uploads its plan afresh
    forget_hessian_plan(s.hws);
    s.hws_bytes = L.hcur - L.hws;
    Hcur = reinterpret_cast<double *>(base + L.hcur);
    Htrial = reinterpret_cast<double *>(base + L.htrial);
    nws = base + L.nws;
    s.hidx = reinterpret_cast<int *>(base + L.hidx);
    s.hdst = Hcur;
  }

  std::vector<double> F(B), gn2(B), Ft(B), gn2t(B), rr(B), rr_new(B), dHd(B), slope(B), slope_t(B), t(B), gstep(B, 0.0);
  // stall detection: best gradient norm so far and iterations since it last fell by 0.1 %
  std::vector<double> best_gn2(B, 0.0);
  std::vector<int> since_best(B, 0);
  const int kStallIters = 8;
  std::vector<double> one(B, 1.0), zero(B, 0.0), minus1(B, -1.0), ca(B), cb(B), flag(B);
  std::vector<int> status(B, TK_ENOTCONV), iters(B, 0), passes(B, 0);
  std::vector<char> active(B, 1), stalled(B, 0);
  // non-positive curvature met in the inner solve: with the exact tensor the
  // Hessian (m-1) K[a^{m-2}] + lambda I is positive definite, so only a rounded
  // (FP32/BF16) stored tensor can show it -- its form is indefinite at the iterate
  std::vector<char> indefinite(B, 0);

  if (O->start_on_y) {
    // a_b = s_b y_b with s_b = argmin_s F(s y_b): F along the ray is the
    // polynomial s^m S_b/m + lambda_b s^2 |y_b|^2 / 2 - s |y_b|^2 with
    // S_b = K[y_b^m] from one contraction pass; its derivative
    // S_b s^{m-1} + (lambda_b s - 1)|y_b|^2 rises from -|y_b|^2 at 0 to
    // S_b / lambda_b^{m-1} >= 0 at 1/lambda_b (m even), so bisection finds the root
    k_fill_y<<<grid_for(B * n), 256, 0, s.st>>>(B, n, P->y, A);
    TK_CUDA_CHECK(cudaGetLastError());
    if (P->mask) {
      k_mask<<<grid_for(B * n), 256, 0, s.st>>>(B, n, P->mask, A);
      TK_CUDA_CHECK(cudaGetLastError());
    }
    TK_TRY(tk_contract(s.m, n, P->storage_dtype, P->K, B, TK_F64, A, s.m - 1, nullptr, s.w.G, s.w.S, s.w.cws,
                       s.w.cws_bytes, s.st));
    for (auto &x : passes) ++x;
    std::vector<double> Sy(B), yy(B), lam(B), sc(B), zero_b(B, 0.0);
    TK_TRY(s.fetch(s.w.S, Sy));
    TK_TRY(s.dots(A, A, yy));
    TK_CUDA_CHECK(cudaMemcpyAsync(lam.data(), P->lambda, B * sizeof(double), cudaMemcpyDeviceToHost, s.st));
    TK_CUDA_CHECK(cudaStreamSynchronize(s.st));
    for (int64_t b = 0; b < B; ++b) {
      double lo = 0.0, hi = 1.0 / lam[b];
      if (!(yy[b] > 0.0) || !(lam[b] > 0.0)) {
        sc[b] = 0.0;
        continue;
      }
      for (int k = 0; k < 200; ++k) {
        const double mid = 0.5 * (lo + hi);
        const double d = Sy[b] * pow(mid, s.m - 1) + (lam[b] * mid - 1.0) * yy[b];
        if (d < 0.0) lo = mid; else hi = mid;
      }
      sc[b] = 0.5 * (lo + hi);
    }
    TK_TRY(s.axpby(sc, A, zero_b, A, A));
  } else if (P->mask) {
    k_mask<<<grid_for(B * n), 256, 0, s.st>>>(B, n, P->mask, A);
    TK_CUDA_CHECK(cudaGetLastError());
  }
  // The floor of F for an exact tensor of even order: K[a^m] >= 0, so
  // F(a) >= (lambda/2)|a|^2 - <y, a> >= -|y|^2 / (2 lambda) over the kept
  // points.  A computed F below it certifies that the stored tensor's form is
  // negative at the point (its rounding has made it indefinite): the problem
  // stops there, not at the end of a run-off along the null space of X^T.
  std::vector<double> yk2(B), lam_b(B);
  k_fill_y<<<grid_for(B * n), 256, 0, s.st>>>(B, n, P->y, s.w.at);
  TK_CUDA_CHECK(cudaGetLastError());
  if (P->mask) {
    k_mask<<<grid_for(B * n), 256, 0, s.st>>>(B, n, P->mask, s.w.at);
    TK_CUDA_CHECK(cudaGetLastError());
  }
  TK_TRY(s.dots(s.w.at, s.w.at, yk2));
  TK_CUDA_CHECK(cudaMemcpyAsync(lam_b.data(), P->lambda, B * sizeof(double), cudaMemcpyDeviceToHost, s.st));
  TK_CUDA_CHECK(cudaStreamSynchronize(s.st));
  auto below_floor = [&](int64_t b, double Fv) {
    return lam_b[b] > 0.0 && Fv < -(1.0 + 1e-9) * yk2[b] / (2.0 * lam_b[b]);
  };

  TK_TRY(s.objective(A, s.w.F, s.w.g, s.w.gn2));
  for (auto &x : passes) ++x;
  TK_TRY(s.fetch(s.w.F, F));
  TK_TRY(s.fetch(s.w.gn2, gn2));
  for (int64_t b = 0; b < B; ++b) {
    best_gn2[b] = gn2[b];
    if (below_floor(b, F[b])) {
      indefinite[b] = 1;
      stalled[b] = 1;
    }
  }

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
      std::vector<int> list;
      for (int k = 0; k < max_cg; ++k) {
        list.clear();
        for (int64_t b = 0; b < B; ++b)
          if (cg[b]) list.push_back((int)b);
        TK_TRY(s.hvp_sub(list, A, s.w.d, s.w.Hd));
        for (int64_t b = 0; b < B; ++b) passes[b] += cg[b];
        TK_TRY(s.dots(s.w.d, s.w.Hd, dHd));
        for (int64_t b = 0; b < B; ++b) {
          ca[b] = (cg[b] && dHd[b] > 0) ? rr[b] / dHd[b] : 0.0;
          if (cg[b] && !(dHd[b] > 0)) {  // (H is positive definite; guards rounding)
            cg[b] = 0;
            indefinite[b] = 1;
          }
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
    } else if (O->method == TK_NEWTON_FULL) {
      // p = -H^{-1} g with H = (m-1) K[a^{m-2}] + lambda I from the Hessian pass
      // that evaluated the current point; systems factorised in chunks
      std::vector<int> list;
      for (int64_t b = 0; b < B; ++b)
        if (active[b]) list.push_back((int)b);
      if (!s.full) {
        for (int b : list) {
          TK_TRY(tk_hessian(s.m, n, P->hvp_storage_dtype, P->K_hvp, A + (size_t)b * n, Hcur + (size_t)b * n * n, s.hws,
                            s.hws_bytes, s.st));
          ++passes[b];
        }
      }
      TK_TRY(s.axpby(zero, s.w.g, zero, s.w.g, s.w.p));
      for (size_t c0 = 0; c0 < list.size(); c0 += kNewtonChunk) {
        const int nb = (int)std::min<size_t>(kNewtonChunk, list.size() - c0);
        TK_CUDA_CHECK(cudaMemcpyAsync(s.hidx, list.data() + c0, nb * sizeof(int), cudaMemcpyHostToDevice, s.st));
        std::vector<int> bad(nb, 0);
        TK_TRY(newton_directions(s.m, n, nb, s.hidx, Hcur, P->lambda, P->mask, s.w.g, s.w.p, nws, bad.data(), s.st));
        for (int j = 0; j < nb; ++j)
          if (bad[j]) {
            // (m-1) K[a^{m-2}] + lambda I is positive definite for a tensor
            // kernel of even order: a failed factorisation shows that the
            // stored tensor's rounding has broken the form at this iterate,
            // where F has no minimiser to approach; the problem stops here
            const int b = list[c0 + j];
            indefinite[b] = 1;
            active[b] = 0;
            stalled[b] = 1;
          }
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
      } else if (active[b] && newton && O->tol_rel_gap > 0 &&
                 -0.5 * slope[b] <= O->tol_rel_gap * std::max(1.0, fabs(F[b]))) {
        // Newton decrement: F - F* ~ -<g, p>/2 is below the relative tolerance
        active[b] = 0;
        status[b] = TK_OK;
        stalled[b] = 1;  // stays finished
      }
    }
    // directions of problems whose slope was repaired: p = -g
    for (int64_t b = 0; b < B; ++b) flag[b] = (active[b] && slope[b] == -gn2[b] && newton) ? 1.0 : 0.0;
    TK_TRY(s.axpby(minus1, s.w.g, zero, s.w.g, s.w.at));
    TK_TRY(s.select(flag, s.w.at, s.w.p));

    // Armijo backtracking, all problems in lockstep; a problem whose step has
    // shrunk 1e8-fold without an accepted point has met its rounding floor
    s.hdst = Htrial;
    std::vector<double> t_first(t);
    std::vector<char> ls(B);
    std::vector<double> accepted(B, 0.0);
    std::vector<char> real_decrease(B, 0);  // accepted by Armijo's test (a decrease F's rounding cannot fake)
    for (int64_t b = 0; b < B; ++b) ls[b] = active[b];
    // at most 10 trials: each shrinks the step 2-10-fold (cubic interpolation),
    // so ten rejections mean F's rounding, not the step, decides
    for (int tries = 0; tries < 10; ++tries) {
      for (int64_t b = 0; b < B; ++b) {
        ca[b] = 1.0;
        // problems that accepted a step keep it: the shared trial buffers
        // (at, gt, Ft) must still hold their accepted point after the others'
        // further trials
        cb[b] = (ls[b] || accepted[b] != 0.0) ? t[b] : 0.0;
      }
      TK_TRY(s.axpby(ca, A, cb, s.w.p, s.w.at));
      std::vector<int> list;
      for (int64_t b = 0; b < B; ++b)
        if (ls[b]) list.push_back((int)b);
      TK_TRY(s.objective_sub(list, s.w.at, s.w.Ft, s.w.gt, s.w.gn2t));
      TK_TRY(s.fetch(s.w.Ft, Ft));
      TK_TRY(s.fetch(s.w.gn2t, gn2t));
      TK_TRY(s.dots(s.w.gt, s.w.p, slope_t));
      bool more = false;
      for (int64_t b = 0; b < B; ++b) {
        if (!ls[b]) continue;
        ++passes[b];
        if (below_floor(b, Ft[b])) {  // the stored form is negative at the trial point
          ls[b] = 0;
          stalled[b] = 1;
          indefinite[b] = 1;
          continue;
        }
        // Armijo sufficient decrease; once the decrease is below the rounding
        // level of F itself, a smaller gradient norm decides instead; a
        // non-positive slope at the trial point certifies decrease (F is
        // convex along the line) when F's rounding hides it
        const bool armijo = Ft[b] <= F[b] + c_arm * t[b] * slope[b];
        const bool in_noise = fabs(Ft[b] - F[b]) <= 1e-12 * std::max(1.0, fabs(F[b])) && gn2t[b] < gn2[b];
        const bool downhill = slope_t[b] <= 0.0 && std::isfinite(Ft[b]);
        if (armijo || in_noise || downhill) {
          ls[b] = 0;
          accepted[b] = 1.0;
          real_decrease[b] = armijo && Ft[b] < F[b] - 1e-12 * std::max(1.0, fabs(F[b]));
        } else {
          t[b] = backtrack_step(t[b], F[b], slope[b], Ft[b], slope_t[b]);
          if (t[b] < 1e-8 * t_first[b]) {
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
    if (s.full) {
      // the accepted points' Hessians become the current ones (s.w.ca holds
      // the accepted flags the selects just uploaded)
      TK_TRY(take_hessians(B, n, s.w.ca, Htrial, Hcur, s.st));
      s.hdst = Hcur;
    }
    for (int64_t b = 0; b < B; ++b) {
      if (accepted[b] != 0.0) {
        F[b] = Ft[b];
        gn2[b] = gn2t[b];
        gstep[b] = t[b];
      }
      if (active[b] && !stalled[b]) {
        // progress: a decrease of F beyond its rounding level, or |grad| below
        // 0.999 of its best (the damped phase may raise |grad| while F falls)
        const bool better_g = gn2[b] < 0.998 * best_gn2[b];
        if (better_g) best_gn2[b] = gn2[b];
        if (better_g || real_decrease[b]) {
          since_best[b] = 0;
        } else if (++since_best[b] >= kStallIters) {
          stalled[b] = 1;  // the rounding floor of the contraction: no further progress
        }
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
    if (R[b].status != TK_OK)
      return fail(TK_ENOTCONV, "problem %lld stopped at |grad F| = %.3e%s", (long long)b, R[b].gradnorm,
                  indefinite[b] ? " after meeting non-positive curvature: the stored tensor's form is indefinite at "
                                  "the iterate (its rounding breaks the sum of m-th powers; see the storage dtype)"
                                : "");
  return TK_OK;
}
