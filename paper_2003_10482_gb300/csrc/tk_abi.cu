// C ABI entry points of libtk: argument checks, workspace layout, launches.
#include <stdarg.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "tk_internal.h"

namespace tk {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int cuda_fail(cudaError_t e, const char *what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return TK_ECUDA;
}

int dev_info(DevInfo *out) {
  static thread_local int cached_dev = -1;
  static thread_local DevInfo cached;
  int dev = 0;
  TK_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev != cached_dev) {
    TK_CUDA_CHECK(cudaDeviceGetAttribute(&cached.sms, cudaDevAttrMultiProcessorCount, dev));
    TK_CUDA_CHECK(cudaDeviceGetAttribute(&cached.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    cached_dev = dev;
  }
  *out = cached;
  return TK_OK;
}

// N = C(n+m-1, m) with an overflow guard: N * 16 must stay below 2^63 so that
// every partial product of the exact binomial evaluation fits.
static int64_t packed_size_checked(int m, int64_t n) {
  if (m < 1 || m > 16 || n < 0) return -1;
  if (n == 0) return 0;
  // evaluate in long double first to reject sizes whose binomial overflows
  long double c = 1.0L;
  for (int i = 0; i < m; ++i) c = c * (long double)(n + m - 1 - i) / (long double)(i + 1);
  if (c * 16.0L > 9.0e18L) return -1;
  return multiset(n, m);
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static int check_order_points(int m, int64_t n) {
  if (m < 2 || m > TK_MAX_ORDER) return fail(TK_EINVAL, "order m=%d outside [2, %d]", m, TK_MAX_ORDER);
  if (n < 1) return fail(TK_EINVAL, "n=%lld must be >= 1", (long long)n);
  if (n > TK_MAX_POINTS) return fail(TK_EUNSUPPORTED, "n=%lld exceeds %d", (long long)n, TK_MAX_POINTS);
  if (packed_size_checked(m, n) < 0) return fail(TK_EOVERFLOW, "C(n+m-1, m) overflows");
  return TK_OK;
}

static bool is_row_start(int m, int64_t n, int64_t off, int64_t N) {
  if (off == N) return true;
  int32_t t[16];
  unrank(m, n, off, t);
  return t[m - 1] == t[m - 2];
}

}  // namespace tk

using namespace tk;

extern "C" {

const char *tk_last_error(void) { return g_err; }

const char *tk_version(void) { return "tk 0.1 (sm_103a)"; }

int64_t tk_packed_size(int m, int64_t n) { return packed_size_checked(m, n); }

int64_t tk_packed_bytes(int m, int64_t n, int dtype) {
  if (dtype < TK_F64 || dtype > TK_BF16) return -1;
  int64_t N = packed_size_checked(m, n);
  if (N < 0) return -1;
  return N * dtype_size(dtype);
}

int tk_rank(int m, int64_t n, const int32_t *idx, int64_t *off) {
  if (!idx || !off) return fail(TK_EINVAL, "tk_rank: NULL pointer");
  if (packed_size_checked(m, n) < 0 || n < 1) return fail(TK_EINVAL, "tk_rank: bad m=%d / n", m);
  for (int j = 0; j < m; ++j) {
    if (idx[j] < 0 || idx[j] >= n || (j > 0 && idx[j] < idx[j - 1]))
      return fail(TK_EINVAL, "tk_rank: tuple is not sorted within [0, n)");
  }
  *off = rank(m, n, idx);
  return TK_OK;
}

int tk_unrank(int m, int64_t n, int64_t off, int32_t *idx) {
  if (!idx) return fail(TK_EINVAL, "tk_unrank: NULL pointer");
  int64_t N = packed_size_checked(m, n);
  if (N < 0 || n < 1) return fail(TK_EINVAL, "tk_unrank: bad m=%d / n", m);
  if (off < 0 || off >= N) return fail(TK_EINVAL, "tk_unrank: offset outside [0, N)");
  unrank(m, n, off, idx);
  return TK_OK;
}

int tk_row_align(int m, int64_t n, int64_t off, int64_t *row_off) {
  if (!row_off) return fail(TK_EINVAL, "tk_row_align: NULL pointer");
  int64_t N = packed_size_checked(m, n);
  if (N < 0 || n < 1 || m < 2) return fail(TK_EINVAL, "tk_row_align: bad m=%d / n", m);
  if (off < 0 || off > N) return fail(TK_EINVAL, "tk_row_align: offset outside [0, N]");
  if (off == N) {
    *row_off = N;
    return TK_OK;
  }
  int32_t t[16];
  unrank(m, n, off, t);
  *row_off = (t[m - 1] == t[m - 2]) ? off : off + (n - t[m - 1]);
  return TK_OK;
}

size_t tk_contract_workspace_size(int m, int64_t n, int64_t B) {
  if (check_order_points(m, n) != TK_OK) return 0;
  DevInfo di;
  if (dev_info(&di) != TK_OK) return 0;
  size_t need = contract_workspace_bytes((int)n, di.sms);
  if (B > 1) need = std::max(need, batched_workspace_bytes((int)n, B, di.sms));
  // room for the tensor-core pass wherever the configuration may take it
  if (tc_covers(m, (int)n, TK_F32, false, B, 0, multiset(n, m))) need = std::max(need, tc_workspace_bytes(m, (int)n, B, di.sms));
  return need;
}

static int contract_impl(int m, int64_t n, int storage, const void *K, int64_t off_lo, int64_t off_hi,
                         int64_t B, int vec_dtype, const void *A, int r, const void *V, void *G, double *S,
                         void *work, size_t work_bytes, void *stream) {
  int rc = check_order_points(m, n);
  if (rc != TK_OK) return rc;
  if (storage < TK_F64 || storage > TK_BF16) return fail(TK_EINVAL, "bad storage dtype %d", storage);
  if (vec_dtype != TK_F64 && vec_dtype != TK_F32) return fail(TK_EINVAL, "bad vector dtype %d", vec_dtype);
  if (r != m - 1 && r != m - 2) return fail(TK_EINVAL, "r=%d must be m-1 or m-2", r);
  if (r == m - 2 && !V) return fail(TK_EINVAL, "r = m-2 needs the direction V");
  if (B < 0) return fail(TK_EINVAL, "B < 0");
  if (B == 0) return TK_OK;
  if (!A || !G || !work) return fail(TK_EINVAL, "NULL A, G or workspace");
  const int64_t N = multiset(n, m);
  if (off_lo < 0 || off_hi > N || off_lo > off_hi) return fail(TK_EINVAL, "range outside [0, N]");
  if (!is_row_start(m, n, off_lo, N) || !is_row_start(m, n, off_hi, N))
    return fail(TK_EINVAL, "range ends must be row starts (tk_row_align)");
  if (off_hi > off_lo && !K) return fail(TK_EINVAL, "NULL K");
  if (!aligned16(K) || !aligned16(work)) return fail(TK_EINVAL, "K and work must be 16-byte aligned");
  DevInfo di;
  rc = dev_info(&di);
  if (rc != TK_OK) return rc;
  const size_t need = contract_workspace_bytes((int)n, di.sms);
  if (work_bytes < need) return fail(TK_ENOMEM, "workspace %zu < %zu bytes", work_bytes, need);

  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int vs = vec_dtype == TK_F64 ? 8 : 4;
  unsigned char *wsb = reinterpret_cast<unsigned char *>(work);
  // One pass for the whole batch when the batched kernel covers the shape and
  // the batch is large enough to pay for it: its launch costs about as much
  // for one vector as for 64 (32 for the HVP), while the single-vector kernel
  // runs at the HBM rate (measured on GB300, m = 4, n = 300: the batched
  // kernel wins from B = 28 for K[a^{m-1}] and from B = 16 for the HVP).
  if (B >= batched_min_batch(r == m - 2) && storage != TK_F64) {
    BatchedArgs ba;
    memset(&ba, 0, sizeof(ba));
    ba.m = m;
    ba.n = (int)n;
    ba.storage = storage;
    ba.K = K;
    ba.off_lo = off_lo;
    ba.off_hi = off_hi;
    ba.B = B;
    ba.vec_dtype = vec_dtype;
    ba.A = A;
    ba.V = (r == m - 2) ? V : nullptr;
    ba.G = G;
    ba.S = (r == m - 1) ? S : nullptr;
    ba.work = work;
    ba.work_bytes = work_bytes;
    if (tc_covers(m, (int)n, storage, r == m - 2, B, off_lo, off_hi)) {
      rc = contract_batched_tc(ba, st);
      if (rc != TK_EUNSUPPORTED) return rc;
    }
    rc = contract_batched(ba, st);
    if (rc != TK_EUNSUPPORTED) return rc;
  }
  for (int64_t b = 0; b < B; ++b) {
    ContractArgs a;
    memset(&a, 0, sizeof(a));
    a.m = m;
    a.n = (int)n;
    a.storage = storage;
    a.K = K;
    a.off_lo = off_lo;
    a.off_hi = off_hi;
    a.vec_dtype = vec_dtype;
    a.alpha = reinterpret_cast<const unsigned char *>(A) + b * n * vs;
    a.v = (r == m - 2) ? reinterpret_cast<const unsigned char *>(V) + b * n * vs : nullptr;
    a.work = wsb;
    a.status = reinterpret_cast<int *>(wsb);
    a.fin.mode = (r == m - 1) ? 0 : 1;
    a.fin.out_dtype = vec_dtype;
    a.fin.G = reinterpret_cast<unsigned char *>(G) + b * n * vs;
    a.fin.S = (S && r == m - 1) ? S + b : nullptr;
    int grid = 0;
    const double *part = nullptr;
    rc = contract_pass(a, &grid, &part, st);
    if (rc != TK_OK) return rc;
  }
  return TK_OK;
}

int tk_contract(int m, int64_t n, int storage, const void *K, int64_t B, int vec_dtype, const void *A, int r,
                const void *V, void *G, double *S, void *work, size_t work_bytes, void *stream) {
  int64_t N = packed_size_checked(m, n);
  if (N < 0) return fail(TK_EOVERFLOW, "C(n+m-1, m) overflows");
  return contract_impl(m, n, storage, K, 0, N, B, vec_dtype, A, r, V, G, S, work, work_bytes, stream);
}

int tk_contract_range(int m, int64_t n, int storage, const void *K_range, int64_t off_lo, int64_t off_hi,
                      int64_t B, int vec_dtype, const void *A, int r, const void *V, void *G, double *S,
                      void *work, size_t work_bytes, void *stream) {
  return contract_impl(m, n, storage, K_range, off_lo, off_hi, B, vec_dtype, A, r, V, G, S, work, work_bytes,
                       stream);
}

int tk_contract_set_config(const tk_contract_config *cfg) {
  if (!cfg) {
    g_contract_cfg = tk_contract_config{0, 0, 0, 0, 0, 0, 0, 0};
    return TK_OK;
  }
  if (cfg->warps < 0 || cfg->warps > 16 || (cfg->block_bytes != 0 && (cfg->block_bytes < 1024 || cfg->block_bytes > 65536 || cfg->block_bytes % 128)) ||
      (cfg->nbuf != 0 && (cfg->nbuf < 2 || cfg->nbuf > 8)) || cfg->ctas_per_sm < 0 || cfg->ctas_per_sm > 2 ||
      cfg->row_cost < 0 || cfg->tri_cost < 0 || cfg->pieces_per_warp < 0 || cfg->pieces_per_warp > 16 || cfg->schedule < 0 || cfg->schedule > 2)
    return fail(TK_EINVAL, "contract config out of range");
  g_contract_cfg = *cfg;
  return TK_OK;
}

int tk_contract_plan(int m, int64_t n, int64_t off_lo, int64_t off_hi, int pieces, int row_cost, int tri_cost,
                     int64_t *bounds) {
  if (!bounds) return fail(TK_EINVAL, "NULL output");
  int rc = check_order_points(m, n);
  if (rc != TK_OK) return rc;
  if (pieces < 1 || row_cost < 0 || tri_cost < 0) return fail(TK_EINVAL, "bad pieces or costs");
  const int64_t N = multiset(n, m);
  if (off_lo < 0 || off_hi > N || off_lo > off_hi) return fail(TK_EINVAL, "range outside [0, N]");
  if (!is_row_start(m, n, off_lo, N) || !is_row_start(m, n, off_hi, N))
    return fail(TK_EINVAL, "range ends must be row starts (tk_row_align)");
  std::vector<WarpPlan> v(pieces);
  build_plan(m, (int)n, off_lo, off_hi, pieces, row_cost, tri_cost, v.data());
  for (int i = 0; i < pieces; ++i) bounds[i] = v[i].start;
  bounds[pieces] = v[pieces - 1].end;
  return TK_OK;
}

int tk_contract_get_config(int m, int64_t n, int storage, int dual, tk_contract_config *out) {
  if (!out) return fail(TK_EINVAL, "NULL output");
  int rc = check_order_points(m, n);
  if (rc != TK_OK) return rc;
  if (storage < TK_F64 || storage > TK_BF16) return fail(TK_EINVAL, "bad storage dtype %d", storage);
  int grid = 0;
  return contract_resolve(m, (int)n, storage, dual != 0, out, &grid);
}

int tk_batched_set_config(const tk_batched_config *cfg) {
  if (!cfg) {
    g_batched_cfg = tk_batched_config{0, 0, 0, 0, 0, 0};
    return TK_OK;
  }
  if (cfg->vpl < 0 || cfg->vpl > 2 ||
      (cfg->block_bytes != 0 && (cfg->block_bytes < 4096 || cfg->block_bytes > 65536 || cfg->block_bytes % 128)) ||
      (cfg->nbuf != 0 && (cfg->nbuf < 2 || cfg->nbuf > 4)) || cfg->slice_mult < 0 || cfg->slice_mult > 2 ||
      cfg->min_batch < 0 || cfg->tensor_cores < -1 || cfg->tensor_cores > 1)
    return fail(TK_EINVAL, "batched config out of range");
  g_batched_cfg = *cfg;
  return TK_OK;
}

int tk_batched_get_config(int m, int64_t n, int storage, int dual, int64_t B, tk_batched_config *out) {
  if (!out) return fail(TK_EINVAL, "NULL output");
  int rc = check_order_points(m, n);
  if (rc != TK_OK) return rc;
  if (storage < TK_F64 || storage > TK_BF16) return fail(TK_EINVAL, "bad storage dtype %d", storage);
  if (B < 1) return fail(TK_EINVAL, "B < 1");
  DevInfo di;
  rc = dev_info(&di);
  if (rc != TK_OK) return rc;
  batched_resolve((int)n, storage, dual != 0, B, di.sms, di.smem_optin, out);
  out->tensor_cores = tc_covers(m, (int)n, storage, dual != 0, B, 0, multiset(n, m)) ? 1 : 0;
  return TK_OK;
}

int tk_status_read(void *work, void *stream) {
  if (!work) return fail(TK_EINVAL, "NULL workspace");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  WsHeader h;
  TK_CUDA_CHECK(cudaMemcpyAsync(&h, work, sizeof(h), cudaMemcpyDeviceToHost, st));
  TK_CUDA_CHECK(cudaStreamSynchronize(st));
  if (h.status != TK_OK) {
    int code = h.status;
    // clear the status word and its site only: the rest of the header records
    // which work plan the workspace holds
    TK_CUDA_CHECK(cudaMemsetAsync(work, 0, 2 * sizeof(int), st));
    TK_CUDA_CHECK(cudaStreamSynchronize(st));
    if (h.where == kSiteStalePlan)
      return fail(code, "a contraction found its workspace planned for another shape and did nothing "
                  "(a CUDA graph replayed after a later call with another shape re-planned it)");
    return fail(code, "device status %d (site %d)", code, h.where);
  }
  return TK_OK;
}

int tk_workspace_release(void *work) {
  if (!work) return fail(TK_EINVAL, "NULL workspace");
  forget_plan(work);
  forget_hessian_plan(work);
  forget_tc_plan(work);
  return TK_OK;
}

int tk_objective(int m, int64_t n, int storage, const void *K, int64_t B, const double *A, const double *y,
                 const double *lambda, double *F, double *grad, double *gnorm, void *work, size_t work_bytes,
                 void *stream) {
  int rc = check_order_points(m, n);
  if (rc != TK_OK) return rc;
  if (storage < TK_F64 || storage > TK_BF16) return fail(TK_EINVAL, "bad storage dtype %d", storage);
  if (B < 0) return fail(TK_EINVAL, "B < 0");
  if (B == 0) return TK_OK;
  if (!K || !A || !y || !lambda || !work) return fail(TK_EINVAL, "NULL pointer");
  if (!aligned16(K) || !aligned16(work)) return fail(TK_EINVAL, "K and work must be 16-byte aligned");
  DevInfo di;
  rc = dev_info(&di);
  if (rc != TK_OK) return rc;
  const size_t need = contract_workspace_bytes((int)n, di.sms);
  if (work_bytes < need) return fail(TK_ENOMEM, "workspace %zu < %zu bytes", work_bytes, need);
  const int64_t N = multiset(n, m);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned char *wsb = reinterpret_cast<unsigned char *>(work);
  for (int64_t b = 0; b < B; ++b) {
    ContractArgs a;
    memset(&a, 0, sizeof(a));
    a.m = m;
    a.n = (int)n;
    a.storage = storage;
    a.K = K;
    a.off_lo = 0;
    a.off_hi = N;
    a.vec_dtype = TK_F64;
    a.alpha = A + b * n;
    a.work = wsb;
    a.status = reinterpret_cast<int *>(wsb);
    a.fin.mode = 2;
    a.fin.alpha = A + b * n;
    a.fin.y = y;
    a.fin.lambda = lambda + b;
    a.fin.F = F ? F + b : nullptr;
    a.fin.grad = grad ? grad + b * n : nullptr;
    a.fin.gnorm = gnorm ? gnorm + b : nullptr;
    int grid = 0;
    const double *part = nullptr;
    rc = contract_pass(a, &grid, &part, st);
    if (rc != TK_OK) return rc;
  }
  return TK_OK;
}

size_t tk_objective_host_workspace_size(int m, int64_t n) {
  const size_t cws = tk_contract_workspace_size(m, n, 1);
  if (cws == 0) return 0;
  return ((cws + 255) & ~size_t(255)) + 2 * (((size_t)(n + 2) * sizeof(double) + 255) & ~size_t(255));
}

int tk_objective_host(int m, int64_t n, int storage, const void *K, const double *A_host, const double *y,
                      const double *lambda, double *out_host, void *work, size_t work_bytes, void *stream) {
  if (!A_host || !out_host) return fail(TK_EINVAL, "NULL host buffer");
  const size_t need = tk_objective_host_workspace_size(m, n);
  if (need == 0) return TK_EINVAL;
  if (!work || work_bytes < need) return fail(TK_ENOMEM, "workspace %zu < %zu bytes", work_bytes, need);
  const size_t cws = (tk_contract_workspace_size(m, n, 1) + 255) & ~size_t(255);
  const size_t vec = ((size_t)(n + 2) * sizeof(double) + 255) & ~size_t(255);
  unsigned char *wsb = reinterpret_cast<unsigned char *>(work);
  double *a_dev = reinterpret_cast<double *>(wsb + cws);
  double *out_dev = reinterpret_cast<double *>(wsb + cws + vec);  // F, |grad|, grad[0..n-1]
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  TK_CUDA_CHECK(cudaMemcpyAsync(a_dev, A_host, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, st));
  int rc = tk_objective(m, n, storage, K, 1, a_dev, y, lambda, out_dev, out_dev + 2, out_dev + 1, work, cws, stream);
  if (rc != TK_OK) return rc;
  TK_CUDA_CHECK(cudaMemcpyAsync(out_host, out_dev, (size_t)(n + 2) * sizeof(double), cudaMemcpyDeviceToHost, st));
  TK_CUDA_CHECK(cudaStreamSynchronize(st));
  return TK_OK;
}

}  // extern "C"
