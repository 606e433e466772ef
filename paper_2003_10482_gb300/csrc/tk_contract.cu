// Host side of the packed contraction: launch configuration of the streaming
// kernel (tk_contract_impl.cuh) and the fixed-order FP64 reduction of the
// per-block partial sums.
#include "tk_contract_impl.cuh"

namespace tk {

int contract_launch_f64(const KParams &, bool, int, int, int, size_t, cudaStream_t);
int contract_launch_f32(const KParams &, bool, int, int, int, size_t, cudaStream_t);
int contract_launch_bf16(const KParams &, bool, int, int, int, size_t, cudaStream_t);

// ------------------------------------------------------------------ finalize
template <int BS>
__device__ double block_sum(double x, double *sh) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < BS / 32; ++i) t += sh[i];
    sh[32] = t;
  }
  __syncthreads();
  return sh[32];
}

__global__ void __launch_bounds__(256) finalize_kernel(FinalizeArgs f) {
  __shared__ double sh[33];
  const int n = f.n, ld = n + 2;
  const int vec = (f.mode == 1) ? 1 : 0;
  const double lam = (f.mode == 2) ? f.lambda[0] : 0.0;
  double ssq = 0.0, aa = 0.0, ya = 0.0;
  for (int l = threadIdx.x; l < n; l += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < f.grid; ++b) s += f.part[(size_t)b * 2 * ld + vec * ld + l];
    if (f.mode == 2) {
      const double a = f.alpha[l], gr = s + lam * a - f.y[l];
      if (f.grad) f.grad[l] = gr;
      ssq += gr * gr;
      aa += a * a;
      ya += f.y[l] * a;
    } else {
      if (f.mode == 1) s /= (double)(f.m - 1);
      if (f.out_dtype == TK_F64) reinterpret_cast<double *>(f.G)[l] = s;
      else reinterpret_cast<float *>(f.G)[l] = (float)s;
    }
  }
  double S = 0.0;
  if (threadIdx.x == 0)
    for (int b = 0; b < f.grid; ++b) S += f.part[(size_t)b * 2 * ld + n];
  if (f.mode == 0) {
    if (threadIdx.x == 0 && f.S) f.S[0] = S;
    return;
  }
  if (f.mode == 1) return;
  const double tssq = block_sum<256>(ssq, sh);
  const double taa = block_sum<256>(aa, sh);
  const double tya = block_sum<256>(ya, sh);
  if (threadIdx.x == 0) {
    if (f.S) f.S[0] = S;
    if (f.F) f.F[0] = S / f.m + 0.5 * lam * taa - tya;
    if (f.gnorm) f.gnorm[0] = sqrt(tssq);
  }
}

// ------------------------------------------------------------------ host
static int pick_nc(int n) {
  const int need = (n + 31) / 32;
  const int opts[] = {1, 2, 4, 8, 12, 16, 20, 24, 32};
  for (int o : opts)
    if (o >= need) return o;
  return -1;
}

static int max_threads_for(int storage, bool dual, int nc) {
  return max_threads_est(storage == TK_F64 ? 8 : 4, dual, nc);
}

size_t contract_part_bytes(int n, int grid) { return (size_t)grid * 2 * (size_t)(n + 2) * sizeof(double); }

int contract_default_grid() {
  DevInfo di;
  if (dev_info(&di) != TK_OK) return -1;
  return di.sms;
}

int contract_pass(const ContractArgs &a, int *grid_out, cudaStream_t st) {
  DevInfo di;
  int rc = dev_info(&di);
  if (rc != TK_OK) return rc;
  const bool dual = a.v != nullptr;
  const int es = dtype_size(a.storage);
  const int cts = a.storage == TK_F64 ? 8 : 4;
  const int nc = pick_nc(a.n);
  if (nc < 0) return fail(TK_EUNSUPPORTED, "contract: n=%d exceeds %d", a.n, TK_MAX_POINTS);

  KParams kp;
  kp.m = a.m;
  kp.n = a.n;
  kp.K = reinterpret_cast<const unsigned char *>(a.K);
  kp.off_lo = a.off_lo;
  kp.off_hi = a.off_hi;
  kp.bytes = (a.off_hi - a.off_lo) * es;
  kp.alpha = a.alpha;
  kp.v = a.v;
  kp.vec_dtype = a.vec_dtype;
  kp.part = a.part;
  kp.status = a.status;

  // ring: a batch of kRB rows (<= kRB * n entries) must fit in NS-1 slots
  kp.slot_log2 = a.slot_log2 > 0 ? a.slot_log2 : 11;
  const int64_t slot = 1ll << kp.slot_log2;
  const int64_t batch_bytes = (int64_t)kRB * a.n * es + 32;
  int need = (int)((batch_bytes + slot - 1) / slot) + 2;
  int ns_log2 = 2;
  while ((1 << ns_log2) < need) ++ns_log2;
  if (a.ns_log2 > 0) {
    if (a.ns_log2 < ns_log2) return fail(TK_EINVAL, "contract: ring of 2^%d slots too small", a.ns_log2);
    ns_log2 = a.ns_log2;
  }
  if (ns_log2 > 4) return fail(TK_EUNSUPPORTED, "contract: ring needs more than 16 slots");
  kp.ns_log2 = ns_log2;
  const int64_t ring = slot << ns_log2;
  kp.vec_bytes = (int)(((int64_t)(dual ? 2 : 1) * a.n * cts + 127) & ~127ll);
  kp.warp_bytes = (int)((128 + ring + (int64_t)(dual ? 2 : 1) * a.n * cts + 127) & ~127ll);
  const int smem_budget = di.smem_optin - 1024;  // static shared + slack
  int warps_fit = (smem_budget - kp.vec_bytes) / kp.warp_bytes;
  int warps = a.warps > 0 ? a.warps : 16;
  warps = std::min(warps, max_threads_for(a.storage, dual, nc) / 32);
  warps = std::min(warps, warps_fit);
  if (warps < 1) return fail(TK_EUNSUPPORTED, "contract: shared memory too small for one warp");
  kp.warps = warps;
  const int cps = a.ctas_per_sm > 0 ? a.ctas_per_sm : 1;
  const int grid = di.sms * cps;
  const size_t smem = (size_t)kp.vec_bytes + (size_t)warps * kp.warp_bytes;
  if (grid_out) *grid_out = grid;

  if (a.storage == TK_F64) return contract_launch_f64(kp, dual, nc, grid, warps * 32, smem, st);
  if (a.storage == TK_F32) return contract_launch_f32(kp, dual, nc, grid, warps * 32, smem, st);
  return contract_launch_bf16(kp, dual, nc, grid, warps * 32, smem, st);
}

int contract_finalize(const FinalizeArgs &f, cudaStream_t st) {
  finalize_kernel<<<1, 256, 0, st>>>(f);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

}  // namespace tk
