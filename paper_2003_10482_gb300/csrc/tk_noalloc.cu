// Contraction entry point that allocates nothing.
//
// Some callers cannot call cudaMalloc or any other allocator: code running
// while a CUDA graph is being captured (allocation is not a capturable
// operation), runtimes whose device memory is fully pre-reserved, or
// embedding environments that hand the library only the tensors they own.
// tk_contract_noalloc serves them: the caller still passes K, the dual vector
// and the outputs, and the contraction's scratch (status header, per-warp
// work plan and per-block partial sums) lives in one file-scope device array
// of fixed size that every GPU loading the library holds until the process
// exits.  The thesis has no counterpart; it is an interface convenience.
#include <string.h>

#include <mutex>

#include "tk_internal.h"

namespace tk {

// 8 MiB covers the largest supported launch (n <= 1024, one block per SM,
// up to 16 pieces per warp on up to 160 SMs).
constexpr size_t kNoAllocScratchBytes = size_t(8) << 20;
constexpr int kNoAllocPlanCap = 16 * 160 * 16;
constexpr int kNoAllocMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Host-side state per device: the device address of the array (the host
// symbol g_noalloc_scratch is only a stand-in, never a device address) and
// which work plan the array's plan region holds.
static void *g_scratch_dev[kNoAllocMaxDevices];
static StaticPlanState g_plan_state[kNoAllocMaxDevices];
static WarpPlan g_host_plan[kNoAllocPlanCap];
static std::mutex g_noalloc_mu;

// The device address of the array on the current device; the first call on
// a device looks it up and zeroes the header (status word, plan key).  With
// `capturing` set, a device whose array is not set up yet is refused before
// anything is issued (the zeroing is a synchronous memset).
static int scratch_for_current_device(bool capturing, void **out, int *dev_out) {
  int dev = 0;
  TK_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(TK_EUNSUPPORTED, "device %d beyond %d", dev, kNoAllocMaxDevices);
  if (!g_scratch_dev[dev]) {
    if (capturing)
      return fail(TK_EINVAL, "tk_contract_noalloc: the first call on a device must come before any stream capture");
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    TK_CUDA_CHECK(cudaMemset(p, 0, sizeof(WsHeader)));
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  *dev_out = dev;
  return TK_OK;
}

}  // namespace tk

using namespace tk;

extern "C" int tk_contract_noalloc(int m, int64_t n, int storage, const void *K, int vec_dtype, const void *alpha,
                                   void *G, double *S, void *stream) {
  if (m < 2 || m > TK_MAX_ORDER) return fail(TK_EINVAL, "order m=%d outside [2, %d]", m, TK_MAX_ORDER);
  if (n < 1 || n > TK_MAX_POINTS) return fail(TK_EINVAL, "n=%lld outside [1, %d]", (long long)n, TK_MAX_POINTS);
  if (storage < TK_F64 || storage > TK_BF16) return fail(TK_EINVAL, "bad storage dtype %d", storage);
  if (vec_dtype != TK_F64 && vec_dtype != TK_F32) return fail(TK_EINVAL, "bad vector dtype %d", vec_dtype);
  if (!K || !alpha || !G) return fail(TK_EINVAL, "NULL K, alpha or G");
  if (((uintptr_t)K & 15u) != 0) return fail(TK_EINVAL, "K must be 16-byte aligned");
  const int64_t N = tk_packed_size(m, n);
  if (N < 0) return fail(TK_EOVERFLOW, "C(n+m-1, m) overflows");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TK_CUDA_CHECK(cudaStreamIsCapturing(st, &cs));
  const bool capturing = cs != cudaStreamCaptureStatusNone;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  void *scratch = nullptr;
  int dev = 0;
  int rc = scratch_for_current_device(capturing, &scratch, &dev);
  if (rc != TK_OK) return rc;
  ContractArgs a;
  memset(&a, 0, sizeof(a));
  a.m = m;
  a.n = (int)n;
  a.storage = storage;
  a.K = K;
  a.off_lo = 0;
  a.off_hi = N;
  a.vec_dtype = vec_dtype;
  a.alpha = alpha;
  a.v = nullptr;
  a.work = scratch;
  a.status = reinterpret_cast<int *>(scratch);
  a.fin.mode = 0;
  a.fin.out_dtype = vec_dtype;
  a.fin.G = G;
  a.fin.S = S;
  int grid = 0;
  const double *part = nullptr;
  return contract_pass_static(a, g_host_plan, kNoAllocPlanCap, &g_plan_state[dev], kNoAllocScratchBytes, capturing,
                              &grid, &part, st);
}

extern "C" int tk_contract_noalloc_status(void *stream) {
  int dev = 0;
  TK_CUDA_CHECK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(TK_EUNSUPPORTED, "device %d beyond %d", dev, kNoAllocMaxDevices);
  void *p = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    p = g_scratch_dev[dev];
  }
  if (!p) return TK_OK;  // no call has run on this device
  return tk_status_read(p, stream);
}
