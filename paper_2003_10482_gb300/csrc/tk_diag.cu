// Diagnostic entry point: exercises the bounded device-side wait that every
// kernel of the library uses on its mbarriers, on a barrier that nothing
// arrives on, so that the timeout path (status word TK_ETIMEOUT, the context
// left usable) can be tested without faulting or hanging the GPU.
#include "tk_contract_impl.cuh"

namespace tk {

__global__ void k_wait_nothing_arrives(int *status, long long budget_cycles) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  __syncthreads();
  // phase 0 of a fresh barrier completes only after one arrival; none comes
  bool ok = mbar_try_wait(&bar, 0);
  const long long t0 = clock64();
  while (!ok && clock64() - t0 < budget_cycles) ok = mbar_try_wait(&bar, 0);
  const bool all_ok = __syncthreads_and(ok ? 1 : 0);
  if (threadIdx.x == 0) {
    if (!all_ok) {
      atomicExch(&reinterpret_cast<WsHeader *>(status)->status, TK_ETIMEOUT);
      reinterpret_cast<WsHeader *>(status)->where = kSiteDiagWait;
    }
    mbar_arrive(&bar);  // complete the phase: the barrier is not left pending
  }
}

// Peak-rate probe: every thread runs `iters` rounds of 16 independent
// multiply-add chains (enough independent work to keep the FMA pipes full),
// 2 * 16 * iters flops per thread.  The chains stay finite (the multiplier is
// just below one); one value per block is written so the work is not removed.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(long long iters, T *out) {
  T a[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) a[i] = T(threadIdx.x + i) * T(1e-3);
  const T mul = T(0.999999), add = T(1e-7);
  for (long long it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 16; ++i) a[i] = a[i] * mul + add;
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < 16; ++i) s += a[i];
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

}  // namespace tk

using namespace tk;

extern "C" int tk_fma_probe(int dtype, int blocks, long long iters, void *out, void *stream) {
  if (blocks < 1 || iters < 1 || !out) return fail(TK_EINVAL, "bad probe arguments");
  if (dtype != TK_F32 && dtype != TK_F64) return fail(TK_EINVAL, "probe dtype must be TK_F32 or TK_F64");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (dtype == TK_F32) k_fma_probe<float><<<blocks, 256, 0, st>>>(iters, reinterpret_cast<float *>(out));
  else k_fma_probe<double><<<blocks, 256, 0, st>>>(iters, reinterpret_cast<double *>(out));
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}

extern "C" int tk_check_bounded_wait(void *work, size_t work_bytes, long long budget_cycles, void *stream) {
  if (!work || work_bytes < sizeof(WsHeader)) return fail(TK_EINVAL, "workspace smaller than its 256-byte header");
  if (budget_cycles < 1 || budget_cycles > (1ll << 31)) return fail(TK_EINVAL, "budget outside [1, 2^31] cycles");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_wait_nothing_arrives<<<1, 32, 0, st>>>(reinterpret_cast<int *>(work), budget_cycles);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}
