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

}  // namespace tk

using namespace tk;

extern "C" int tk_check_bounded_wait(void *work, size_t work_bytes, long long budget_cycles, void *stream) {
  if (!work || work_bytes < sizeof(WsHeader)) return fail(TK_EINVAL, "workspace smaller than its 256-byte header");
  if (budget_cycles < 1 || budget_cycles > (1ll << 31)) return fail(TK_EINVAL, "budget outside [1, 2^31] cycles");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  k_wait_nothing_arrives<<<1, 32, 0, st>>>(reinterpret_cast<int *>(work), budget_cycles);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}
