// Instantiations of the packed contraction kernel for bf16 storage.
#include "tk_contract_impl.cuh"

namespace tk {

int contract_launch_bf16(const KParams &kp, bool dual, int nc, int grid, int threads, size_t smem,
                          cudaStream_t st) {
  return dual ? launch_typed<__nv_bfloat16, float, true>(kp, nc, grid, threads, smem, st)
              : launch_typed<__nv_bfloat16, float, false>(kp, nc, grid, threads, smem, st);
}

}  // namespace tk
