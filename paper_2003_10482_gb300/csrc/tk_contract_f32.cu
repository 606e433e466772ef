// Instantiations of the packed contraction kernel for f32 storage.
#include "tk_contract_impl.cuh"

namespace tk {

int contract_launch_f32(const KParams &kp, bool dual, int nc, int grid, int threads, size_t smem,
                          cudaStream_t st) {
  return dual ? launch_typed<float, float, true>(kp, nc, grid, threads, smem, st)
              : launch_typed<float, float, false>(kp, nc, grid, threads, smem, st);
}

}  // namespace tk
