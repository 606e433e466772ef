// Diagnostic entry point of the tensor-core building blocks (tk_umma.cuh): one
// 128 x N tile D = A B^T computed by tcgen05.mma (kind::tf32, FP32
// accumulation in tensor memory) from operands staged in the K-major
// 128-byte-swizzled layout, optionally with the 3-term TF32 split
// (hi*hi' + hi*lo' + lo*hi').  Compared with a host product by the tests, it
// pins the descriptor encodings, the swizzle, the tensor-memory read-out and
// the split that the tensor-core kernels rely on.
#include "tk_umma.cuh"

namespace tk {

constexpr int kProbeM = 128;

__global__ void __launch_bounds__(128) k_umma_probe(const float *A, const float *B, float *D, int N, int K,
                                                    int split, int *status) {
  extern __shared__ unsigned char probe_smem[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tbase;
  unsigned char *sm = reinterpret_cast<unsigned char *>((reinterpret_cast<uintptr_t>(probe_smem) + 1023) &
                                                        ~uintptr_t(1023));
  const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
  const int kc = K / 32;
  const uint32_t a_bytes = kProbeM * 128, b_bytes = (uint32_t)N * 128;
  unsigned char *a_hi = sm, *a_lo = sm + kc * a_bytes;
  unsigned char *b_hi = sm + 2 * kc * a_bytes, *b_lo = b_hi + kc * b_bytes;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)N) ncols <<= 1;

  // operands into the swizzled layout (chunk c holds k in [32c, 32c + 32))
  for (int i = tid; i < kProbeM * K; i += blockDim.x) {
    const int r = i / K, k = i % K;
    float h = A[i], l = 0.f;
    if (split) umma::split_tf32(A[i], h, l);
    const uint32_t off = (k / 32) * a_bytes + umma::sw128_offset(r, k % 32);
    *reinterpret_cast<float *>(a_hi + off) = h;
    *reinterpret_cast<float *>(a_lo + off) = l;
  }
  for (int i = tid; i < N * K; i += blockDim.x) {
    const int r = i / K, k = i % K;
    float h = B[i], l = 0.f;
    if (split) umma::split_tf32(B[i], h, l);
    const uint32_t off = (k / 32) * b_bytes + umma::sw128_offset(r, k % 32);
    *reinterpret_cast<float *>(b_hi + off) = h;
    *reinterpret_cast<float *>(b_lo + off) = l;
  }
  if (w == 0) {
    umma::tmem_alloc(&tbase, ncols);
    umma::tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar, 1);
    fence_barrier_init();
  }
  fence_proxy_async();  // the operands written above become visible to the tensor cores
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tbase;
  if (tid == 0) {
    const uint32_t id = umma::idesc_tf32(kProbeM, N);
    for (int c = 0; c < kc; ++c) {
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t ko = 32u * ks;
        const uint64_t ah = umma::desc_sw128(saddr(a_hi + c * a_bytes) + ko);
        const uint64_t bh = umma::desc_sw128(saddr(b_hi + c * b_bytes) + ko);
        umma::mma_tf32(tmem, ah, bh, id, (c | ks) != 0);
        if (split) {
          const uint64_t al = umma::desc_sw128(saddr(a_lo + c * a_bytes) + ko);
          const uint64_t bl = umma::desc_sw128(saddr(b_lo + c * b_bytes) + ko);
          umma::mma_tf32(tmem, ah, bl, id, 1);
          umma::mma_tf32(tmem, al, bh, id, 1);
        }
      }
    }
    umma::mma_commit(&bar);
  }
  __syncwarp();
  const bool ok = mbar_wait_bounded(&bar, 0);
  umma::fence_after_sync();
  const int row = 32 * w + lane;
  for (int c0 = 0; c0 < N; c0 += 16) {
    float v[16];
    umma::tmem_ld16(tmem + ((uint32_t)(32 * w) << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int j = 0; j < 16; ++j) D[(size_t)row * N + c0 + j] = v[j];
  }
  umma::fence_before_sync();
  __syncthreads();
  if (w == 0) umma::tmem_dealloc(tmem, ncols);
  if (!__syncthreads_and(ok ? 1 : 0) && tid == 0) {
    atomicExch(&reinterpret_cast<WsHeader *>(status)->status, TK_ETIMEOUT);
    reinterpret_cast<WsHeader *>(status)->where = kSiteUmmaWait;
  }
}

}  // namespace tk

using namespace tk;

extern "C" int tk_umma_probe(int n_cols, int k, int split, const float *A, const float *B, float *D, void *work,
                             size_t work_bytes, void *stream) {
  if (n_cols < 16 || n_cols > 256 || n_cols % 16 != 0)
    return fail(TK_EINVAL, "n_cols=%d: must be a multiple of 16 in [16, 256]", n_cols);
  if (k != 32 && k != 64) return fail(TK_EINVAL, "k=%d: must be 32 or 64", k);
  if (split != 0 && split != 1) return fail(TK_EINVAL, "split must be 0 or 1");
  if (!A || !B || !D || !work) return fail(TK_EINVAL, "NULL pointer");
  if (work_bytes < sizeof(WsHeader)) return fail(TK_ENOMEM, "work must hold the %zu-byte header", sizeof(WsHeader));
  int dev = 0, major = 0;
  TK_CUDA_CHECK(cudaGetDevice(&dev));
  TK_CUDA_CHECK(cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev));
  if (major != 10) return fail(TK_EUNSUPPORTED, "tcgen05 needs a compute capability 10.x device (got %d.x)", major);
  const size_t smem = 1024 + 2 * (size_t)(k / 32) * (kProbeM * 128 + (size_t)n_cols * 128);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  TK_CUDA_CHECK(cudaFuncSetAttribute(k_umma_probe, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_umma_probe<<<1, 128, smem, st>>>(A, B, D, n_cols, k, split, reinterpret_cast<int *>(work));
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}
