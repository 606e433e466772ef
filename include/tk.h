/*
 * tk.h -- C ABI of libtk, the GB300 (sm_103a) implementation of the packed
 * tensor-kernel method for l^p-regularised regression of
 * F. Hibraj, "Efficient Tensor Kernel methods for sparse regression".
 *
 * Notation.  m is the (even) tensor order, the thesis's q; p = m/(m-1).
 * n is the number of points the tensor is built over (all training points,
 * or the n' Nystrom landmarks of Section 6).  d is the feature dimension.
 * lambda = 1/gamma is the regularisation weight of the dual (Section 4,
 * eq. dual_tensor_kernel written with 1/(2 gamma) = lambda/2).
 *
 * Packed layout (Section 5).  The order-m symmetric tensor K is stored as the
 * N = C(n+m-1, m) entries whose indices are sorted, i_1 <= i_2 <= ... <= i_m,
 * in the order of the thesis's nested loops: lexicographic, i_1 slowest and
 * i_m fastest.  Offset 0 is (0,...,0); offset N-1 is (n-1,...,n-1).  A "row"
 * is the run of entries sharing i_1..i_{m-1}; it holds n - i_{m-1} entries.
 * Entry types: TK_F64 (8 B), TK_F32 (4 B), TK_BF16 (2 B, round-to-nearest-even
 * from the FP32 accumulator).
 *
 * Conventions.
 *   - Every function returns TK_OK (0) or a TK_E* code; tk_last_error() gives
 *     a message for the calling thread's last failure.
 *   - The caller owns all memory.  Unless marked "host", pointers are device
 *     pointers.  The library allocates no device memory on any call path
 *     below except where stated; scratch space is sized by the matching
 *     *_workspace_size call and passed in as `work`.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Device calls are asynchronous on that stream unless noted.
 *   - Device buffers must be 16-byte aligned (every cudaMalloc / PyTorch
 *     allocation is).
 *   - No floating-point atomics; every reduction runs in a fixed order, and
 *     with the default schedule (tk_contract_config.schedule) results are
 *     bit-reproducible from run to run.
 */
#ifndef TK_H
#define TK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- codes */
enum {
    TK_OK = 0,
    TK_EINVAL = 1,       /* bad argument (sizes, dtype, order, pointer, alignment) */
    TK_EOVERFLOW = 2,    /* N or an offset does not fit the 64-bit index space */
    TK_ENOMEM = 3,       /* the workspace passed in is smaller than required */
    TK_ECUDA = 4,        /* a CUDA runtime call failed (message has the CUDA error) */
    TK_ENOTCONV = 5,     /* the solver stopped at max_iter before reaching tol */
    TK_ETIMEOUT = 6,     /* a bounded device-side wait ran out (see tk_status_read) */
    TK_EUNSUPPORTED = 7  /* valid input outside what this build implements */
};

enum { TK_F64 = 0, TK_F32 = 1, TK_BF16 = 2 };

/* Feature maps of the tensor kernels of Section 4:
 *   TK_FEAT_LINEAR  k = sum_j prod_l x'_{l,j}           (linear tensor kernel)
 *   TK_FEAT_POLY    k = (sum_j prod_l x'_{l,j})^degree   (polynomial tensor kernel,
 *                                                         eq. poly_tensor)
 *   TK_FEAT_EXP     k = exp(sum_j prod_l x'_{l,j})       (exponential tensor kernel) */
enum { TK_FEAT_LINEAR = 0, TK_FEAT_POLY = 1, TK_FEAT_EXP = 2 };

/* Dual solver methods (the thesis does not state its algorithm). */
enum { TK_NEWTON_CG = 0, TK_GD_BT = 1, TK_NEWTON_FULL = 2 };

/* Largest supported order and point count of the device contraction. */
#define TK_MAX_ORDER 8
#define TK_MAX_POINTS 1024

const char *tk_last_error(void);
const char *tk_version(void);

/* ------------------------------------------------------------ layout (host) */

/* N = C(n+m-1, m): the number of stored entries of the order-m symmetric
 * tensor over n points (Section 5: b_matrix, b_cube, b_tensor4 are m = 2,3,4).
 * Returns -1 if m < 1, n < 0, or N (or N*8) overflows int64. */
int64_t tk_packed_size(int m, int64_t n);

/* Bytes of N entries of `dtype`; -1 on error. */
int64_t tk_packed_bytes(int m, int64_t n, int dtype);

/* Offset of the sorted tuple idx_host[0..m-1] (host) in the packed order
 * (Section 5, eqs. index_2d, v3d, v4d and their extension to any m).  The
 * tuple must be non-decreasing with entries in [0, n): else TK_EINVAL. */
int tk_rank(int m, int64_t n, const int32_t *idx_host, int64_t *off_host);

/* Inverse of tk_rank: the sorted tuple stored at `off` (0 <= off < N). */
int tk_unrank(int m, int64_t n, int64_t off, int32_t *idx_host);

/* First row start at or after `off` (a row start is an offset whose tuple
 * has i_{m-1} == i_m); returns N when off > last row start.  Used to cut the
 * packed array into row-aligned shards. */
int tk_row_align(int m, int64_t n, int64_t off, int64_t *row_off_host);

/* ------------------------------------------------------------ build */

/* Packed build (Section 4 tensor kernel, stored as in Section 5):
 *   K[o] = k(x_{i_1}, ..., x_{i_m}) for the sorted tuple i at offset o.
 * X: n x d row-major FP64 (device).  K: N entries of storage_dtype (device,
 * caller-allocated with tk_packed_bytes bytes).  Accumulation is FP64 for
 * TK_F64 storage and FP32 otherwise; TK_BF16 rounds the FP32 result to
 * nearest-even.  `degree` is used by TK_FEAT_POLY only.  No workspace. */
int tk_build_packed(int m, int64_t n, int64_t d, const double *X, int feat,
                    int degree, int storage_dtype, void *K, void *stream);

/* Which kernel builds FP32 / BF16 storage: 0 (default) and -1 = the SIMT
 * build, 1 = the tensor-core build (tcgen05.mma kind::tf32 with the 3-term
 * split, a warp-specialised pipeline over 128 x 128 tiles of each triangle),
 * which is correct but measured slower on GB300.  FP64 storage always takes
 * the SIMT build.  Process-wide. */
int tk_build_set_config(int tensor_cores);

/* Status of the tensor-core builds issued so far on the current device:
 * TK_ETIMEOUT if one of their bounded waits ran out (its entries are then not
 * to be trusted), else TK_OK; reading clears it.  Synchronises `stream`. */
int tk_build_status(void *stream);

/* 1 if a build of d features into storage_dtype takes the tensor-core build
 * under the current configuration on the current device, else 0. */
int tk_build_path(int64_t d, int storage_dtype);

/* Same for the offsets [off_lo, off_hi) only: K_range[o - off_lo] = K[o].
 * Lets a shard of the packed array be built on its own device. */
int tk_build_packed_range(int m, int64_t n, int64_t d, const double *X, int feat,
                          int degree, int storage_dtype, int64_t off_lo,
                          int64_t off_hi, void *K_range, void *stream);

/* ------------------------------------------------------------ contraction */

/* Bytes of workspace tk_contract / tk_objective need for (m, n, B).  The
 * workspace carries a cached copy of the per-warp work plan between calls
 * (reused while m, n, the range and the launch configuration stay the same,
 * keyed by the workspace's address): callers must not write into it, and call
 * tk_workspace_release on memory that is new at an address a workspace held
 * before.  Its header records the plan's key, which every contraction checks
 * before it reads the plan (TK_EINVAL through tk_status_read on a mismatch). */
size_t tk_contract_workspace_size(int m, int64_t n, int64_t B);

/* Contractions of the symmetric tensor over its packed entries, each equal to
 * the full sum over all n^m index tuples of Section 4, eq. dual_tensor_kernel:
 *
 *   r = m-1:  G[b] = K[A_b^{m-1}]   (n-vector; K[a^{m-1}]_l = sum over i_2..i_m of
 *                                     K_{l,i_2..i_m} a_{i_2} ... a_{i_m})
 *             S[b] = K[A_b^m]       (optional, S may be NULL)
 *   r = m-2:  G[b] = K[A_b^{m-2}, V_b] (the Hessian-vector product of
 *             K[a^m]/(m(m-1)); V required)
 *
 * G excludes the factor m of the gradient m K[a^{m-1}]; callers scale.
 * A, V, G: B x n row-major, vec_dtype TK_F64 or TK_F32.  S: B FP64 values.
 * Arithmetic: FP64 for TK_F64 storage; FP32 for TK_F32 / TK_BF16 storage with
 * the cross-block reduction and S in FP64.  Each packed entry is read from
 * HBM once per pass.  For TK_F32 / TK_BF16 storage and B at least the
 * batched configuration's min_batch (by default 28, or 16 for r = m-2; see
 * tk_batched_config) one launch serves the whole batch (each entry read once
 * for all B vectors, 2B multiply-adds per entry; 4B for r = m-2); otherwise
 * the single-vector pass runs once per b.  Asynchronous; errors that only the
 * device can see (a bounded wait that ran out) are recorded in `work` and
 * returned by tk_status_read. */
int tk_contract(int m, int64_t n, int storage_dtype, const void *K, int64_t B,
                int vec_dtype, const void *A, int r, const void *V, void *G,
                double *S, void *work, size_t work_bytes, void *stream);

/* Same over the row-aligned offset range [off_lo, off_hi) (see tk_row_align);
 * K_range points at the entry of offset off_lo.  G and S receive the partial
 * sums over that range, so that shards on several devices add up to the full
 * contraction. */
int tk_contract_range(int m, int64_t n, int storage_dtype, const void *K_range,
                      int64_t off_lo, int64_t off_hi, int64_t B, int vec_dtype,
                      const void *A, int r, const void *V, void *G, double *S,
                      void *work, size_t work_bytes, void *stream);

/* Launch configuration of the streaming contraction kernel.  Zero fields keep
 * the library's choice.
 *   warps        warps per block (each warp walks its own row-aligned piece)
 *   block_bytes  bytes of one staging buffer (one bulk copy per row block), a
 *                multiple of 128 in [1024, 65536]; 0 = the largest that fits
 *                the shared memory with `warps` warps
 *   nbuf         staging buffers per warp (nbuf-1 copies in flight), 2..8
 *   ctas_per_sm  blocks per SM (1 or 2)
 *   row_cost     cost of one row, in entries, when the range is cut into pieces
 *   tri_cost     cost of entering a triangle (prefix i_1..i_{m-2}), in entries
 *   pieces_per_warp  the range is cut into this many pieces per warp (1..16)
 *   schedule     1: warp w takes pieces w, w+W, w+2W, ... (W warps; results are
 *                bit-reproducible); 2: warps take the next free piece from a
 *                shared counter as they finish (balances better; the order in
 *                which partial sums meet varies, so results vary in the last
 *                bits).  0 = library choice (1). */
typedef struct {
    int warps;
    int block_bytes;
    int nbuf;
    int ctas_per_sm;
    int row_cost;
    int tri_cost;
    int pieces_per_warp;
    int schedule;
} tk_contract_config;

/* Sets the process-wide contraction configuration (NULL restores the
 * defaults).  Used by the autotuner; not thread-safe against concurrent
 * contractions. */
int tk_contract_set_config(const tk_contract_config *cfg);

/* The configuration a contraction of (m, n, storage_dtype) would launch with
 * under the current settings (dual != 0: the HVP variant). */
int tk_contract_get_config(int m, int64_t n, int storage_dtype, int dual, tk_contract_config *out);

/* Launch configuration of the batched contraction (B vectors per pass).  Zero
 * fields keep the library's choice.
 *   vpl          vectors per lane (1 or 2): a block serves 32 * vpl vectors
 *   block_bytes  bytes of one staging buffer (a multiple of 128 in [4096, 65536])
 *   nbuf         staging buffers per block, 2..4
 *   slice_mult   blocks per group of vectors = slice_mult * SMs / groups (1 or 2)
 *   min_batch    smallest B that takes the batched kernel (below it the
 *                single-vector pass runs once per vector); 0 = 28 (16 for
 *                r = m-2); a value sets both
 *   tensor_cores the tensor-core pass for r = m-1 (tcgen05.mma, TF32 with a
 *                3-term split; the whole tensor, FP32 or BF16 storage,
 *                n <= 320): 0 = where it pays (m = 3 or 4, n >= 64, B >= 128),
 *                1 = wherever it covers the call, -1 = never.  In the result of
 *                tk_batched_get_config: 1 when the call would take it, else 0 */
typedef struct {
    int vpl;
    int block_bytes;
    int nbuf;
    int slice_mult;
    int min_batch;
    int tensor_cores;
} tk_batched_config;

/* Sets the process-wide batched configuration (NULL restores the defaults).
 * Used by the autotuner; not thread-safe against concurrent contractions. */
int tk_batched_set_config(const tk_batched_config *cfg);

/* The configuration a batched contraction of (m, n, storage_dtype, B) would
 * launch with under the current settings (dual != 0: r = m-2).  vpl = 0 in
 * the result means the batched kernel does not cover the shape. */
int tk_batched_get_config(int m, int64_t n, int storage_dtype, int dual, int64_t B, tk_batched_config *out);

/* Host-only: the row-aligned cut of [off_lo, off_hi) into `pieces` consecutive
 * pieces of near-equal cost (entries + row_cost per row + tri_cost per
 * triangle entered), as the contraction assigns them to warps.
 * bounds_host receives pieces+1 offsets (bounds[0] = off_lo, bounds[pieces] =
 * off_hi); every bound is a row start.  off_lo and off_hi must be row starts. */
int tk_contract_plan(int m, int64_t n, int64_t off_lo, int64_t off_hi, int pieces, int row_cost,
                     int tri_cost, int64_t *bounds_host);

/* K[a^{m-1}] and K[a^m] of one dual vector, like tk_contract with B = 1 and
 * r = m-1, for callers that cannot allocate device memory (code running under
 * CUDA graph capture, runtimes with pre-reserved memory, hosts that only lend
 * the library their own tensors).  The thesis has no counterpart.  The caller
 * passes K, alpha (n values of vec_dtype), G (n values of vec_dtype) and S
 * (one FP64 value, may be NULL), all device pointers; no workspace.
 *
 * Scratch lives in a static 8 MiB device array inside the library, held by
 * every GPU that loads it until the process exits; the contraction's needs
 * (status header, work plan, per-block partials) must fit in it, else
 * TK_ENOMEM with the size it would need.  No cudaMalloc, cudaFree or other
 * allocator is called.  The first call on a device looks the array up
 * (cudaGetSymbolAddress) and zeroes its header; a call whose shape (m, n)
 * or launch configuration (tk_contract_set_config) differs from the previous
 * call's re-plans: it uploads the work plan from host memory and waits for
 * the copy.  Make the first call, and the first call after every change of
 * shape or configuration, outside stream capture: under capture such a call
 * returns TK_EINVAL before it issues anything, so the capture stays valid.
 * Every call on a device shares the array and leaves the last call's contents
 * in it; calls whose executions overlap on the GPU (other streams, other host
 * threads' streams) race on it and must be serialised by the caller.  A
 * captured call replayed after a later call re-planned the array for another
 * shape finds the plan key in the array's header changed, writes nothing to G
 * or S and records TK_EINVAL, which tk_contract_noalloc_status returns. */
int tk_contract_noalloc(int m, int64_t n, int storage_dtype, const void *K, int vec_dtype, const void *alpha,
                        void *G, double *S, void *stream);

/* Reads and clears the status word of the tk_contract_noalloc scratch on the
 * current device: TK_OK, TK_ETIMEOUT (a bounded wait of an earlier call ran
 * out) or TK_EINVAL (a replayed call found the scratch planned for another
 * shape).  Synchronises `stream`.  TK_OK when no call ran on this device. */
int tk_contract_noalloc_status(void *stream);

/* Host only: forget which work plan the workspace at `work` holds.  A
 * workspace caches its plan between calls, keyed by its address; call this
 * before handing the library new memory at an address that held a workspace
 * earlier (a freed and reallocated buffer), or after writing into a
 * workspace, so that the next call uploads the plan again. */
int tk_workspace_release(void *work);

/* Reads (and clears) the device-side status word of a workspace: TK_OK,
 * TK_ETIMEOUT if a bounded wait of an earlier call on it ran out, or TK_EINVAL
 * if a contraction found the workspace's plan region planned for another
 * shape (a replayed CUDA graph) and did nothing.  Synchronises `stream`. */
int tk_status_read(void *work, void *stream);

/* Diagnostic: one block waits, with the library's bounded wait and a budget of
 * `budget_cycles` SM cycles (1 .. 2^31), on an mbarrier that nothing arrives
 * on, then records TK_ETIMEOUT in the status word of `work` (at least its
 * 256-byte header) as every kernel does when a wait runs out; tk_status_read
 * returns it.  The wait ends by itself and the context stays usable: the
 * timeout path can be tested without faulting or hanging the device. */
int tk_check_bounded_wait(void *work, size_t work_bytes, long long budget_cycles, void *stream);

/* Diagnostic: the FP32 or FP64 multiply-add rate of the device's vector
 * units.  Launches `blocks` blocks of 256 threads, each thread running 16
 * independent multiply-add chains for `iters` rounds: 2 * 16 * iters * 256 *
 * blocks floating-point operations, which the caller divides by the time it
 * measures (CUDA events on `stream`).  out: `blocks` values of dtype (device).
 * The rate is the denominator of the rooflines of the kernels bound by
 * vector arithmetic rather than memory (build, batched contraction). */
int tk_fma_probe(int dtype, int blocks, long long iters, void *out, void *stream);

/* Diagnostic of the tensor-core building blocks: one 128 x n_cols tile
 * D = A B^T by tcgen05.mma (kind::tf32, FP32 accumulation in tensor memory),
 * the operands staged in the K-major 128-byte-swizzled shared-memory layout
 * the tensor-core kernels use; split = 1 carries each operand as two TF32
 * parts (x = hi + lo) and sums hi*hi' + hi*lo' + lo*hi', which keeps about
 * 2^-21 relative accuracy per product.  A: 128 x k, B: n_cols x k, D: 128 x
 * n_cols, FP32 row-major (device); k = 32 or 64; n_cols a multiple of 16 in
 * [16, 256].  work: at least the 256-byte header (a timed-out wait on the
 * MMA's completion is reported by tk_status_read as TK_ETIMEOUT).  One block,
 * asynchronous on `stream`.  TK_EUNSUPPORTED on a device without tcgen05. */
int tk_umma_probe(int n_cols, int k, int split, const float *A, const float *B, float *D, void *work,
                  size_t work_bytes, void *stream);

/* ------------------------------------------------------------ dual objective */

/* Dual objective and gradient (Section 4, eqs. dual_tensor_kernel and jq, with
 * lambda = 1/gamma), in FP64 on the device:
 *   F[b]     = K[A_b^m]/m + (lambda_b/2) |A_b|^2 - <y, A_b>
 *   grad[b]  = K[A_b^{m-1}] + lambda_b A_b - y        (optional, B x n FP64)
 *   gnorm[b] = |grad[b]|_2                            (optional)
 * A: B x n FP64, y: n FP64, lambda: B FP64 (all device).  One contraction pass. */
int tk_objective(int m, int64_t n, int storage_dtype, const void *K, int64_t B,
                 const double *A, const double *y, const double *lambda, double *F,
                 double *grad, double *gnorm, void *work, size_t work_bytes,
                 void *stream);

/* Bytes of workspace tk_objective_host needs for (m, n): the contraction's
 * workspace plus device staging for the dual vector and the results. */
size_t tk_objective_host_workspace_size(int m, int64_t n);

/* tk_objective for one dual vector held in HOST memory, results back in HOST
 * memory, in one call: copies A_host (n FP64) to the device, runs the pass,
 * copies out_host[0] = F, out_host[1] = |grad F|_2, out_host[2..n+1] = grad F
 * (n + 2 FP64) back and synchronises `stream`.  y and lambda (1 value) are
 * device pointers.  Host buffers may be pageable; pinned ones let the copies
 * run at full speed.  Returns after out_host is written. */
int tk_objective_host(int m, int64_t n, int storage_dtype, const void *K, const double *A_host,
                      const double *y, const double *lambda, double *out_host, void *work,
                      size_t work_bytes, void *stream);

/* Dual objective and gradient from contractions that were already reduced
 * (for instance summed over the shards of several devices):
 *   F[b] = S[b]/m + (lambda_b/2)|A_b|^2 - <y, A_b>,  grad[b] = G[b] + lambda_b A_b - y,
 *   gnorm[b] = |grad[b]|_2   (Section 4, eqs. dual_tensor_kernel and jq).
 * G: B x n FP64 (K[A_b^{m-1}]), S: B FP64 (K[A_b^m]); everything FP64 on the
 * device.  grad and gnorm may be NULL.  No workspace. */
int tk_assemble_objective(int m, int64_t n, int64_t B, const double *G, const double *S, const double *A,
                          const double *y, const double *lambda, double *F, double *grad, double *gnorm,
                          void *stream);

/* Hessian-vector products of the dual objective (Section 4, second derivative
 * of eq. dual_tensor_kernel, lambda = 1/gamma), FP64 on the device:
 *   HV[b] = (m-1) K[A_b^{m-2}, V_b] + lambda_b V_b
 * A, V, HV: B x n FP64; lambda: B FP64 (all device).  One dual-number pass
 * over K (tk_contract with r = m-2) and an elementwise finish; the workspace
 * is tk_contract's for (m, n, B). */
int tk_dual_hvp(int m, int64_t n, int storage_dtype, const void *K, int64_t B, const double *A,
                const double *V, const double *lambda, double *HV, void *work, size_t work_bytes,
                void *stream);

/* The full Hessian of the tensor term (Section 4, second derivative of
 * eq. dual_tensor_kernel divided by m(m-1)):
 *   H[i][j] = K[a^{m-2}]_{ij} = sum over i_3..i_m of K_{i,j,i_3..i_m} a_{i_3}...a_{i_m},
 * a dense symmetric n x n FP64 matrix (row-major, device), from one pass over
 * the packed tensor (each entry read once).  a: n FP64 (device).  Arithmetic
 * as in tk_contract (FP32 with FP64 cross-block sums for FP32/BF16 storage);
 * the few entries whose rows and columns are both prefix values
 * (i, j <= the triangle's last prefix value) are summed with FP64 atomic
 * adds, so they may vary in the last bits from run to run.  n up to 768
 * (FP32/BF16 storage) or 384 (FP64 storage), else TK_EUNSUPPORTED.
 * Workspace: tk_hessian_workspace_size bytes, which carry a cached work plan
 * like the contraction's. */
size_t tk_hessian_workspace_size(int m, int64_t n);
int tk_hessian(int m, int64_t n, int storage_dtype, const void *K, const double *alpha, double *H, void *work,
               size_t work_bytes, void *stream);

/* ------------------------------------------------------------ primal side */

/* Representer map of Section 4 (eq. tensor_representer) for the linear tensor
 * kernel: w_b = J_q(X^T a_b) with q = m, i.e. w_k = sign(u_k)|u_k|^{m-1},
 * u = X^T a_b (= u_k^{m-1} for even m).  X: n x d row-major, A: B x n,
 * W: B x d; FP64 device pointers. */
int tk_primal(int m, int64_t n, int64_t d, const double *X, int64_t B, const double *A, double *W, void *stream);

/* Test-phase estimate of Section 4 (eq. tensor_1) with the linear kernel:
 * Yhat[b][j] = <w_b, x_j> for the t rows of Xtest (t x d row-major).
 * W: B x d, Yhat: B x t; FP64 device pointers. */
int tk_predict(int64_t t, int64_t d, const double *Xtest, int64_t B, const double *W, double *Yhat, void *stream);

/* Adaptive feature selection of Section 6.3: keep[b][j] = 1 when
 * |W[b][j]| > 2 std(W[b]) (population standard deviation over the d weights
 * of problem b), else 0; count[b] = number kept (count may be NULL).
 * W: B x d FP64, keep: B x d bytes, count: B int64 (device).  FP64 sums in a
 * fixed order, so the decision is reproducible. */
int tk_support_threshold(int64_t d, int64_t B, const double *W, uint8_t *keep, int64_t *count, void *stream);

/* Nystrom-like subsampling of Section 6.1: n_prime of the N training indices,
 * uniform without replacement, sorted ascending, written to idx_host (host).
 * Generator (so that any implementation reproduces the same indices):
 * SplitMix64 (Steele, Lea and Flood 2014) seeded with `seed`; for
 * j = N - n_prime .. N-1, draw x until x < (2^64 - 1) - ((2^64 - 1) mod (j + 1)),
 * r = x mod (j + 1), and take r unless it was taken already, else take j
 * (Floyd's algorithm, Bentley and Floyd 1987).  Host only. */
int tk_nystrom_select(int64_t N, int64_t n_prime, uint64_t seed, int64_t *idx_host);

/* ------------------------------------------------------------ dual solver */

/* One or several dual problems over the same packed tensor (Section 4,
 * eq. dual_tensor_kernel, lambda = 1/gamma):
 *   min_a  K[a^m]/m + (lambda_b/2)|a|^2 - <y, a>,   a_i = 0 where mask_b[i] = 0.
 * The objective is strongly convex (modulus lambda_b), so each problem has one
 * minimiser whatever the algorithm; the thesis does not name its algorithm. */
typedef struct {
    int m;
    int64_t n;
    int storage_dtype;
    const void *K;          /* N entries (device) */
    const double *y;        /* n targets (device) */
    int64_t B;              /* number of problems */
    const double *lambda;   /* B regularisation weights (device) */
    const uint8_t *mask;    /* B x n, 1 = point kept, 0 = held out (device); NULL = all kept */
    const void *K_hvp;      /* optional second copy of the same tensor (N entries of
                               hvp_storage_dtype, device) that the Hessian-vector passes of
                               Newton-CG and the Hessian passes of NEWTON_FULL read instead
                               of K; NULL = K.  The objective and gradient (which fix the
                               minimiser) always read K, so a lower-precision copy here
                               cheapens most passes while the solution stays that of K's
                               precision */
    int hvp_storage_dtype;
} tk_problem;

typedef struct {
    int method;             /* TK_NEWTON_CG (default), TK_GD_BT or TK_NEWTON_FULL */
    double tol_gradnorm;    /* stop a problem when |grad F|_2 <= tol */
    int max_iter;           /* outer iterations */
    int max_cg;             /* conjugate-gradient steps per Newton step */
    double armijo_c;        /* sufficient-decrease constant (0: 1e-4) */
    double tol_rel_gap;     /* Newton methods: also stop a problem when its Newton
                               decrement estimate -<grad F, p>/2 (p the Newton direction,
                               F(a) - F* to second order) is <= tol_rel_gap * max(1, |F|);
                               0 = off */
    int start_on_y;         /* 1: ignore A_inout's values and start each problem at the
                               minimiser of F along the ray s y_b (y_b = y on its kept
                               points): F(s y_b) = s^m K[y_b^m]/m + (lambda_b/2) s^2 |y_b|^2
                               - s |y_b|^2, one contraction pass for K[y_b^m], then the
                               positive root of its derivative; 0: start from A_inout */
} tk_solve_opts;

typedef struct {
    int iters;              /* outer iterations taken */
    int passes;             /* passes over the packed tensor (objective + HVP) */
    double gradnorm;        /* final |grad F|_2 */
    double F;               /* final objective */
    int status;             /* TK_OK, TK_ENOTCONV (max_iter or no further decrease possible) */
} tk_solve_report;

/* Bytes of workspace tk_solve_dual needs with TK_NEWTON_CG or TK_GD_BT. */
size_t tk_solve_workspace_size(const tk_problem *P);

/* Bytes of workspace tk_solve_dual needs with the method of O (TK_NEWTON_FULL
 * adds the Hessian pass's workspace and the Newton systems of up to 64
 * problems). */
size_t tk_solve_workspace_size_opts(const tk_problem *P, const tk_solve_opts *O);

/* Solves the B problems from the starting points in A_inout (B x n FP64,
 * device; masked entries are zeroed), in FP64 vector arithmetic on the device
 * (workspace: tk_solve_workspace_size_opts bytes):
 *   Newton-CG:  H p = -grad F by conjugate gradients with forcing term
 *               min(0.5, sqrt|grad F|), H v = (m-1) K[a^{m-2}, v] + lambda v,
 *               then backtracking (halving the step) until either Armijo's
 *               sufficient decrease holds or <grad F(a + t p), p> <= 0 (F is
 *               convex along the line, so the latter certifies F(a + t p) <=
 *               F(a) from gradients alone when F's rounding noise hides the
 *               decrease);
 *   NEWTON_FULL: p = -H^{-1} grad F with the full H = (m-1) K[a^{m-2}] +
 *               lambda I on the kept points and an FP64 Cholesky factorisation
 *               on the device.  Without K_hvp every evaluation of a point is
 *               one Hessian pass over K (tk_hessian), which by Euler's identity
 *               (K[a^{m-1}] = K[a^{m-2}] a, K[a^m] = a . K[a^{m-1}]) also gives F
 *               and grad F, so an accepted step costs one pass; with K_hvp the
 *               evaluations are contraction passes over K and each new point's
 *               Hessian is one pass over K_hvp.  The same backtracking.  H is
 *               positive definite for a tensor kernel of even order, so a
 *               problem whose H fails to factorise (a rounded tensor whose form
 *               has turned indefinite at the iterate, as FP32/BF16 storage does
 *               along null(X^T) when |a| grows like 1/lambda) stops there with
 *               TK_ENOTCONV;
 *   GD_BT:      steepest descent with Armijo backtracking, step initialised
 *               from the previous accepted step.
 * A line search takes at most 10 trials (the cubic interpolation shrinks the
 * step 2-10-fold per trial); a problem whose step shrank 10^8-fold, or that
 * used its 10 trials without an accepted point, stops unconverged.  So does a
 * problem whose computed F falls below -|y|^2/(2 lambda) (kept points): K[a^m]
 * >= 0 for an exact tensor of even order, so F cannot go lower, and a value
 * below it shows that the stored tensor's rounding made its form negative.
 * Every objective is one contraction pass and every H v one dual-number pass
 * (tk_contract with r = m-2).  Writes one report per problem (host array of
 * B entries); returns TK_ENOTCONV if any problem missed tol (a problem also
 * stops, unconverged, after 8 iterations in which neither F fell by more
 * than its rounding level under Armijo's test nor |grad F| fell below 0.999
 * of its best value: the rounding floor of the contraction, which rises with
 * |a|^{m-1}, has been reached).  Synchronises
 * `stream` once per step to read the per-problem scalars. */
int tk_solve_dual(const tk_problem *P, const tk_solve_opts *O, double *A_inout, tk_solve_report *R_host,
                  void *work, size_t work_bytes, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* TK_H */
