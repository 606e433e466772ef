// Internal declarations shared by the translation units of libtk.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/tk.h"
#include "tk_core.h"

namespace tk {

// thread-local last error message (tk_last_error)
void set_error(const char *fmt, ...);
int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

#define TK_CUDA_CHECK(call)                                     \
  do {                                                          \
    cudaError_t e__ = (call);                                   \
    if (e__ != cudaSuccess) return ::tk::cuda_fail(e__, #call); \
  } while (0)

// Layout of every workspace: a 256-byte header (status word and reserved
// counters) followed by the per-block partial sums of the contraction.
struct WsHeader {
  int status;                 // TK_OK, TK_ETIMEOUT or TK_EINVAL, set by kernels, read by tk_status_read
  int where;                  // which check or wait failed (diagnostic; kSite* below)
  unsigned long long ticket;  // next piece of the contraction to hand out
  unsigned int done;          // blocks of the current pass that have written their partials
  // key of the work plan the plan region holds, written with every upload;
  // the contraction kernel compares it with its own launch parameters and
  // returns before any load when they differ (a CUDA graph replayed after a
  // later call re-planned the region for another shape)
  int plan_m, plan_n, plan_pieces;
  long long plan_lo, plan_hi;
  int pad[52];
};
static_assert(sizeof(WsHeader) == 256, "header size");

// where-codes of the status word
enum { kSiteContractWait = 1, kSiteBatchedWait = 3, kSiteStalePlan = 4, kSiteUmmaWait = 5, kSiteTcWait = 6,
       kSiteDiagWait = 9 };

// The key to write into a workspace header after its plan region was filled.
inline WsHeader plan_key(int m, int n, int64_t lo, int64_t hi, int pieces) {
  WsHeader h{};
  h.plan_m = m;
  h.plan_n = n;
  h.plan_pieces = pieces;
  h.plan_lo = lo;
  h.plan_hi = hi;
  return h;
}

// Work of one warp of the contraction: rows [start, end) (row-aligned
// offsets); t[0..m-3] is the prefix Q of the first row, t[m-2] its c.
struct WarpPlan {
  int64_t start, end;
  int32_t t[kMaxOrder];
};
static_assert(sizeof(WarpPlan) == 48, "plan record");

// Row-aligned cut of [lo, hi) into `pieces` near-equal-cost pieces.
void build_plan(int m, int n, int64_t lo, int64_t hi, int pieces, int64_t row_cost, int64_t tri_cost,
                WarpPlan *out);

// Upload (once, cached per workspace address) the cut of [lo, hi) into
// `pieces` pieces into the plan region of workspace `work` (right after its
// header) and record the plan's key in the header.
int plan_to_device(int m, int n, int64_t lo, int64_t hi, int pieces, int row_cost, int tri_cost, void *work,
                   cudaStream_t st);
// Drop the host's record of which plan the workspace at `work` holds (the
// memory is about to hold something else, or is new memory at an address a
// workspace used before).
void forget_plan(void *work);
// The same for the Hessian pass's plan cached for the workspace at `work`.
void forget_hessian_plan(void *work);
// The same for the tensor-core batched contraction's plan.
void forget_tc_plan(void *work);

// Batched contraction (one pass for B vectors); returns TK_EUNSUPPORTED when
// the shape is outside what the batched kernel covers (callers then loop).
struct BatchedArgs {
  int m, n, storage;
  const void *K;
  int64_t off_lo, off_hi;
  int64_t B;
  int vec_dtype;
  const void *A;   // B x n
  const void *V;   // B x n or NULL (dual pass)
  void *G;         // B x n, vec_dtype (r = m-1: K[a^{m-1}]; dual: K[a^{m-2}, v])
  double *S;       // B or NULL (r = m-1 only)
  void *work;
  size_t work_bytes;
};
int contract_batched(const BatchedArgs &a, cudaStream_t st);
// Tensor-core batched contraction (r = m-1, whole tensor, FP32/BF16 storage,
// n <= 320): whether the current configuration takes it for this call, the
// workspace it needs, and the pass itself.
bool tc_covers(int m, int n, int storage, bool dual, int64_t B, int64_t off_lo, int64_t off_hi);
size_t tc_workspace_bytes(int m, int n, int64_t B, int sms);
int contract_batched_tc(const BatchedArgs &a, cudaStream_t st);
// Tensor-core packed build (FP32 / BF16 storage) and its status flag.
int build_tc(int m, int n, int d, const double *X, int feat, int degree, int storage, int64_t off_lo,
             int64_t off_hi, void *K, cudaStream_t st);
int build_tc_status(cudaStream_t st);
extern int g_build_tc_mode;  // 0: where it pays, 1: always (FP32/BF16), -1: never
extern tk_batched_config g_batched_cfg;
// resolved batched launch shape; returns false when the kernel does not cover it
bool batched_resolve(int n, int storage, bool dual, int64_t B, int sms, int smem_optin, tk_batched_config *out);
int64_t batched_min_batch(bool dual);
size_t batched_workspace_bytes(int n, int64_t B, int sms);

// Device properties cached per device.
struct DevInfo {
  int sms;
  int smem_optin;  // max dynamic shared memory per block
};
int dev_info(DevInfo *out);

// Sum the per-block partials of one pass into outputs (FP64, fixed order).
//   mode 0: G = value part (vec_dtype), S
//   mode 1: G = derivative part / (m-1)  (HVP)
//   mode 2: objective: F, grad (FP64), gnorm with alpha/y/lambda
struct FinalizeArgs {
  int mode;
  int m, n, grid;
  const double *part;
  int out_dtype;
  void *G;
  double *S;
  const double *alpha;  // mode 2
  const double *y;
  const double *lambda;
  double *F;
  double *grad;
  double *gnorm;
};
// One contraction pass of the single-vector kernel.
struct ContractArgs {
  int m;
  int n;
  int storage;      // TK_F64 / TK_F32 / TK_BF16
  const void *K;    // entry off_lo
  int64_t off_lo, off_hi;
  int vec_dtype;    // dtype of alpha / v
  const void *alpha;
  const void *v;    // non-NULL: dual pass (HVP)
  void *work;       // workspace: header, plan region, per-block partials
  int *status;      // workspace status word
  FinalizeArgs fin; // what the last block writes (part and grid are filled in by the pass)
};

// Launch the main pass; the partial sums land in args.part (layout
// part[block][vec][n + 2]: vec 0 = value, vec 1 = derivative; entry n = S).
int contract_pass(const ContractArgs &a, int *grid_out, const double **part_out, cudaStream_t st);

// Process-wide overrides of the contraction launch configuration.
extern tk_contract_config g_contract_cfg;
// Resolve the configuration of a pass (no launch); fills the kernel's ring,
// warps and grid parameters.
int contract_resolve(int m, int n, int storage, bool dual, tk_contract_config *out, int *grid);

// Plan state kept by a caller that owns a fixed scratch region: which plan
// (m, n, range, pieces, costs) its plan region currently holds.
struct StaticPlanState {
  int valid;
  int m, n;
  int64_t lo, hi;
  int pieces, rc, tc;
};

// Same pass as contract_pass, on a fixed scratch region of `scratch_bytes`
// bytes (header, plan region, partials laid out as in a workspace).  The plan
// is built into host_plan (capacity host_cap records; no host or device
// allocation) and uploaded only when it differs from *state; with
// `capturing` set, a pass that would have to upload a plan is refused
// (TK_EINVAL) before anything is issued on the stream.
int contract_pass_static(const ContractArgs &a, WarpPlan *host_plan, int host_cap, StaticPlanState *state,
                         size_t scratch_bytes, bool capturing, int *grid_out, const double **part_out,
                         cudaStream_t st);

// Bytes of the workspace regions (plan records for every warp of the largest
// launch, then the per-block partial sums).
size_t contract_plan_bytes(int sms);
size_t contract_part_bytes(int n, int grid);
size_t contract_workspace_bytes(int n, int sms);

}  // namespace tk
