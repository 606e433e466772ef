// Host side of the packed contraction: the cost-balanced cut of the packed
// range into row-aligned pieces (cached per workspace), the launch
// configuration and the launch of the streaming kernel (tk_contract_impl.cuh,
// whose last block sums the per-block partials in a fixed order).
#include <stddef.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tk_contract_impl.cuh"

namespace tk {

int contract_launch_f64(const KParams &, bool, int, int, int, size_t, cudaStream_t);
int contract_launch_f32(const KParams &, bool, int, int, int, size_t, cudaStream_t);
int contract_launch_bf16(const KParams &, bool, int, int, int, size_t, cudaStream_t);

// ------------------------------------------------------------------ host
static int pick_nc(int n) {
  const int need = (n + 31) / 32;
  const int opts[] = {1, 2, 4, 8, 12, 16, 20, 24, 32};
  for (int o : opts)
    if (o >= need) return o;
  return -1;
}


tk_contract_config g_contract_cfg = {0, 0, 0, 0, 0, 0, 0, 0};

static const int kMaxWarps = 16;

static const int kMaxPiecesPerWarp = 16;
size_t contract_plan_bytes(int sms) { return (size_t)kMaxPiecesPerWarp * 2 * sms * kMaxWarps * sizeof(WarpPlan); }
size_t contract_part_bytes(int n, int grid) { return (size_t)grid * 2 * (size_t)(n + 2) * sizeof(double); }
size_t contract_workspace_bytes(int n, int sms) {
  return sizeof(WsHeader) + contract_plan_bytes(sms) + contract_part_bytes(n, 2 * sms);
}

// ------------------------------------------------------------------ plan
// Walk rows from `lo` in layout order.  Row c of triangle Q holds n - c
// entries; a triangle's remaining rows c..n-1 hold (n-c)(n-c+1)/2 entries.
struct RowCursor {
  int m, n;
  int32_t t[kMaxOrder];  // Q in t[0..m-3], c in t[m-2]
  int64_t pos;
  bool next_triangle() {
    if (m <= 2) return false;
    if (!next_sorted(m - 2, n, t)) return false;
    t[m - 2] = t[m - 3];
    return true;
  }
};

void build_plan(int m, int n, int64_t lo, int64_t hi, int pieces, int64_t row_cost, int64_t tri_cost,
                WarpPlan *out) {
  RowCursor cu;
  cu.m = m;
  cu.n = n;
  for (int j = 0; j < kMaxOrder; ++j) cu.t[j] = 0;
  if (lo < hi) unrank(m, n, lo, cu.t);
  cu.pos = lo;
  // pass 1: total cost
  int64_t total = 0;
  {
    RowCursor w = cu;
    while (w.pos < hi) {
      total += tri_cost;
      const int64_t R = n - w.t[m - 2];
      const int64_t E = R * (R + 1) / 2;
      if (w.pos + E <= hi) {
        total += E + row_cost * R;
        w.pos += E;
        if (w.pos < hi && !w.next_triangle()) break;
      } else {
        while (w.pos < hi) {
          total += (n - w.t[m - 2]) + row_cost;
          w.pos += n - w.t[m - 2];
          w.t[m - 2] += 1;
        }
      }
    }
  }
  // pass 2: the first row start whose preceding cost reaches w * total / pieces
  int wi = 1;
  auto target = [&](int w) { return (int64_t)((__int128)total * w / pieces); };
  auto emit = [&](const RowCursor &at) {
    out[wi - 1].end = at.pos;
    out[wi].start = at.pos;
    for (int j = 0; j < kMaxOrder; ++j) out[wi].t[j] = at.t[j];
    ++wi;
  };
  out[0].start = lo;
  for (int j = 0; j < kMaxOrder; ++j) out[0].t[j] = cu.t[j];
  int64_t cum = 0;
  RowCursor w = cu;
  while (w.pos < hi && wi < pieces) {
    cum += tri_cost;
    const int64_t R = n - w.t[m - 2];
    const int64_t E = R * (R + 1) / 2;
    const bool whole = w.pos + E <= hi;
    if (whole && cum + E + row_cost * R < target(wi)) {
      cum += E + row_cost * R;
      w.pos += E;
      if (w.pos < hi && !w.next_triangle()) break;
      continue;
    }
    // a cut falls inside this triangle (or the range ends in it): row by row
    while (w.pos < hi && w.t[m - 2] < n) {
      while (wi < pieces && cum >= target(wi)) emit(w);
      cum += (n - w.t[m - 2]) + row_cost;
      w.pos += n - w.t[m - 2];
      w.t[m - 2] += 1;
    }
    if (w.pos < hi && !w.next_triangle()) break;
  }
  RowCursor endc = w;
  endc.pos = hi;
  while (wi < pieces) emit(endc);
  out[pieces - 1].end = hi;
}

struct PlanKey {
  int m, n;
  int64_t lo, hi;
  int pieces, rc, tc;
  bool operator<(const PlanKey &o) const {
    return std::tie(m, n, lo, hi, pieces, rc, tc) < std::tie(o.m, o.n, o.lo, o.hi, o.pieces, o.rc, o.tc);
  }
  bool operator==(const PlanKey &o) const { return !(*this < o) && !(o < *this); }
};

static std::mutex g_plan_mu;
static std::map<PlanKey, std::vector<WarpPlan>> g_plans;
static std::map<std::pair<int, const void *>, PlanKey> g_uploaded;

// Record in a workspace header which plan its plan region now holds (the
// kernel checks the record against its launch parameters).
static int write_plan_key(void *work, const PlanKey &key, cudaStream_t st) {
  const WsHeader h = plan_key(key.m, key.n, key.lo, key.hi, key.pieces);
  unsigned char *dst = reinterpret_cast<unsigned char *>(work) + offsetof(WsHeader, plan_m);
  const size_t bytes = offsetof(WsHeader, pad) - offsetof(WsHeader, plan_m);
  TK_CUDA_CHECK(cudaMemcpyAsync(dst, reinterpret_cast<const unsigned char *>(&h) + offsetof(WsHeader, plan_m), bytes,
                                cudaMemcpyHostToDevice, st));
  return TK_OK;
}

// Make sure the plan for `key` sits in the plan region of workspace `work`
// (the region starts right after the 256-byte header).
static int ensure_plan(const PlanKey &key, void *work, cudaStream_t st) {
  int dev = 0;
  TK_CUDA_CHECK(cudaGetDevice(&dev));
  void *plan_region = reinterpret_cast<unsigned char *>(work) + sizeof(WsHeader);
  {
    std::lock_guard<std::mutex> lk(g_plan_mu);
    auto up = g_uploaded.find({dev, plan_region});
    if (up != g_uploaded.end() && up->second == key) return TK_OK;
  }
  // this upload overwrites what the Hessian and tensor-core passes may have
  // recorded for the same workspace
  forget_hessian_plan(work);
  forget_tc_plan(work);
  std::lock_guard<std::mutex> lk(g_plan_mu);
  auto it = g_plans.find(key);
  if (it == g_plans.end()) {
    if (g_plans.size() > 32) g_plans.clear();
    std::vector<WarpPlan> v(key.pieces);
    build_plan(key.m, key.n, key.lo, key.hi, key.pieces, key.rc, key.tc, v.data());
    it = g_plans.emplace(key, std::move(v)).first;
  }
  TK_CUDA_CHECK(cudaMemcpyAsync(plan_region, it->second.data(), it->second.size() * sizeof(WarpPlan),
                                cudaMemcpyHostToDevice, st));
  int rc = write_plan_key(work, key, st);
  if (rc != TK_OK) return rc;
  g_uploaded[{dev, plan_region}] = key;
  return TK_OK;
}

int plan_to_device(int m, int n, int64_t lo, int64_t hi, int pieces, int row_cost, int tri_cost, void *work,
                   cudaStream_t st) {
  PlanKey key{m, n, lo, hi, pieces, row_cost, tri_cost};
  return ensure_plan(key, work, st);
}

void forget_plan(void *work) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  void *plan_region = reinterpret_cast<unsigned char *>(work) + sizeof(WsHeader);
  std::lock_guard<std::mutex> lk(g_plan_mu);
  g_uploaded.erase({dev, plan_region});
}

// ------------------------------------------------------------------ launch config
struct Resolved {
  int nc, warps, nbuf, buf_bytes, cap, vec_bytes, warp_bytes, grid, cps, row_cost, tri_cost, ppw, schedule;
  size_t smem;
};

static int resolve(int m, int n, int storage, bool dual, Resolved *r) {
  DevInfo di;
  int rc = dev_info(&di);
  if (rc != TK_OK) return rc;
  const int es = dtype_size(storage);
  const int cts = storage == TK_F64 ? 8 : 4;
  r->nc = pick_nc(n);
  if (r->nc < 0) return fail(TK_EUNSUPPORTED, "contract: n=%d exceeds %d", n, TK_MAX_POINTS);
  const tk_contract_config &o = g_contract_cfg;
  r->nbuf = o.nbuf > 0 ? o.nbuf : 2;
  if (r->nbuf < 2 || r->nbuf > 8) return fail(TK_EINVAL, "nbuf outside [2, 8]");
  const int fixed = cts == 8 ? (dual ? warp_fixed_bytes<double, true>() : warp_fixed_bytes<double, false>())
                              : (dual ? warp_fixed_bytes<float, true>() : warp_fixed_bytes<float, false>());
  const int gbytes = ((dual ? 2 : 1) * n * cts + 127) & ~127;
  // staged vectors, then the rows-fit table (n+1 shorts) at the end of the region
  r->vec_bytes = ((dual ? 2 : 1) * n * cts + 2 * (n + 1) + 2 + 127) & ~127;
  r->cps = o.ctas_per_sm > 0 ? o.ctas_per_sm : 1;
  if (r->cps > 2) return fail(TK_EINVAL, "ctas_per_sm must be 1 or 2");
  // keep 4 KB for the kernel's static shared memory (warp S partials, final reduction)
  const int smem_budget = (di.smem_optin - 4096) / r->cps;
  // a buffer holds one full row (n entries) plus the alignment slack of its copy
  const int min_buf = (n * es + 32 + 127) & ~127;
  int warps = o.warps > 0 ? o.warps : kMaxWarps;
  warps = std::min(warps, max_threads_est(cts, dual, r->nc) / 32);
  int buf = 0;
  for (; warps >= 1; --warps) {
    const int per_warp = (smem_budget - r->vec_bytes) / warps;
    const int room = ((per_warp - fixed - gbytes) / r->nbuf) & ~127;
    buf = o.block_bytes > 0 ? o.block_bytes : std::min(room, 32768);
    if (buf >= min_buf && buf <= room) break;
    if (o.block_bytes > 0 && o.block_bytes < min_buf)
      return fail(TK_EINVAL, "block_bytes %d below one row (%d bytes)", o.block_bytes, min_buf);
  }
  if (warps < 1) return fail(TK_EUNSUPPORTED, "contract: shared memory too small for one warp");
  r->warps = warps;
  r->buf_bytes = buf;
  r->cap = (buf - 32) / es;
  r->warp_bytes = (fixed + gbytes + r->nbuf * r->buf_bytes + 127) & ~127;
  r->grid = di.sms * r->cps;
  r->smem = (size_t)r->vec_bytes + (size_t)warps * r->warp_bytes;
  // cost weights of the work cut: the dual (HVP) pass, BF16 storage and the
  // many small triangles of m >= 5 balance best with cheap rows and dear
  // triangles (measured on GB300 by the launch-configuration sweep: HVP m = 4,
  // n = 400 FP32 3.48 -> 3.80 TB/s; BF16 n = 600 3.70 -> 3.84 TB/s and its HVP
  // 2.40 -> 2.59 TB/s; m = 6, n = 80 0.60 -> 0.66 TB/s); the single FP32/FP64
  // pass at m <= 4 keeps 256 / 1024
  const bool cheap_rows = dual || storage == TK_BF16 || m >= 5;
  r->row_cost = o.row_cost > 0 ? o.row_cost : (cheap_rows ? 64 : 256);
  r->tri_cost = o.tri_cost > 0 ? o.tri_cost : (cheap_rows ? 4096 : 4 * r->row_cost);
  r->ppw = o.pieces_per_warp > 0 ? o.pieces_per_warp : 16;
  if (r->ppw > kMaxPiecesPerWarp) return fail(TK_EINVAL, "pieces_per_warp above %d", kMaxPiecesPerWarp);
  r->schedule = o.schedule > 0 ? o.schedule : 1;
  if (r->schedule > 2) return fail(TK_EINVAL, "schedule must be 1 or 2");
  return TK_OK;
}

int contract_resolve(int m, int n, int storage, bool dual, tk_contract_config *out, int *grid) {
  Resolved r;
  int rc = resolve(m, n, storage, dual, &r);
  if (rc != TK_OK) return rc;
  out->warps = r.warps;
  out->block_bytes = r.buf_bytes;
  out->nbuf = r.nbuf;
  out->ctas_per_sm = r.cps;
  out->row_cost = r.row_cost;
  out->tri_cost = r.tri_cost;
  out->pieces_per_warp = r.ppw;
  out->schedule = r.schedule;
  if (grid) *grid = r.grid;
  return TK_OK;
}

// Launch parameters of one pass over the workspace or scratch region at
// a.work (plan region after the header, partials after `plan_bytes`).
static KParams make_kparams(const ContractArgs &a, const Resolved &r, int pieces, size_t plan_bytes) {
  unsigned char *ws = reinterpret_cast<unsigned char *>(a.work);
  WsHeader *hdr = reinterpret_cast<WsHeader *>(ws);
  KParams kp;
  kp.m = a.m;
  kp.n = a.n;
  kp.K = reinterpret_cast<const unsigned char *>(a.K);
  kp.off_lo = a.off_lo;
  kp.off_hi = a.off_hi;
  kp.bytes = (a.off_hi - a.off_lo) * dtype_size(a.storage);
  kp.alpha = a.alpha;
  kp.v = a.v;
  kp.vec_dtype = a.vec_dtype;
  kp.part = reinterpret_cast<double *>(ws + sizeof(WsHeader) + plan_bytes);
  kp.status = a.status;
  kp.plan = reinterpret_cast<const WarpPlan *>(ws + sizeof(WsHeader));
  kp.pieces = pieces;
  kp.ticket = &hdr->ticket;
  kp.done = &hdr->done;
  kp.dynamic = r.schedule == 2;
  kp.fin = a.fin;
  kp.fin.part = kp.part;
  kp.fin.grid = r.grid;
  kp.fin.m = a.m;
  kp.fin.n = a.n;
  kp.warps = r.warps;
  kp.nbuf = r.nbuf;
  kp.buf_bytes = r.buf_bytes;
  kp.cap = r.cap;
  kp.vec_bytes = r.vec_bytes;
  kp.warp_bytes = r.warp_bytes;
  return kp;
}

static int launch_pass(const ContractArgs &a, const KParams &kp, const Resolved &r, bool dual, cudaStream_t st) {
  WsHeader *hdr = reinterpret_cast<WsHeader *>(a.work);
  TK_CUDA_CHECK(cudaMemsetAsync(&hdr->ticket, 0, sizeof(hdr->ticket) + sizeof(hdr->done), st));
  if (a.storage == TK_F64) return contract_launch_f64(kp, dual, r.nc, r.grid, r.warps * 32, r.smem, st);
  if (a.storage == TK_F32) return contract_launch_f32(kp, dual, r.nc, r.grid, r.warps * 32, r.smem, st);
  return contract_launch_bf16(kp, dual, r.nc, r.grid, r.warps * 32, r.smem, st);
}

int contract_pass(const ContractArgs &a, int *grid_out, const double **part_out, cudaStream_t st) {
  const bool dual = a.v != nullptr;
  Resolved r;
  int rc = resolve(a.m, a.n, a.storage, dual, &r);
  if (rc != TK_OK) return rc;
  DevInfo di;
  dev_info(&di);
  const int pieces = r.ppw * r.grid * r.warps;
  PlanKey key{a.m, a.n, a.off_lo, a.off_hi, pieces, r.row_cost, r.tri_cost};
  rc = ensure_plan(key, a.work, st);
  if (rc != TK_OK) return rc;
  const KParams kp = make_kparams(a, r, pieces, contract_plan_bytes(di.sms));
  if (grid_out) *grid_out = r.grid;
  if (part_out) *part_out = kp.part;
  return launch_pass(a, kp, r, dual, st);
}

int contract_pass_static(const ContractArgs &a, WarpPlan *host_plan, int host_cap, StaticPlanState *state,
                         size_t scratch_bytes, bool capturing, int *grid_out, const double **part_out,
                         cudaStream_t st) {
  const bool dual = a.v != nullptr;
  Resolved r;
  int rc = resolve(a.m, a.n, a.storage, dual, &r);
  if (rc != TK_OK) return rc;
  const int pieces = r.ppw * r.grid * r.warps;
  const size_t plan_bytes = (size_t)pieces * sizeof(WarpPlan);
  const size_t need = sizeof(WsHeader) + plan_bytes + contract_part_bytes(a.n, r.grid);
  if (pieces > host_cap || need > scratch_bytes)
    return fail(TK_ENOMEM, "contraction needs %zu bytes of scratch (%d plan records); the static scratch holds %zu",
                need, pieces, scratch_bytes);
  const bool current = state->valid && state->m == a.m && state->n == a.n && state->lo == a.off_lo &&
                       state->hi == a.off_hi && state->pieces == pieces && state->rc == r.row_cost &&
                       state->tc == r.tri_cost;
  if (!current) {
    // re-planning copies from host memory and waits for the copy: neither
    // may happen inside a stream capture, so refuse before touching the stream
    if (capturing)
      return fail(TK_EINVAL, "the static scratch holds no plan for m=%d, n=%d under the current launch "
                  "configuration: make one call with this shape outside stream capture first", a.m, a.n);
    build_plan(a.m, a.n, a.off_lo, a.off_hi, pieces, r.row_cost, r.tri_cost, host_plan);
    unsigned char *ws = reinterpret_cast<unsigned char *>(a.work);
    TK_CUDA_CHECK(cudaMemcpyAsync(ws + sizeof(WsHeader), host_plan, plan_bytes, cudaMemcpyHostToDevice, st));
    PlanKey key{a.m, a.n, a.off_lo, a.off_hi, pieces, r.row_cost, r.tri_cost};
    rc = write_plan_key(a.work, key, st);
    if (rc != TK_OK) return rc;
    // the host records are reused by the next rebuild: wait for the copy
    TK_CUDA_CHECK(cudaStreamSynchronize(st));
    *state = StaticPlanState{1, a.m, a.n, a.off_lo, a.off_hi, pieces, r.row_cost, r.tri_cost};
  }
  const KParams kp = make_kparams(a, r, pieces, plan_bytes);
  if (grid_out) *grid_out = r.grid;
  if (part_out) *part_out = kp.part;
  return launch_pass(a, kp, r, dual, st);
}


}  // namespace tk
