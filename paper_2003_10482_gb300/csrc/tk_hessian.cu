// Full Hessian of the tensor-kernel term: Hk = K[a^{m-2}] as a dense n x n
// matrix, in one pass over the packed tensor (the dual Hessian of Section 4,
// eq. dual_tensor_kernel, is (m-1) Hk + lambda I).
//
// What is computed.  With S(a) = K[a^m] = sum_t mu(t) K_t a^t over the stored
// sorted tuples t (mu(t) = m!/prod_v cnt_t(v)!, the number of full index
// tuples t stands for), Hk = (1/(m(m-1))) d^2 S / da^2, and the second
// derivative of the monomial a^t = prod_k a_{t_k} is, over ordered pairs of
// distinct positions (k, l),
//   d^2 a^t / da_i da_j = sum_{k != l: t_k = i, t_l = j} prod_{r != k, l} a_{t_r}.
// Split every t into its triangle prefix Q = (t_1..t_{m-2}) (last value b) and
// its last two positions (c, d), b <= c <= d, and write w = mu(t)/(m(m-1)):
//   (A) positions (c, d):      Hk[c][d] and Hk[d][c] += w K A_Q   (A_Q = prod_Q a)
//   (B) a Q position k and c or d:
//                              Hk[Q_k][j] and Hk[j][Q_k] += B_k v_Q[j],
//       v_Q[j] = sum_{d >= j} w K_{Qjd} a_d + sum_{c <= j} w K_{Qcj} a_c,
//       B_k = A_Q without the factor of position k;
//   (C) two Q positions k != l: Hk[Q_k][Q_l] += B_kl tau_Q,
//       tau_Q = sum_{c <= d} w K_{Qcd} a_c a_d.
// The multinomial weight per entry: with M' = m!/prod_v cnt_Q(v)! and
// kb = cnt_Q(b): w = M'/(m(m-1)) times 1 (c > b, d > c), 1/2 (c = d > b),
// 1/(kb+1) (c = b < d) or 1/((kb+1)(kb+2)) (c = d = b).
//
// GB300 mapping.  The output is cut into 32 x 32 tiles of the upper triangle
// (rows c, columns d >= c).  A work item is one tile and a range of triangles
// in layout order, cut on the host so that items hold near-equal numbers of
// entries; one block of 8 warps runs an item.  Warp w owns rows c0+w+8i
// (i < 4) and lane j column d0+j: for each triangle every thread loads its
// four entries (row segments of the packed triangle: coalesced), adds term A
// into registers, and forms the row and column parts of v_Q and of tau_Q.  The
// row parts are reduced across lanes, the column parts across warps through
// shared memory; term B is then accumulated per prefix value q into a
// shared-memory table Z[q][j] (q <= the tile's last row, j the tile's 64 row
// and column indices), term C into the FP64 matrix C with atomic adds.  Items
// write their term-A tile and Z table to their own slots; a second kernel sums
// the slots in a fixed order and adds C.  Every entry is read from HBM once.
#include <cuda_bf16.h>
#include <stddef.h>
#include <string.h>

#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "tk_contract_impl.cuh"

namespace tk {

constexpr int kHT = 32;       // tile rows and columns
constexpr int kHW = 8;        // warps per block
constexpr int kHFlush = 64;   // triangles between flushes of the term-A registers (FP32 storage)
constexpr int kHMaxZBytes = 200 * 1024;

// One work item: tile (ti, tj) and the triangles whose (m-2)-tuple rank lies
// in [q_lo, q_hi); Q is the first of them, base the packed offset of (Q, b, b).
struct HItem {
  int ti, tj;
  int zrows;      // rows of the Z table (prefix values 0 .. zrows-1)
  int pad;
  int64_t q_lo, q_hi;
  int64_t base;
  int64_t zoff;   // offset of the item's Z slot (in values)
  int32_t Q[kMaxOrder];
};
static_assert(sizeof(HItem) == 80, "hessian item");

struct HParams {
  int m, n;
  const unsigned char *K;
  const double *alpha;
  const HItem *items;
  int nitems;
  int nt;              // tiles per side
  double *Apart;       // [item][32][32]
  double *Zpart;       // per item: [zrows][64]
  double *C;           // n x n, term C (atomic adds)
  int *status;
  int pieces;          // plan key: number of items
};

// First triangle at or after Q (lexicographic over sorted (m-2)-tuples) whose
// last value b is <= cmax: the prefix before the first position holding a
// value above cmax is advanced.  Returns false when none is left.
__host__ __device__ inline bool skip_to_useful(int m, int n, int cmax, int32_t *Q) {
  if (m <= 2) return true;
  const int len = m - 2;
  for (;;) {
    int j = 0;
    while (j < len && Q[j] <= cmax) ++j;
    if (j == len) return true;
    if (j == 0) return false;
    if (!next_sorted(j, n, Q)) return false;
    for (int i = j; i < len; ++i) Q[i] = Q[j - 1];
  }
}

// offset of (Q, b, b): the rank of the (m)-tuple Q b b
__host__ __device__ inline int64_t tri_base(int m, int n, const int32_t *Q) {
  if (m <= 2) return 0;
  int32_t t[kMaxOrder];
  for (int j = 0; j < m - 2; ++j) t[j] = Q[j];
  t[m - 2] = t[m - 1] = Q[m - 3];
  return rank(m, n, t);
}

__host__ __device__ inline int64_t qrank(int m, int n, const int32_t *Q) { return m <= 2 ? 0 : rank(m - 2, n, Q); }

template <typename ST, typename CT>
__device__ __forceinline__ CT ld_k(const unsigned char *K, int64_t off) {
  return ld_elem<ST, CT>(reinterpret_cast<const ST *>(K) + off);
}
template <>
__device__ __forceinline__ double ld_k<float, double>(const unsigned char *K, int64_t off) {
  return (double)reinterpret_cast<const float *>(K)[off];
}

template <typename ST, typename CT>
__global__ void __launch_bounds__(kHW * 32) hess_kernel(HParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  if (plan_is_stale(p.status, m, n, p.pieces, -1, -1)) return;
  const HItem it = p.items[blockIdx.x];
  const int c0 = kHT * it.ti, d0 = kHT * it.tj;
  const int cmax = min(c0 + kHT, n) - 1;
  const bool diag = it.ti == it.tj;
  CT *a_s = reinterpret_cast<CT *>(smem);                        // [n]
  CT *Z = a_s + ((n + 1) & ~1);                                  // [zrows][64]
  CT *rowbuf = Z + (size_t)it.zrows * 64;                        // [2][32]
  CT *colbuf = rowbuf + 2 * 32;                                  // [2][8][32]
  CT *taubuf = colbuf + 2 * kHW * 32;                            // [2][8]
  for (int i = threadIdx.x; i < n; i += blockDim.x) a_s[i] = (CT)p.alpha[i];
  for (int i = threadIdx.x; i < it.zrows * 64; i += blockDim.x) Z[i] = CT(0);
  __syncthreads();

  const int d = d0 + lane;
  const CT ad = d < n ? a_s[d] : CT(0);
  int crow[4];
  CT arow[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    crow[i] = c0 + w + 8 * i;
    arow[i] = crow[i] < n ? a_s[crow[i]] : CT(0);
  }
  CT accA[4] = {CT(0), CT(0), CT(0), CT(0)};
  double accA64[4] = {0.0, 0.0, 0.0, 0.0};
  const CT inv_mm1 = CT(1) / CT(m * (m - 1));

  int32_t Q[kMaxOrder];
  for (int j = 0; j < kMaxOrder; ++j) Q[j] = it.Q[j];
  int64_t qr = it.q_lo;
  int64_t base = it.base;
  int parity = 0, since_flush = 0;
  while (qr < it.q_hi) {
    const int b = (m > 2) ? Q[m - 3] : -1;
    if (b > cmax) {
      if (!skip_to_useful(m, n, cmax, Q)) break;
      qr = qrank(m, n, Q);
      base = tri_base(m, n, Q);
      continue;
    }
    // triangle constants (uniform over the block)
    uint64_t mp = 1;
    for (int i = 2; i <= m; ++i) mp *= (uint64_t)i;
    CT AQ = CT(1);
    int run = 0;
    for (int j = 0; j < m - 2; ++j) {
      AQ *= a_s[Q[j]];
      run = (j > 0 && Q[j] == Q[j - 1]) ? run + 1 : 1;
      if (run > 1) mp = exact_div_small(mp, run);
    }
    const int kb = (m > 2) ? run : 0;
    const CT w0 = CT(mp) * inv_mm1;
    const CT f_first = CT(1) / CT(kb + 1), f_firstdiag = CT(1) / CT(kb + 2);
    const int bb = b < 0 ? 0 : b;
    const int L = n - bb;

    // the four entries of this thread (rows c >= b, columns d >= c)
    CT x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int c = crow[i];
      const bool ok = c >= bb && c < n && d >= c && d < n;
      const int64_t ro = (int64_t)(c - bb) * (2 * n - bb - c + 1) / 2;
      x[i] = ok ? ld_k<ST, CT>(p.K, base + ro + (d - c)) : CT(0);
    }
    CT rowp[4], colp = CT(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int c = crow[i];
      const bool first = c == b, dg = d == c;
      const CT f = (first ? f_first : CT(1)) * (dg ? (first ? f_firstdiag : CT(0.5)) : CT(1));
      const CT wx = w0 * f * x[i];
      accA[i] += AQ * (dg ? CT(2) * wx : wx);
      rowp[i] = wx * ad;
      colp += wx * arow[i];
    }
    CT tau_w = CT(0);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      CT r = rowp[i];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
      rowp[i] = r;
      tau_w += arow[i] * r;
    }
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) rowbuf[parity * 32 + w + 8 * i] = rowp[i];
      taubuf[parity * kHW + w] = tau_w;
    }
    colbuf[(parity * kHW + w) * 32 + lane] = colp;
    __syncthreads();
    // term B: Z[q][slot] += cnt_q B_q v_Q[slot] for each distinct q of Q
    if (m > 2 && threadIdx.x < 64 && (!diag || threadIdx.x < 32)) {
      const int t = threadIdx.x;
      CT v;
      if (t < 32) {
        v = rowbuf[parity * 32 + t];
        if (diag)
          for (int ww = 0; ww < kHW; ++ww) v += colbuf[(parity * kHW + ww) * 32 + t];
      } else {
        v = CT(0);
        for (int ww = 0; ww < kHW; ++ww) v += colbuf[(parity * kHW + ww) * 32 + t - 32];
      }
      for (int j = 0; j < m - 2; ++j) {
        if (j > 0 && Q[j] == Q[j - 1]) continue;
        const int q = Q[j];
        int cnt = 0;
        CT Bq = CT(1);
        bool skipped = false;
        for (int jj = 0; jj < m - 2; ++jj) {
          if (Q[jj] == q) {
            ++cnt;
            if (!skipped) {
              skipped = true;
              continue;
            }
          }
          Bq *= a_s[Q[jj]];
        }
        Z[(size_t)q * 64 + t] += CT(cnt) * Bq * v;
      }
    }
    // term C: Hk[q][q'] += (ordered pairs of Q positions holding q, q') B tau
    if (m > 3 && threadIdx.x == 64) {
      CT tau = CT(0);
      for (int ww = 0; ww < kHW; ++ww) tau += taubuf[parity * kHW + ww];
      for (int j = 0; j < m - 2; ++j) {
        if (j > 0 && Q[j] == Q[j - 1]) continue;
        for (int k = 0; k < m - 2; ++k) {
          if (k > 0 && Q[k] == Q[k - 1]) continue;
          const int q = Q[j], q2 = Q[k];
          int cq = 0, cq2 = 0;
          for (int jj = 0; jj < m - 2; ++jj) {
            cq += Q[jj] == q;
            cq2 += Q[jj] == q2;
          }
          const int pairs = (q == q2) ? cq * (cq - 1) : cq * cq2;
          if (pairs == 0) continue;
          // B without one copy of q and one of q2
          CT Bqq = CT(1);
          int skip_q = 1, skip_q2 = 1;
          for (int jj = 0; jj < m - 2; ++jj) {
            if (Q[jj] == q && skip_q) {
              skip_q = 0;
              continue;
            }
            if (Q[jj] == q2 && skip_q2) {
              skip_q2 = 0;
              continue;
            }
            Bqq *= a_s[Q[jj]];
          }
          atomicAdd(&p.C[(size_t)q * n + q2], (double)(CT(pairs) * Bqq * tau));
        }
      }
    }
    parity ^= 1;
    if (sizeof(CT) == 4 && ++since_flush == kHFlush) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        accA64[i] += (double)accA[i];
        accA[i] = CT(0);
      }
      since_flush = 0;
    }
    base += (int64_t)L * (L + 1) / 2;
    if (m <= 2 || !next_sorted(m - 2, n, Q)) break;
    ++qr;
  }
  __syncthreads();
  // the item's slots: term-A tile and Z table
  double *A = p.Apart + (size_t)blockIdx.x * kHT * kHT;
#pragma unroll
  for (int i = 0; i < 4; ++i) A[(w + 8 * i) * kHT + lane] = accA64[i] + (double)accA[i];
  double *Zo = p.Zpart + it.zoff;
  for (int i = threadIdx.x; i < it.zrows * 64; i += blockDim.x) Zo[i] = (double)Z[i];
}

// Hk[r][s] from the item slots in a fixed order: term A of the tile holding
// (min(r,s), max(r,s)), term B of every item whose tile has r or s among its
// row or column indices, and term C.
__global__ void hess_assemble(int m, int n, int nt, const HItem *items, const int *item_of_tile,
                              const double *Apart, const double *Zpart, const double *C, double *H) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (s >= n) return;
  const int lo = min(r, s), hi = max(r, s);
  double h = 0.0;
  {  // term A
    const int ti = lo / kHT, tj = hi / kHT;
    const int tile = ti * nt - ti * (ti - 1) / 2 + (tj - ti);
    for (int k = item_of_tile[tile]; k < item_of_tile[tile + 1]; ++k)
      h += Apart[(size_t)k * kHT * kHT + (lo % kHT) * kHT + (hi % kHT)];
  }
  // term B: Z[q][slot j] of items, placed at (q, j) and (j, q)
  auto zsum = [&](int q, int j) -> double {
    double z = 0.0;
    const int tj_of_j = j / kHT;
    for (int ti = 0; ti < nt; ++ti) {
      for (int tj = ti; tj < nt; ++tj) {
        int slot = -1;
        if (ti == tj_of_j && tj == tj_of_j) slot = j % kHT;  // diagonal tile: combined slot
        else if (ti == tj_of_j) slot = j % kHT;              // j among the rows
        else if (tj == tj_of_j) slot = 32 + j % kHT;         // j among the columns
        if (slot < 0) continue;
        const int tile = ti * nt - ti * (ti - 1) / 2 + (tj - ti);
        for (int k = item_of_tile[tile]; k < item_of_tile[tile + 1]; ++k) {
          if (q >= items[k].zrows) continue;
          z += Zpart[items[k].zoff + (size_t)q * 64 + slot];
        }
      }
    }
    return z;
  };
  if (m > 2) h += zsum(r, s) + zsum(s, r);
  if (m > 3) h += C[(size_t)r * n + s];
  H[(size_t)r * n + s] = h;
}

// ------------------------------------------------------------------ host
struct HPlan {
  std::vector<HItem> items;
  std::vector<int> item_of_tile;  // tiles + 1 prefix
  int64_t zvalues;
  int zrows_max;
};

static void build_hplan(int m, int n, int target_items, HPlan *out) {
  const int nt = (n + kHT - 1) / kHT;
  std::vector<std::pair<int, int>> tiles;
  for (int ti = 0; ti < nt; ++ti)
    for (int tj = ti; tj < nt; ++tj) tiles.push_back({ti, tj});
  // cost of a triangle with last value b in a tile: its entries there plus a
  // fixed per-triangle overhead of the loop
  const int64_t kTriCost = 256;
  auto tile_cost = [&](int ti, int tj, std::vector<int64_t> &cost_b) {
    const int c0 = kHT * ti, c1 = std::min(c0 + kHT, n) - 1, d0 = kHT * tj, d1 = std::min(d0 + kHT, n) - 1;
    cost_b.assign(n + 1, 0);
    for (int b = -1; b < n; ++b) {
      int64_t e = 0;
      for (int c = std::max(std::max(b, 0), c0); c <= c1; ++c) e += std::max(0, d1 - std::max(c, d0) + 1);
      cost_b[b + 1] = (b <= c1) ? e + kTriCost : 0;
    }
  };
  // total cost
  std::vector<int64_t> cost_b;
  int64_t total = 0;
  const int64_t ntri = (m > 2) ? multiset(n, m - 2) : 1;
  for (auto &t : tiles) {
    tile_cost(t.first, t.second, cost_b);
    if (m <= 2) {
      total += cost_b[0];
      continue;
    }
    int32_t Q[kMaxOrder] = {0};
    const int cmax = std::min(kHT * t.first + kHT, n) - 1;
    for (;;) {
      if (!skip_to_useful(m, n, cmax, Q)) break;
      total += cost_b[Q[m - 3] + 1];
      if (!next_sorted(m - 2, n, Q)) break;
    }
  }
  const int64_t target = std::max<int64_t>(1, total / std::max(1, target_items));
  out->items.clear();
  out->item_of_tile.assign(tiles.size() + 1, 0);
  int64_t zoff = 0;
  int zmax = 0;
  for (size_t ti = 0; ti < tiles.size(); ++ti) {
    out->item_of_tile[ti] = (int)out->items.size();
    const int tI = tiles[ti].first, tJ = tiles[ti].second;
    tile_cost(tI, tJ, cost_b);
    const int cmax = std::min(kHT * tI + kHT, n) - 1;
    const int zrows = cmax + 1;
    auto emit = [&](const int32_t *Qs, int64_t qlo, int64_t qhi) {
      HItem h;
      memset(&h, 0, sizeof(h));
      h.ti = tI;
      h.tj = tJ;
      h.zrows = (m > 2) ? zrows : 0;
      h.q_lo = qlo;
      h.q_hi = qhi;
      for (int j = 0; j < kMaxOrder; ++j) h.Q[j] = Qs[j];
      h.base = tri_base(m, n, Qs);
      h.zoff = zoff;
      zoff += (int64_t)h.zrows * 64;
      zmax = std::max(zmax, h.zrows);
      out->items.push_back(h);
    };
    int32_t Q[kMaxOrder] = {0};
    if (m <= 2) {
      emit(Q, 0, 1);
      continue;
    }
    if (!skip_to_useful(m, n, cmax, Q)) continue;
    int32_t Qs[kMaxOrder];
    memcpy(Qs, Q, sizeof(Qs));
    int64_t qs = qrank(m, n, Q), acc = 0;
    for (;;) {
      acc += cost_b[Q[m - 3] + 1];
      int32_t Qn[kMaxOrder];
      memcpy(Qn, Q, sizeof(Qn));
      const bool more = next_sorted(m - 2, n, Qn) && skip_to_useful(m, n, cmax, Qn);
      if (!more) {
        emit(Qs, qs, ntri);
        break;
      }
      if (acc >= target) {
        const int64_t qn = qrank(m, n, Qn);
        emit(Qs, qs, qn);
        memcpy(Qs, Qn, sizeof(Qs));
        qs = qn;
        acc = 0;
      }
      memcpy(Q, Qn, sizeof(Q));
    }
  }
  out->item_of_tile[tiles.size()] = (int)out->items.size();
  out->zvalues = zoff;
  out->zrows_max = zmax;
}

struct HKey {
  int m, n, target;
  bool operator<(const HKey &o) const { return std::tie(m, n, target) < std::tie(o.m, o.n, o.target); }
};
static std::mutex g_hmu;
static std::map<HKey, HPlan> g_hplans;
static std::map<std::pair<int, const void *>, HKey> g_hup;

static int hess_target(int sms) { return sms * 4; }

static const HPlan &hplan_for(int m, int n, int sms) {
  HKey k{m, n, hess_target(sms)};
  auto it = g_hplans.find(k);
  if (it == g_hplans.end()) {
    if (g_hplans.size() > 16) g_hplans.clear();
    HPlan p;
    build_hplan(m, n, k.target, &p);
    it = g_hplans.emplace(k, std::move(p)).first;
  }
  return it->second;
}

// workspace: header | items (cap) | item_of_tile (cap) | Apart | Zpart | C
struct HLayout {
  size_t items, iot, apart, zpart, cmat, total;
};
static HLayout hess_layout(int n, const HPlan &pl) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  HLayout L;
  size_t off = sizeof(WsHeader);
  L.items = off;
  off = al(off + pl.items.size() * sizeof(HItem));
  L.iot = off;
  off = al(off + pl.item_of_tile.size() * sizeof(int));
  L.apart = off;
  off = al(off + pl.items.size() * kHT * kHT * sizeof(double));
  L.zpart = off;
  off = al(off + (size_t)pl.zvalues * sizeof(double));
  L.cmat = off;
  off = al(off + (size_t)n * n * sizeof(double));
  L.total = off;
  return L;
}

}  // namespace tk

using namespace tk;

extern "C" size_t tk_hessian_workspace_size(int m, int64_t n) {
  if (m < 2 || m > TK_MAX_ORDER || n < 1 || n > TK_MAX_POINTS) return 0;
  DevInfo di;
  if (dev_info(&di) != TK_OK) return 0;
  std::lock_guard<std::mutex> lk(g_hmu);
  const HPlan &pl = hplan_for(m, (int)n, di.sms);
  return hess_layout((int)n, pl).total;
}

extern "C" int tk_hessian(int m, int64_t n, int storage, const void *K, const double *alpha, double *H, void *work,
                          size_t work_bytes, void *stream) {
  if (m < 2 || m > TK_MAX_ORDER) return fail(TK_EINVAL, "order m=%d outside [2, %d]", m, TK_MAX_ORDER);
  if (n < 1) return fail(TK_EINVAL, "n must be >= 1");
  if (storage < TK_F64 || storage > TK_BF16) return fail(TK_EINVAL, "bad storage dtype %d", storage);
  if (!K || !alpha || !H || !work) return fail(TK_EINVAL, "NULL pointer");
  const int csize = storage == TK_F64 ? 8 : 4;
  const int64_t zrows_cap = (int64_t)n;  // prefix values lie in [0, n)
  const size_t zbytes = (size_t)zrows_cap * 64 * csize + ((n + 1) & ~1) * csize + (2 * 32 + 2 * kHW * 32 + 2 * kHW) * csize;
  if (n > TK_MAX_POINTS || zbytes > (size_t)kHMaxZBytes)
    return fail(TK_EUNSUPPORTED, "hessian pass: n=%lld too large for the shared-memory table (%zu bytes)",
                (long long)n, zbytes);
  if (tk_packed_size(m, n) < 0) return fail(TK_EOVERFLOW, "C(n+m-1, m) overflows");
  if (((uintptr_t)work & 15u) != 0) return fail(TK_EINVAL, "work must be 16-byte aligned");
  DevInfo di;
  int rc = dev_info(&di);
  if (rc != TK_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  TK_CUDA_CHECK(cudaGetDevice(&dev));
  unsigned char *ws = reinterpret_cast<unsigned char *>(work);
  std::lock_guard<std::mutex> lk(g_hmu);
  const HPlan &pl = hplan_for(m, (int)n, di.sms);
  const HLayout L = hess_layout((int)n, pl);
  if (work_bytes < L.total) return fail(TK_ENOMEM, "workspace %zu < %zu bytes", work_bytes, L.total);
  const int nitems = (int)pl.items.size();
  HKey key{m, (int)n, hess_target(di.sms)};
  auto up = g_hup.find({dev, work});
  if (up == g_hup.end() || up->second < key || key < up->second) {
    TK_CUDA_CHECK(cudaMemcpyAsync(ws + L.items, pl.items.data(), pl.items.size() * sizeof(HItem),
                                  cudaMemcpyHostToDevice, st));
    TK_CUDA_CHECK(cudaMemcpyAsync(ws + L.iot, pl.item_of_tile.data(), pl.item_of_tile.size() * sizeof(int),
                                  cudaMemcpyHostToDevice, st));
    const WsHeader h = plan_key(m, (int)n, -1, -1, nitems);
    TK_CUDA_CHECK(cudaMemcpyAsync(ws + offsetof(WsHeader, plan_m),
                                  reinterpret_cast<const unsigned char *>(&h) + offsetof(WsHeader, plan_m),
                                  offsetof(WsHeader, pad) - offsetof(WsHeader, plan_m), cudaMemcpyHostToDevice, st));
    TK_CUDA_CHECK(cudaStreamSynchronize(st));  // the plan lives in a cache that may be rebuilt
    g_hup[{dev, work}] = key;
  }
  HParams hp;
  hp.m = m;
  hp.n = (int)n;
  hp.K = reinterpret_cast<const unsigned char *>(K);
  hp.alpha = alpha;
  hp.items = reinterpret_cast<const HItem *>(ws + L.items);
  hp.nitems = nitems;
  hp.nt = (int)((n + kHT - 1) / kHT);
  hp.Apart = reinterpret_cast<double *>(ws + L.apart);
  hp.Zpart = reinterpret_cast<double *>(ws + L.zpart);
  hp.C = reinterpret_cast<double *>(ws + L.cmat);
  hp.status = reinterpret_cast<int *>(ws);
  hp.pieces = nitems;
  TK_CUDA_CHECK(cudaMemsetAsync(hp.C, 0, (size_t)n * n * sizeof(double), st));
  const size_t smem = (size_t)pl.zrows_max * 64 * csize + ((n + 1) & ~1) * csize +
                      (2 * 32 + 2 * kHW * 32 + 2 * kHW) * csize;
  if (nitems > 0) {
    if (storage == TK_F64) {
      TK_CUDA_CHECK(cudaFuncSetAttribute(hess_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
      hess_kernel<double, double><<<nitems, kHW * 32, smem, st>>>(hp);
    } else if (storage == TK_F32) {
      TK_CUDA_CHECK(cudaFuncSetAttribute(hess_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
      hess_kernel<float, float><<<nitems, kHW * 32, smem, st>>>(hp);
    } else {
      TK_CUDA_CHECK(cudaFuncSetAttribute(hess_kernel<__nv_bfloat16, float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      hess_kernel<__nv_bfloat16, float><<<nitems, kHW * 32, smem, st>>>(hp);
    }
    TK_CUDA_CHECK(cudaGetLastError());
  }
  dim3 g((unsigned)((n + 127) / 128), (unsigned)n);
  hess_assemble<<<g, 128, 0, st>>>(m, (int)n, hp.nt, hp.items, reinterpret_cast<const int *>(ws + L.iot), hp.Apart,
                                   hp.Zpart, hp.C, H);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}
