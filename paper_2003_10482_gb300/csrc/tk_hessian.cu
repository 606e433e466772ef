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
// (rows c, columns d >= c).  The triangles that reach a tile (last prefix
// value b <= the tile's last row) are listed on the host once per (m, n) --
// a table of every triangle's packed offset, prefix and multiplicities, and
// per work item a list of triangle indices -- and a work item is one tile and
// a run of its list, cut so that items hold near-equal numbers of entries.
// One block of 8 warps runs an item, 8 triangles at a time: 8 threads fetch
// the batch's records and form its prefix products; every thread issues its
// 32 loads (warp w owns rows c0+w+8i, i < 4, lane j column d0+j: row segments
// of the packed triangles, coalesced), adds term A into registers and forms
// the row and column parts of v_Q and tau_Q; the warp's 32 row sums are
// reduced by one butterfly reduce-scatter, the column parts across warps
// through shared memory.  Term B is accumulated per prefix value q into a
// shared-memory table Z[q][j] (q <= the tile's last row, j the tile's 64 row
// and column indices) by 64 threads, each owning one column j and taking the
// batch's triangles in order; term C goes into the FP64 matrix C with atomic
// adds.  Items write their term-A tile and Z table to their own slots; a
// second kernel sums the slots in a fixed order and adds C.  Every entry is
// read from HBM once.
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
constexpr int kHB = 8;        // triangles per batch (one barrier pair per batch)
constexpr int kHMaxZBytes = 200 * 1024;

// One work item: tile (ti, tj) and the triangles pairs[pair_lo, pair_hi) of
// the triangle table (all of them reach the tile).
struct HItem {
  int ti, tj;
  int zrows;      // rows of the Z table (prefix values 0 .. zrows-1)
  int pad;
  int64_t pair_lo, pair_hi;
  int64_t zoff;   // offset of the item's Z slot (in values)
};
static_assert(sizeof(HItem) == 40, "hessian item");

// One triangle: its packed offset (of (Q, b, b)), prefix values, last prefix
// value b, its multiplicity kb = cnt_Q(b) and M' = m!/prod_v cnt_Q(v)!.
struct HTriRec {
  int64_t base;
  uint16_t Q[kMaxOrder];
  int32_t b, kb;
  int32_t mprime, pad;
};
static_assert(sizeof(HTriRec) == 40, "triangle record");

struct HParams {
  int m, n;
  const unsigned char *K;
  const double *alpha;
  const HItem *items;
  const HTriRec *tris;
  const int32_t *pairs;
  int nitems;
  int nt;              // tiles per side
  double *Apart;       // [item][32][32]
  double *Zpart;       // per item: [zrows][64]
  double *C;           // n x n, term C (atomic adds)
  int *status;
  int pieces;          // plan key: number of items
};

template <typename ST, typename CT>
__device__ __forceinline__ CT ld_k(const unsigned char *K, int64_t off) {
  return ld_elem<ST, CT>(reinterpret_cast<const ST *>(K) + off);
}
template <>
__device__ __forceinline__ double ld_k<float, double>(const unsigned char *K, int64_t off) {
  return (double)reinterpret_cast<const float *>(K)[off];
}

// Per-triangle constants of a batch in shared memory: the prefix and, for
// term B, the distinct prefix values q with their coefficients cnt_q B_q.
template <typename CT>
struct HTri {
  int32_t Q[kMaxOrder];
  int nq;
  int qv[kMaxOrder];
  CT qc[kMaxOrder];
};

// Per (triangle, tile row) constants: the offset of the row's entry at column
// 0 (base + row offset - c; -1 when the row is not in the triangle), the
// entry weight w, the term-A weight A_Q w, and the extra factor of the head
// entry d = c.
template <typename CT>
struct HRow {
  int64_t base;
  CT cw, ca, dg;
};

// Sum of the 32 values v[0..31] held by every lane over the warp's lanes,
// scattered so that lane l ends with the sum of v[l]: five halving exchange
// steps (16 + 8 + 4 + 2 + 1 shuffles).
template <typename CT>
__device__ __forceinline__ CT warp_reduce_scatter32(CT (&v)[32], int lane) {
#pragma unroll
  for (int k = 16; k >= 1; k >>= 1) {
    const bool up = (lane & k) != 0;
#pragma unroll
    for (int j = 0; j < k; ++j) {
      // keep the half of the pair this lane is responsible for, send the other
      const CT send = up ? v[j] : v[j + k];
      const CT keep = up ? v[j + k] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, k);
    }
  }
  return v[0];
}

template <typename ST, typename CT>
__global__ void __launch_bounds__(kHW * 32) hess_kernel(HParams p) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int m = p.m, n = p.n;
  if (plan_is_stale(p.status, m, n, p.pieces, -1, -1)) return;
  const HItem it = p.items[blockIdx.x];
  const int c0 = kHT * it.ti, d0 = kHT * it.tj;
  const bool diag = it.ti == it.tj;
  CT *a_s = reinterpret_cast<CT *>(smem);                       // [n]
  CT *Z = a_s + ((n + 1) & ~1);                                 // [zrows][64]
  CT *rowbuf = Z + (size_t)it.zrows * 64;                       // [kHB][32]
  CT *colbuf = rowbuf + kHB * 32;                               // [kHB][8][32]
  CT *taubuf = colbuf + kHB * kHW * 32;                         // [kHB][8]
  HTri<CT> *tri = reinterpret_cast<HTri<CT> *>(taubuf + kHB * kHW);  // [kHB]
  HRow<CT> *rows = reinterpret_cast<HRow<CT> *>(tri + kHB);          // [kHB][32]
  for (int i = threadIdx.x; i < n; i += blockDim.x) a_s[i] = (CT)p.alpha[i];
  for (int i = threadIdx.x; i < it.zrows * 64; i += blockDim.x) Z[i] = CT(0);

  const int d = d0 + lane;
  int crow[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) crow[i] = c0 + w + 8 * i;
  CT accA[4] = {CT(0), CT(0), CT(0), CT(0)};
  double accA64[4] = {0.0, 0.0, 0.0, 0.0};
  const CT inv_mm1 = CT(1) / CT(m * (m - 1));
  int since_flush = 0;
  __syncthreads();
  const CT ad = d < n ? a_s[d] : CT(0);
  CT arow[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) arow[i] = crow[i] < n ? a_s[crow[i]] : CT(0);

  for (int64_t pos = it.pair_lo; pos < it.pair_hi; pos += kHB) {
    const int nb = (int)(it.pair_hi - pos < kHB ? it.pair_hi - pos : kHB);
    // ---- the batch's constants: thread (q, r) takes triangle q, tile row r
    {
      const int q = threadIdx.x >> 5, r = threadIdx.x & 31;
      if (q < nb) {
        const HTriRec rec = p.tris[p.pairs[pos + q]];
        CT AQ = CT(1);
        for (int j = 0; j < m - 2; ++j) AQ *= a_s[rec.Q[j]];
        const int b = rec.b, bb = b < 0 ? 0 : b;
        const int c = c0 + r;
        const bool in = c >= bb && c < n;
        const bool first = c == b;
        HRow<CT> hr;
        hr.base = in ? rec.base + (int64_t)(c - bb) * (2 * n - bb - c + 1) / 2 - c : -1;
        hr.cw = CT(rec.mprime) * inv_mm1 * (first ? kInvSmall<CT>[rec.kb + 1] : CT(1));
        hr.ca = AQ * hr.cw;
        hr.dg = first ? kInvSmall<CT>[rec.kb + 2] : CT(0.5);
        rows[q * 32 + r] = hr;
        if (r == 0) {
          // term B: the distinct prefix values and cnt_q B_q (B_q = A_Q without one factor of q)
          HTri<CT> &t = tri[q];
          int nq = 0;
          for (int j = 0; j < m - 2; ++j) {
            t.Q[j] = rec.Q[j];
            if (j > 0 && rec.Q[j] == rec.Q[j - 1]) continue;
            const int qv = rec.Q[j];
            int cnt = 0;
            CT Bq = CT(1);
            bool skipped = false;
            for (int jj = 0; jj < m - 2; ++jj) {
              if (rec.Q[jj] == qv) {
                ++cnt;
                if (!skipped) {
                  skipped = true;
                  continue;
                }
              }
              Bq *= a_s[rec.Q[jj]];
            }
            t.qv[nq] = qv;
            t.qc[nq] = CT(cnt) * Bq;
            ++nq;
          }
          t.nq = nq;
        }
      }
    }
    __syncthreads();

    // ---- loads of every triangle of the batch first, then the sums
    CT x[kHB][4];
#pragma unroll
    for (int q = 0; q < kHB; ++q) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        x[q][i] = CT(0);
        if (q < nb) {
          const int64_t rb = rows[q * 32 + w + 8 * i].base;
          if (rb >= 0 && d >= crow[i] && d < n) x[q][i] = ld_k<ST, CT>(p.K, rb + d);
        }
      }
    }
    CT rv[32];
    CT colp[kHB];
#pragma unroll
    for (int q = 0; q < kHB; ++q) {
      colp[q] = CT(0);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const HRow<CT> &hr = rows[q * 32 + w + 8 * i];
        const bool dgl = d == crow[i];
        // slots past the batch's last triangle and rows outside a triangle
        // hold x = 0; their constants are never used unguarded
        const CT xe = (q < nb) ? x[q][i] : CT(0);
        const CT cw = (q < nb) ? hr.cw : CT(0), ca = (q < nb) ? hr.ca : CT(0);
        const CT f = dgl ? ((q < nb) ? hr.dg : CT(0)) : CT(1);
        const CT wx = cw * f * xe;
        accA[i] += ca * (dgl ? CT(2) * f : f) * xe;
        rv[q * 4 + i] = wx * ad;
        colp[q] += wx * arow[i];
      }
    }
    // lane l: the row part of row c0 + w + 8 (l & 3) for triangle l >> 2
    const CT rsum = warp_reduce_scatter32(rv, lane);
    {
      const int q = lane >> 2, i = lane & 3;
      CT tv = arow[0];
#pragma unroll
      for (int k = 1; k < 4; ++k) tv = (i == k) ? arow[k] : tv;
      tv *= rsum;
      tv += __shfl_xor_sync(0xffffffffu, tv, 1);
      tv += __shfl_xor_sync(0xffffffffu, tv, 2);
      rowbuf[q * 32 + w + 8 * i] = rsum;
      if (i == 0) taubuf[q * kHW + w] = tv;
    }
#pragma unroll
    for (int q = 0; q < kHB; ++q) colbuf[(q * kHW + w) * 32 + lane] = colp[q];
    __syncthreads();

    // ---- term B: thread t < 64 owns column slot t of the Z table and adds
    // the batch's triangles in order
    if (m > 2 && threadIdx.x < 64 && (!diag || threadIdx.x < 32)) {
      const int t = threadIdx.x;
      for (int q = 0; q < nb; ++q) {
        CT v;
        if (t < 32) {
          v = rowbuf[q * 32 + t];
          if (diag)
            for (int ww = 0; ww < kHW; ++ww) v += colbuf[(q * kHW + ww) * 32 + t];
        } else {
          v = CT(0);
          for (int ww = 0; ww < kHW; ++ww) v += colbuf[(q * kHW + ww) * 32 + t - 32];
        }
        const HTri<CT> &tq = tri[q];
        for (int j = 0; j < tq.nq; ++j) Z[(size_t)tq.qv[j] * 64 + t] += tq.qc[j] * v;
      }
    }
    // ---- term C: one thread per triangle (warp 2)
    if (m > 3 && threadIdx.x >= 64 && threadIdx.x < 64 + nb) {
      const int q = threadIdx.x - 64;
      const int32_t *Qq = tri[q].Q;
      CT tau = CT(0);
      for (int ww = 0; ww < kHW; ++ww) tau += taubuf[q * kHW + ww];
      for (int j = 0; j < m - 2; ++j) {
        if (j > 0 && Qq[j] == Qq[j - 1]) continue;
        for (int k = 0; k < m - 2; ++k) {
          if (k > 0 && Qq[k] == Qq[k - 1]) continue;
          const int qa = Qq[j], qb = Qq[k];
          int ca = 0, cb = 0;
          for (int jj = 0; jj < m - 2; ++jj) {
            ca += Qq[jj] == qa;
            cb += Qq[jj] == qb;
          }
          const int pairs = (qa == qb) ? ca * (ca - 1) : ca * cb;
          if (pairs == 0) continue;
          CT Bqq = CT(1);
          int skip_a = 1, skip_b = 1;
          for (int jj = 0; jj < m - 2; ++jj) {
            if (Qq[jj] == qa && skip_a) {
              skip_a = 0;
              continue;
            }
            if (Qq[jj] == qb && skip_b) {
              skip_b = 0;
              continue;
            }
            Bqq *= a_s[Qq[jj]];
          }
          atomicAdd(&p.C[(size_t)qa * n + qb], (double)(CT(pairs) * Bqq * tau));
        }
      }
    }
    since_flush += nb;
    if (sizeof(CT) == 4 && since_flush >= kHFlush) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        accA64[i] += (double)accA[i];
        accA[i] = CT(0);
      }
      since_flush = 0;
    }
    __syncthreads();  // the batch's tables are read; the next batch may overwrite them
  }
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
                              const double *Apart, const double *Zpart, const double *C, double *H,
                              const int *status, int nitems) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (s >= n) return;
  // the plan the items come from must be this launch's (see hess_kernel):
  // on a mismatch write nothing and read no item
  const volatile WsHeader *wh = reinterpret_cast<const volatile WsHeader *>(status);
  if (!(wh->plan_m == m && wh->plan_n == n && wh->plan_pieces == nitems && wh->plan_lo == -1 && wh->plan_hi == -1))
    return;
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
  std::vector<HTriRec> tris;      // every triangle, layout order
  std::vector<int32_t> pairs;     // per item, the triangles it takes
  int64_t zvalues;
  int zrows_max;
};

static void build_hplan(int m, int n, int target_items, HPlan *out) {
  const int nt = (n + kHT - 1) / kHT;
  // every triangle in layout order, with its offset and multiplicities; the
  // triangles of each last prefix value b in a list of their own
  out->tris.clear();
  std::vector<std::vector<int32_t>> by_b(n + 1);  // index b + 1 (m = 2: b = -1)
  {
    int32_t Q[kMaxOrder] = {0};
    int64_t base = 0;
    uint64_t mfact = 1;
    for (int i = 2; i <= m; ++i) mfact *= (uint64_t)i;
    for (;;) {
      HTriRec r;
      memset(&r, 0, sizeof(r));
      r.base = base;
      for (int j = 0; j < kMaxOrder; ++j) r.Q[j] = (uint16_t)Q[j];
      uint64_t mp = mfact;
      int run = 0;
      for (int j = 0; j < m - 2; ++j) {
        run = (j > 0 && Q[j] == Q[j - 1]) ? run + 1 : 1;
        if (run > 1) mp = exact_div_small(mp, run);
      }
      r.b = (m > 2) ? Q[m - 3] : -1;
      r.kb = (m > 2) ? run : 0;
      r.mprime = (int32_t)mp;
      by_b[r.b + 1].push_back((int32_t)out->tris.size());
      out->tris.push_back(r);
      const int L = n - (r.b < 0 ? 0 : r.b);
      base += (int64_t)L * (L + 1) / 2;
      if (m <= 2 || !next_sorted(m - 2, n, Q)) break;
    }
  }
  std::vector<std::pair<int, int>> tiles;
  for (int ti = 0; ti < nt; ++ti)
    for (int tj = ti; tj < nt; ++tj) tiles.push_back({ti, tj});
  // cost of a triangle with last value b in a tile: its entries there plus a
  // fixed per-triangle overhead
  const int64_t kTriCost = 256;
  std::vector<std::vector<int64_t>> cost(tiles.size(), std::vector<int64_t>(n + 1, 0));
  int64_t total = 0;
  for (size_t k = 0; k < tiles.size(); ++k) {
    const int c0 = kHT * tiles[k].first, c1 = std::min(c0 + kHT, n) - 1;
    const int d0 = kHT * tiles[k].second, d1 = std::min(d0 + kHT, n) - 1;
    for (int b = -1; b <= c1 && b < n; ++b) {
      int64_t e = 0;
      for (int c = std::max(std::max(b, 0), c0); c <= c1; ++c) e += std::max(0, d1 - std::max(c, d0) + 1);
      cost[k][b + 1] = e + kTriCost;
      total += cost[k][b + 1] * (int64_t)by_b[b + 1].size();
    }
  }
  const int64_t target = std::max<int64_t>(1, total / std::max(1, target_items));
  out->items.clear();
  out->pairs.clear();
  out->item_of_tile.assign(tiles.size() + 1, 0);
  int64_t zoff = 0;
  int zmax = 0;
  for (size_t k = 0; k < tiles.size(); ++k) {
    out->item_of_tile[k] = (int)out->items.size();
    const int cmax = std::min(kHT * tiles[k].first + kHT, n) - 1;
    const int zrows = (m > 2) ? cmax + 1 : 0;
    int64_t lo = (int64_t)out->pairs.size(), acc = 0;
    auto emit = [&]() {
      HItem h;
      memset(&h, 0, sizeof(h));
      h.ti = tiles[k].first;
      h.tj = tiles[k].second;
      h.zrows = zrows;
      h.pair_lo = lo;
      h.pair_hi = (int64_t)out->pairs.size();
      h.zoff = zoff;
      zoff += (int64_t)zrows * 64;
      zmax = std::max(zmax, zrows);
      out->items.push_back(h);
      lo = h.pair_hi;
      acc = 0;
    };
    for (int b = -1; b <= cmax && b < n; ++b) {
      for (int32_t t : by_b[b + 1]) {
        out->pairs.push_back(t);
        acc += cost[k][b + 1];
        if (acc >= target) emit();
      }
    }
    if ((int64_t)out->pairs.size() > lo || out->items.size() == (size_t)out->item_of_tile[k]) emit();
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

void forget_hessian_plan(void *work) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  std::lock_guard<std::mutex> lk(g_hmu);
  g_hup.erase({dev, work});
}

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

// workspace: header | items | item_of_tile | triangle table | pairs | Apart | Zpart | C
struct HLayout {
  size_t items, iot, tris, pairs, apart, zpart, cmat, total;
};
static HLayout hess_layout(int n, const HPlan &pl) {
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  HLayout L;
  size_t off = sizeof(WsHeader);
  L.items = off;
  off = al(off + pl.items.size() * sizeof(HItem));
  L.iot = off;
  off = al(off + pl.item_of_tile.size() * sizeof(int));
  L.tris = off;
  off = al(off + pl.tris.size() * sizeof(HTriRec));
  L.pairs = off;
  off = al(off + pl.pairs.size() * sizeof(int32_t));
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
  const size_t tri_bytes = (storage == TK_F64) ? sizeof(HTri<double>) : sizeof(HTri<float>);
  const size_t row_bytes = (storage == TK_F64) ? sizeof(HRow<double>) : sizeof(HRow<float>);
  const size_t fixed = ((n + 1) & ~1) * csize + (size_t)(kHB * 32 + kHB * kHW * 32 + kHB * kHW) * csize + 16 +
                       kHB * tri_bytes + 16 + kHB * 32 * row_bytes;
  const size_t zbytes = (size_t)zrows_cap * 64 * csize + fixed;
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
  // the Hessian plan occupies the same region of a workspace as the
  // contraction plans: whatever those recorded for this address is void
  forget_plan(work);
  forget_tc_plan(work);
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
    TK_CUDA_CHECK(cudaMemcpyAsync(ws + L.tris, pl.tris.data(), pl.tris.size() * sizeof(HTriRec),
                                  cudaMemcpyHostToDevice, st));
    TK_CUDA_CHECK(cudaMemcpyAsync(ws + L.pairs, pl.pairs.data(), pl.pairs.size() * sizeof(int32_t),
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
  hp.tris = reinterpret_cast<const HTriRec *>(ws + L.tris);
  hp.pairs = reinterpret_cast<const int32_t *>(ws + L.pairs);
  hp.nitems = nitems;
  hp.nt = (int)((n + kHT - 1) / kHT);
  hp.Apart = reinterpret_cast<double *>(ws + L.apart);
  hp.Zpart = reinterpret_cast<double *>(ws + L.zpart);
  hp.C = reinterpret_cast<double *>(ws + L.cmat);
  hp.status = reinterpret_cast<int *>(ws);
  hp.pieces = nitems;
  TK_CUDA_CHECK(cudaMemsetAsync(hp.C, 0, (size_t)n * n * sizeof(double), st));
  const size_t smem = (size_t)pl.zrows_max * 64 * csize + fixed;
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
                                   hp.Zpart, hp.C, H, hp.status, nitems);
  TK_CUDA_CHECK(cudaGetLastError());
  return TK_OK;
}
