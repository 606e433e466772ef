/*
 * Plain FP64 CPU oracle for the packed symmetric tensor-kernel method
 * ("Efficient Tensor Kernel methods for sparse regression", Hibraj).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code with the CUDA library.
 *
 * Everything here is written to be checked against the thesis by eye, not to
 * be fast: single thread, FP64, one sorted index tuple at a time, in the
 * nested-loop storage order of Section 5.
 *
 *   - storage order (Section 5, the nested loops r <= c <= d <= t and the
 *     remark that higher orders nest one loop per index): lexicographic order
 *     of non-decreasing tuples i_1 <= ... <= i_m, first index slowest.
 *   - tensor entry (Section 4, general tensor kernel with the linear feature
 *     map phi(x) = x): K_{i_1..i_m} = sum_k prod_j x_{i_j,k}.
 *   - contraction (Section 4, eq. dual_tensor_kernel): the full sum over all
 *     n^m index tuples, evaluated over the stored (sorted) tuples by counting
 *     how many full tuples each stored tuple stands for (the multinomial
 *     coefficient of its index multiplicities).  The thesis does not spell
 *     the multiplicities out; this is the only weighting under which the
 *     packed sum equals the full-tensor sum.
 */
#include <stdint.h>
#include <stddef.h>
#include <string.h>
#include <math.h>

#define OR_MMAX 16

/* factorial as a double; exact for the small arguments used here (<= 16) */
static double or_fact(int k) {
    double f = 1.0;
    for (int i = 2; i <= k; ++i) f *= (double)i;
    return f;
}

/* Number of non-decreasing r-tuples with values in a set of k values
 * ("multiset coefficient"), computed by the product formula C(k+r-1, r).
 * Each partial product is itself a binomial coefficient, so every division
 * is exact. */
int64_t or_multichoose(int64_t k, int r) {
    if (r == 0) return 1;
    if (k <= 0) return 0;
    int64_t top = k + r - 1;
    int64_t c = 1;
    for (int i = 0; i < r; ++i) {
        c = c * (top - i) / (i + 1);
    }
    return c;
}

/* Number of stored entries of an order-m symmetric tensor over n points:
 * the count of sorted index tuples (Section 5: b_matrix, b_cube, b_tensor4
 * are the m = 2, 3, 4 cases). */
int64_t or_packed_size(int m, int64_t n) { return or_multichoose(n, m); }

/* Lexicographic rank of a sorted tuple: the number of sorted tuples that come
 * before it in the nested-loop order.  A tuple u comes before t iff at the
 * first position j where they differ u_j < t_j; for each position j and each
 * smaller value v in [t_{j-1}, t_j) the remaining m-j positions can hold any
 * sorted tuple with values in [v, n). */
int64_t or_rank(int m, int64_t n, const int32_t *t) {
    int64_t r = 0;
    int64_t lo = 0;
    for (int j = 0; j < m; ++j) {
        for (int64_t v = lo; v < t[j]; ++v) r += or_multichoose(n - v, m - 1 - j);
        lo = t[j];
    }
    return r;
}

/* Inverse of or_rank: walk the positions left to right and, at each, step the
 * value up while the block of tuples that start with the current value lies
 * entirely before the wanted offset. */
void or_unrank(int m, int64_t n, int64_t off, int32_t *t) {
    int64_t lo = 0;
    for (int j = 0; j < m; ++j) {
        int64_t v = lo;
        for (;;) {
            int64_t block = or_multichoose(n - v, m - 1 - j);
            if (off < block) break;
            off -= block;
            ++v;
        }
        t[j] = (int32_t)v;
        lo = v;
    }
}

/* Advance a sorted tuple to its successor in the nested-loop order.  Returns
 * 0 when t was the last tuple (all indices n-1). */
int or_next(int m, int64_t n, int32_t *t) {
    int j = m - 1;
    while (j >= 0 && t[j] == n - 1) --j;
    if (j < 0) return 0;
    t[j] += 1;
    for (int i = j + 1; i < m; ++i) t[i] = t[j];
    return 1;
}

/* Write every sorted tuple, in the nested-loop order, into out[N*m]. */
int64_t or_enumerate(int m, int64_t n, int32_t *out, int64_t cap) {
    int32_t t[OR_MMAX];
    for (int j = 0; j < m; ++j) t[j] = 0;
    int64_t k = 0;
    if (n <= 0) return 0;
    do {
        if (k >= cap) return -1;
        memcpy(out + k * m, t, sizeof(int32_t) * (size_t)m);
        ++k;
    } while (or_next(m, n, t));
    return k;
}

/* Tensor-kernel feature maps of Section 4.  feat 0: linear tensor kernel
 * k = sum_k prod_l x'_{l,k};  feat 1: polynomial tensor kernel of degree s,
 * (linear value)^s;  feat 2: exponential tensor kernel, exp(linear value). */
static double or_entry(int m, int64_t d, const double *X, const int32_t *t,
                       int feat, int s) {
    double acc = 0.0;
    for (int64_t k = 0; k < d; ++k) {
        double p = 1.0;
        for (int j = 0; j < m; ++j) p *= X[(int64_t)t[j] * d + k];
        acc += p;
    }
    if (feat == 1) {
        double v = 1.0;
        for (int i = 0; i < s; ++i) v *= acc;
        return v;
    }
    if (feat == 2) return exp(acc);
    return acc;
}

/* Packed build: K[o - lo] = k(x_{t_1}, ..., x_{t_m}) for the tuples t at
 * offsets o in [lo, hi).  X is n x d row-major. */
void or_build(int m, int64_t n, int64_t d, const double *X, int feat, int s,
              int64_t lo, int64_t hi, double *K) {
    int32_t t[OR_MMAX];
    if (hi <= lo) return;
    or_unrank(m, n, lo, t);
    for (int64_t o = lo; o < hi; ++o) {
        K[o - lo] = or_entry(m, d, X, t, feat, s);
        or_next(m, n, t);
    }
}

/* distinct values of a sorted tuple and their multiplicities */
static int or_runs(int m, const int32_t *t, int32_t *val, int *cnt) {
    int k = 0;
    for (int j = 0; j < m; ++j) {
        if (k > 0 && val[k - 1] == t[j]) {
            cnt[k - 1] += 1;
        } else {
            val[k] = t[j];
            cnt[k] = 1;
            ++k;
        }
    }
    return k;
}

/* number of distinct orderings of a multiset with the given multiplicities */
static double or_multinomial(const int *cnt, int k) {
    int tot = 0;
    double den = 1.0;
    for (int i = 0; i < k; ++i) {
        tot += cnt[i];
        den *= or_fact(cnt[i]);
    }
    return or_fact(tot) / den;
}

/* product of alpha over the multiset (val, cnt) */
static double or_prod(const int32_t *val, const int *cnt, int k, const double *alpha) {
    double p = 1.0;
    for (int i = 0; i < k; ++i)
        for (int c = 0; c < cnt[i]; ++c) p *= alpha[val[i]];
    return p;
}

/* Contraction over the stored entries with offsets in [lo, hi); K holds those
 * entries (K[0] is offset lo).  Adds into g[n] and *S (the caller zeroes them):
 *
 *   S   += mu(t) K_t prod_{j} alpha_{t_j}                  (K[alpha^m])
 *   g_l += K_t mu_{m-1}(t \ l) prod_{t \ l} alpha           (K[alpha^{m-1}]_l)
 *
 * for every distinct value l of t, where t \ l drops one copy of l and mu is
 * the multinomial coefficient of the multiplicities.  Summed over all sorted
 * tuples this is the full sum over n^m index tuples of eq. dual_tensor_kernel
 * (and of its gradient), because each stored tuple stands for exactly mu(t)
 * full tuples (respectively mu_{m-1}(t \ l) full tuples with first index l). */
void or_contract(int m, int64_t n, const double *K, int64_t lo, int64_t hi,
                 const double *alpha, double *g, double *S) {
    int32_t t[OR_MMAX], val[OR_MMAX];
    int cnt[OR_MMAX];
    if (hi <= lo) return;
    or_unrank(m, n, lo, t);
    double s = 0.0;
    for (int64_t o = lo; o < hi; ++o) {
        double k_t = K[o - lo];
        int k = or_runs(m, t, val, cnt);
        s += or_multinomial(cnt, k) * k_t * or_prod(val, cnt, k, alpha);
        for (int i = 0; i < k; ++i) {
            cnt[i] -= 1; /* t \ l */
            g[val[i]] += k_t * or_multinomial(cnt, k) * or_prod(val, cnt, k, alpha);
            cnt[i] += 1;
        }
        or_next(m, n, t);
    }
    *S += s;
}

/* Second-order contraction K[alpha^{m-2}] as a dense n x n matrix (row-major,
 * added into H):  H_{l,l'} += K_t mu_{m-2}(t \ {l,l'}) prod_{t \ {l,l'}} alpha
 * for every distinct l in t and every distinct l' in t \ l.  The dual Hessian
 * of eq. dual_tensor_kernel is (m-1) H + I/gamma. */
void or_hessian(int m, int64_t n, const double *K, int64_t lo, int64_t hi,
                const double *alpha, double *H) {
    int32_t t[OR_MMAX], val[OR_MMAX];
    int cnt[OR_MMAX];
    if (hi <= lo || m < 2) return;
    or_unrank(m, n, lo, t);
    for (int64_t o = lo; o < hi; ++o) {
        double k_t = K[o - lo];
        int k = or_runs(m, t, val, cnt);
        for (int i = 0; i < k; ++i) {
            cnt[i] -= 1;
            for (int i2 = 0; i2 < k; ++i2) {
                if (cnt[i2] == 0) continue;
                cnt[i2] -= 1;
                H[(int64_t)val[i] * n + val[i2]] +=
                    k_t * or_multinomial(cnt, k) * or_prod(val, cnt, k, alpha);
                cnt[i2] += 1;
            }
            cnt[i] += 1;
        }
        or_next(m, n, t);
    }
}

/* Mixed contraction K[alpha^{m-2}, v]_l (the Hessian-vector product without
 * the factor m-1), added into hv[n]:
 *   hv_l += K_t sum_{distinct l' in t \ l} mu_{m-2}(t \ {l,l'}) v_{l'} prod alpha */
void or_hvp(int m, int64_t n, const double *K, int64_t lo, int64_t hi,
            const double *alpha, const double *v, double *hv) {
    int32_t t[OR_MMAX], val[OR_MMAX];
    int cnt[OR_MMAX];
    if (hi <= lo || m < 2) return;
    or_unrank(m, n, lo, t);
    for (int64_t o = lo; o < hi; ++o) {
        double k_t = K[o - lo];
        int k = or_runs(m, t, val, cnt);
        for (int i = 0; i < k; ++i) {
            cnt[i] -= 1;
            for (int i2 = 0; i2 < k; ++i2) {
                if (cnt[i2] == 0) continue;
                cnt[i2] -= 1;
                hv[val[i]] += k_t * or_multinomial(cnt, k) * v[val[i2]] *
                              or_prod(val, cnt, k, alpha);
                cnt[i2] += 1;
            }
            cnt[i] += 1;
        }
        or_next(m, n, t);
    }
}

/* SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the state advances by the golden-ratio
 * increment and each output is the state passed through the published
 * variant-13 finaliser of MurmurHash3. */
static uint64_t or_splitmix64(uint64_t *state) {
    uint64_t z = (*state += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* uniform integer in [0, bound] by rejection on the top of the 64-bit range */
static uint64_t or_uniform(uint64_t *state, uint64_t bound) {
    uint64_t range = bound + 1;
    if (range == 0) return or_splitmix64(state);
    uint64_t limit = UINT64_MAX - (UINT64_MAX % range);
    uint64_t x;
    do { x = or_splitmix64(state); } while (x >= limit);
    return x % range;
}

/* Nystrom-like subsampling of Section 6.1: n' of the N training points drawn
 * uniformly without replacement.  Floyd's algorithm (Bentley and Floyd,
 * "Programming Pearls: A sample of brilliance", CACM 1987): for j = N-n' .. N-1
 * draw r uniform in [0, j]; take r unless already taken, else take j.  The
 * taken set is returned sorted ascending.  Membership is checked by a linear
 * scan: slow and obviously correct. */
int or_nystrom_select(int64_t N, int64_t np, uint64_t seed, int64_t *out) {
    if (np < 0 || np > N) return -1;
    uint64_t state = seed;
    int64_t k = 0;
    for (int64_t j = N - np; j < N; ++j) {
        int64_t r = (int64_t)or_uniform(&state, (uint64_t)j);
        int taken = 0;
        for (int64_t i = 0; i < k; ++i) if (out[i] == r) { taken = 1; break; }
        out[k++] = taken ? j : r;
    }
    /* insertion sort */
    for (int64_t i = 1; i < k; ++i) {
        int64_t x = out[i], j = i - 1;
        while (j >= 0 && out[j] > x) { out[j + 1] = out[j]; --j; }
        out[j + 1] = x;
    }
    return 0;
}
