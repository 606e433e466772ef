"""Helpers of the GPU parity tests: storage rounding on the host and the
error bounds the tests assert (derived from the kernels' arithmetic)."""
import numpy as np
import torch

import oracle

U32 = 2.0 ** -24   # unit roundoff of FP32
U64 = 2.0 ** -53
UBF16 = 2.0 ** -8  # unit roundoff of BF16 (8-bit significand incl. the implicit bit)

TORCH = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}


def round_storage(K64: np.ndarray, storage: str) -> torch.Tensor:
    """K rounded to the storage type on the host (round-to-nearest-even)."""
    return torch.from_numpy(np.ascontiguousarray(K64)).to(TORCH[storage])


def as_f64(Kt: torch.Tensor) -> np.ndarray:
    return Kt.to(torch.float64).cpu().numpy()


def max_warp_triangles(m: int, n: int, storage: str = "f32", lo: int = 0, hi: int | None = None,
                       dual: bool = False) -> int:
    """The most triangles (prefixes i_1..i_{m-2}) one warp of the contraction
    kernel enters under the default (static) schedule: the range is cut by
    tk_contract_plan into pieces_per_warp x W pieces and warp w takes pieces
    w, w+W, ...  A piece from offset s to e spans the triangles of the
    (m-2)-prefixes of its first and last entries and all between them."""
    import paper_2003_10482_gb300 as tk
    if m <= 2:
        return 1
    hi = oracle.packed_size(m, n) if hi is None else hi
    if hi <= lo:
        return 0
    cfg = tk.tk_contract_get_config(m, n, storage, dual)
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    W = sms * cfg["ctas_per_sm"] * cfg["warps"]
    pieces = cfg["pieces_per_warp"] * W
    cuts = tk.tk_contract_plan(m, n, lo, hi, pieces, cfg["row_cost"], cfg["tri_cost"])

    def tri(off):
        return oracle.rank(m - 2, n, oracle.unrank(m, n, off)[: m - 2])

    per_warp = [0] * W
    for i in range(pieces):
        s, e = cuts[i], cuts[i + 1]
        if e > s:
            per_warp[i % W] += tri(e - 1) - tri(s) + 1
    return max(per_warp)


def accumulation_depth(n: int, warp_triangles: int) -> int:
    """Longest chain of FP32 roundings on the way to one output of the
    contraction: <= n row contributions summed into a lane register within a
    triangle; per triangle a warp enters, at most three adds into its
    shared-memory slot of g (the register flush, the row epilogue of row l,
    the prefix term of l); <= 32 chunk terms per row dot, 5 shuffle levels and
    the O(m) products of the coefficients (the 64).  The cross-block sums are
    FP64."""
    return n + 3 * warp_triangles + 64


def contraction_bound(n: int, abs_terms: np.ndarray, storage: str, m: int, lo: int = 0, hi: int | None = None,
                      dual: bool = False, dynamic: bool = False) -> np.ndarray:
    """Entrywise bound on |computed - exact| for a contraction of an
    already-rounded K: gamma_k * sum |terms| with k = accumulation_depth.
    Under the shared-ticket schedule (dynamic) any warp may enter every
    triangle of the range, so T_w is the range's triangle count."""
    if dynamic:
        tw = oracle.packed_size(m - 2, n) if m > 2 else 1
    else:
        tw = max_warp_triangles(m, n, storage, lo, hi, dual)
    k = accumulation_depth(n, tw)
    if storage == "f64":
        return 2.0 * k * U64 * abs_terms + 1e-300
    return 1.01 * k * U32 * abs_terms + 1e-30


def batched_accumulation_depth(n: int, m: int, dual: bool = False) -> int:
    """Longest chain of FP32 roundings on the way to one output of the batched
    kernel (tk_batched.cu), read off its accumulation structure:

    * a thread's column accumulator receives at most one add per row of the
      block's slice (the entry's multiply-add, or the row's own epilogue for
      its own column) and one per triangle entered (the prefix terms); it is
      flushed to FP64 once 2048 rows have passed, checked after blocks of at
      most 16 rows: <= 2 (2048 + 15) + 1 adds between flushes;
    * a row dot: <= ceil(n/16) column terms in a thread, then the sum over the
      16 warps; a triangle's T: <= ceil(n/16) rows per warp, then 16 warps;
    * the products of a term: the FP64 -> FP32 conversions of its m-1 vector
      factors, the prefix product, the multinomial and 1/m scalings, the
      epilogue's few operations: <= 3m + 8;
    * the dual-number (HVP) pass adds, per product, the add of the product
      rule: <= 2m more.
    Cross-slice sums are FP64."""
    rows = 2048 + 16 - 1
    per = -(-n // 16)
    k = (2 * rows + 1) + 2 * (per + 16) + 3 * m + 8
    return k + (2 * m if dual else 0)


def batched_bound(abs_terms: np.ndarray, storage: str, n: int, m: int, dual: bool = False) -> np.ndarray:
    """Entrywise bound on |computed - exact| for the batched kernel on an
    already-rounded K: gamma_k * sum |terms| with k = batched_accumulation_depth."""
    k = batched_accumulation_depth(n, m, dual)
    return 1.01 * k * U32 * abs_terms + 1e-30


def hessian_bound(n: int, m: int, abs_terms: np.ndarray, storage: str) -> np.ndarray:
    """Entrywise bound on |computed - exact| for tk_hessian on an
    already-rounded K: gamma_k * sum |terms| with k the longest chain of
    roundings in the pass (tk_hessian.cu): a prefix-value table entry adds
    once per triangle of its work item (at most every triangle,
    C(n+m-3, m-2)); the term-A registers at most 64 triangles before an FP64
    flush; a row part 5 shuffle levels, a column part 4 rows and 8 warps; the
    products of a term (vector conversions, prefix products, weights) at most
    3m + 8.  Item slots are summed in FP64."""
    tri = oracle.packed_size(m - 2, n) if m > 2 else 1
    k = max(tri, 64) + 5 + 12 + 3 * m + 8
    u = U64 if storage == "f64" else U32
    return 1.01 * k * u * abs_terms + 1e-300


def tc_batched_rel(n: int, m: int) -> float:
    """Relative bound (times 2 sum |terms|) of the tensor-core batched
    contraction on an already-rounded K, from its arithmetic:
      * each product of the 3-term TF32 split misses x*a by at most
        3.01 * 2^-22 |x a| (lo*lo' and the two residuals of the split), after
        one rounding of the weighted entry and one of the FP64 vector (2u);
      * one accumulator sums the 3 (n + 31) products of a row (hi*hi',
        hi*lo', lo*hi' over at most n + 31 columns), each addition off by at
        most one FP32 ulp (2u; no rounding mode of the tensor cores assumed);
      * the epilogue: A_Q (M'/m) with 2m - 3 roundings plus the product, at
        most 2 x 128 additions into the FP32 g accumulator between FP64
        flushes (one row and one prefix addition per job), the quadratic-form
        sum over <= n rows, about 12 roundings in the triangle's finish and
        m + 2 in a prefix term.
    The factor 2 on sum |terms| covers the quadratic form: its absolute
    counterpart counts the column-b pairs twice (once in the row sum P, once
    in the a_b r_b correction)."""
    u = U32
    e_prod = 3.01 * 2.0 ** -22 + 2 * u
    e_acc = 2 * u * 3 * (n + 31)
    e_epi = u * ((2 * m - 2) + 2 * 128 + n + 12 + (m + 2))
    return e_prod + e_acc + e_epi


def tc_batched_bound(abs_terms: np.ndarray, n: int, m: int) -> np.ndarray:
    return 2.0 * tc_batched_rel(n, m) * abs_terms + 1e-30


def tc_build_rel(d: int, m: int) -> float:
    """Relative bound (times sum_k prod_j |x|) of the tensor-core build of FP32
    storage, from its arithmetic: w_Q rounded to FP32 and w_Q x (or x) in
    FP64 rounded to FP32 (3u per product); the 3-term TF32 split misses a
    product by at most 3.01 * 2^-22 of it; the hi*hi' accumulator sums at most
    d_pad = 32 ceil(d / 32) products, the cross-term one 2 d_pad products
    2^-10 smaller, each addition off by at most one FP32 ulp (2u: no rounding
    mode of the tensor cores assumed); one rounding joins the two
    accumulators."""
    u = U32
    d_pad = 32 * ((d + 31) // 32)
    return 3 * u + 3.01 * 2.0 ** -22 + 2 * u * d_pad + 2 * u * 2 * d_pad * 2.0 ** -10 * 1.001 + u


def build_rel(d: int, m: int, storage: str, tensor_cores: bool) -> float:
    """Relative bound (times sum_k prod_j |x|) of the linear build before the
    storage rounding: the SIMT build's FP32 (FP64) sum of d products of m
    factors, gamma_{d+m+2}, or the tensor-core build's (tc_build_rel)."""
    if storage != "f64" and tensor_cores:
        return tc_build_rel(d, m)
    u = U64 if storage == "f64" else U32
    return 1.01 * (d + m + 2) * u
