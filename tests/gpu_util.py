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
                      dual: bool = False) -> np.ndarray:
    """Entrywise bound on |computed - exact| for a contraction of an
    already-rounded K: gamma_k * sum |terms| with k = accumulation_depth."""
    k = accumulation_depth(n, max_warp_triangles(m, n, storage, lo, hi, dual))
    if storage == "f64":
        return 2.0 * k * U64 * abs_terms + 1e-300
    return 1.01 * k * U32 * abs_terms + 1e-30


def batched_bound(abs_terms: np.ndarray, storage: str, n: int) -> np.ndarray:
    """The batched kernel flushes its FP32 partials to FP64 every 2048 rows:
    gamma_k * sum |terms| with k = 2 max(n, 2048) + 64."""
    k = 2 * max(n, 2048) + 64
    if storage == "f64":
        return 2.0 * k * U64 * abs_terms + 1e-300
    return 1.01 * k * U32 * abs_terms + 1e-30
