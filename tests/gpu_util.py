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


def accumulation_depth(n: int) -> int:
    """Longest chain of FP32 roundings on the way to one output of the
    contraction: <= n row contributions summed into a lane register or a
    warp's shared-memory slot per triangle, <= 32 chunk terms per row dot,
    5 shuffle levels, the per-triangle flushes of one warp (bounded by the
    number of triangles a warp can finish, <= n) and the O(m) products of
    the coefficients.  The cross-block sums are FP64."""
    return 2 * n + 64


def contraction_bound(n: int, abs_terms: np.ndarray, storage: str) -> np.ndarray:
    """Entrywise bound on |computed - exact| for a contraction of an
    already-rounded K: gamma_k * sum |terms| with k = accumulation_depth."""
    if storage == "f64":
        k = accumulation_depth(n)
        return 2.0 * k * U64 * abs_terms + 1e-300
    k = accumulation_depth(n)
    return 1.01 * k * U32 * abs_terms + 1e-30
