"""Python binding of libtk (include/tk.h): packed tensor-kernel l^p regression on GB300.

Thin argument marshalling over the C ABI, with the same function names.  Every
computation runs in the CUDA library; PyTorch only provides device memory and
streams.  There is no CPU fallback: if ``libtk.so`` has not been built the
import of the library fails loudly.

Tensor conventions: device tensors, contiguous; storage dtypes torch.float64 /
torch.float32 / torch.bfloat16 map to TK_F64 / TK_F32 / TK_BF16.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtk.so")

TK_OK, TK_EINVAL, TK_EOVERFLOW, TK_ENOMEM, TK_ECUDA, TK_ENOTCONV, TK_ETIMEOUT, TK_EUNSUPPORTED = range(8)
TK_F64, TK_F32, TK_BF16 = 0, 1, 2
TK_FEAT_LINEAR, TK_FEAT_POLY, TK_FEAT_EXP = 0, 1, 2
TK_NEWTON_CG, TK_GD_BT, TK_NEWTON_FULL = 0, 1, 2
_METHODS = {"newton_cg": TK_NEWTON_CG, "gd_bt": TK_GD_BT, "newton_full": TK_NEWTON_FULL}

_DT = {torch.float64: TK_F64, torch.float32: TK_F32, torch.bfloat16: TK_BF16}
_TORCH = {TK_F64: torch.float64, TK_F32: torch.float32, TK_BF16: torch.bfloat16}
_NAMES = {"f64": TK_F64, "f32": TK_F32, "bf16": TK_BF16}
_FEAT = {"linear": TK_FEAT_LINEAR, "poly": TK_FEAT_POLY, "exp": TK_FEAT_EXP}


class TKError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libtk error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def lib():
    """Load libtk.so (built by ``build_lib.build()``); raises if it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise ImportError(
                    f"{LIB_PATH} is missing: build it with "
                    "`python -m paper_2003_10482_gb300.build_lib` (no CPU fallback exists)")
            L = ctypes.CDLL(LIB_PATH)
            _declare(L)
            _lib = L
    return _lib


def _declare(L):
    i32, i64, u64, sz, dbl = ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_size_t, ctypes.c_double
    P = ctypes.c_void_p
    sig = {
        "tk_last_error": (ctypes.c_char_p, []),
        "tk_version": (ctypes.c_char_p, []),
        "tk_packed_size": (i64, [i32, i64]),
        "tk_packed_bytes": (i64, [i32, i64, i32]),
        "tk_rank": (i32, [i32, i64, P, P]),
        "tk_unrank": (i32, [i32, i64, i64, P]),
        "tk_row_align": (i32, [i32, i64, i64, P]),
        "tk_build_packed": (i32, [i32, i64, i64, P, i32, i32, i32, P, P]),
        "tk_build_packed_range": (i32, [i32, i64, i64, P, i32, i32, i32, i64, i64, P, P]),
        "tk_contract_workspace_size": (sz, [i32, i64, i64]),
        "tk_contract": (i32, [i32, i64, i32, P, i64, i32, P, i32, P, P, P, P, sz, P]),
        "tk_contract_range": (i32, [i32, i64, i32, P, i64, i64, i64, i32, P, i32, P, P, P, P, sz, P]),
        "tk_status_read": (i32, [P, P]),
        "tk_check_bounded_wait": (i32, [P, sz, ctypes.c_longlong, P]),
        "tk_contract_set_config": (i32, [P]),
        "tk_contract_get_config": (i32, [i32, i64, i32, i32, P]),
        "tk_batched_set_config": (i32, [P]),
        "tk_batched_get_config": (i32, [i32, i64, i32, i32, i64, P]),
        "tk_contract_plan": (i32, [i32, i64, i64, i64, i32, i32, i32, P]),
        "tk_objective": (i32, [i32, i64, i32, P, i64, P, P, P, P, P, P, P, sz, P]),
        "tk_assemble_objective": (i32, [i32, i64, i64, P, P, P, P, P, P, P, P, P]),
        "tk_objective_host_workspace_size": (sz, [i32, i64]),
        "tk_objective_host": (i32, [i32, i64, i32, P, P, P, P, P, P, sz, P]),
        "tk_contract_noalloc": (i32, [i32, i64, i32, P, i32, P, P, P, P]),
        "tk_contract_noalloc_status": (i32, [P]),
        "tk_workspace_release": (i32, [P]),
        "tk_dual_hvp": (i32, [i32, i64, i32, P, i64, P, P, P, P, P, sz, P]),
        "tk_support_threshold": (i32, [i64, i64, P, P, P, P]),
        "tk_solve_workspace_size": (sz, [P]),
        "tk_solve_workspace_size_opts": (sz, [P, P]),
        "tk_hessian_workspace_size": (sz, [i32, i64]),
        "tk_hessian": (i32, [i32, i64, i32, P, P, P, P, sz, P]),
        "tk_fma_probe": (i32, [i32, i32, ctypes.c_longlong, P, P]),
        "tk_umma_probe": (i32, [i32, i32, i32, P, P, P, P, sz, P]),
        "tk_build_set_config": (i32, [i32]),
        "tk_build_status": (i32, [P]),
        "tk_build_path": (i32, [i64, i32]),
        "tk_primal": (i32, [i32, i64, i64, P, i64, P, P, P]),
        "tk_predict": (i32, [i64, i64, P, i64, P, P, P]),
        "tk_nystrom_select": (i32, [i64, i64, u64, P]),
        "tk_solve_dual": (i32, [P, P, P, P, P, sz, P]),
    }
    for name, (res, args) in sig.items():
        if hasattr(L, name):
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args


def exported_symbols():
    """Names of the tk_* functions declared in include/tk.h."""
    import re
    hdr = os.path.join(os.path.dirname(_HERE), "include", "tk.h")
    with open(hdr) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(tk_[a-z0-9_]+)\s*\(", text)))


def _check(rc):
    if rc != TK_OK:
        raise TKError(rc, lib().tk_last_error().decode())


def _p(t):
    return ctypes.c_void_p(0 if t is None else t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def dtype_code(dt) -> int:
    if isinstance(dt, str):
        return _NAMES[dt]
    if isinstance(dt, int):
        return dt
    return _DT[dt]


def torch_dtype(code) -> torch.dtype:
    return _TORCH[dtype_code(code)]


# ------------------------------------------------------------------ layout (host)
def tk_packed_size(m: int, n: int) -> int:
    v = lib().tk_packed_size(m, n)
    if v < 0:
        raise TKError(TK_EOVERFLOW, f"C(n+m-1, m) invalid for m={m}, n={n}")
    return int(v)


def tk_packed_bytes(m: int, n: int, dtype) -> int:
    v = lib().tk_packed_bytes(m, n, dtype_code(dtype))
    if v < 0:
        raise TKError(TK_EINVAL, "bad size or dtype")
    return int(v)


def tk_rank(m: int, n: int, idx) -> int:
    a = (ctypes.c_int32 * m)(*[int(i) for i in idx])
    off = ctypes.c_int64()
    _check(lib().tk_rank(m, n, a, ctypes.byref(off)))
    return off.value


def tk_unrank(m: int, n: int, off: int) -> list[int]:
    a = (ctypes.c_int32 * m)()
    _check(lib().tk_unrank(m, n, off, a))
    return list(a)


def tk_row_align(m: int, n: int, off: int) -> int:
    r = ctypes.c_int64()
    _check(lib().tk_row_align(m, n, off, ctypes.byref(r)))
    return r.value


# ------------------------------------------------------------------ workspace
_ws_cache: dict = {}


def workspace(m: int, n: int, B: int = 1, device=None) -> torch.Tensor:
    """A cached device workspace large enough for contractions of (m, n, B)."""
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    with torch.cuda.device(dev):
        need = int(lib().tk_contract_workspace_size(m, n, B))
    if need == 0:
        raise TKError(TK_EINVAL, lib().tk_last_error().decode())
    key = dev.index
    t = _ws_cache.get(key)
    if t is None or t.numel() < need:
        t = new_workspace(need, dev)
        _ws_cache[key] = t
    return t


def new_workspace(nbytes: int, device) -> torch.Tensor:
    """Zeroed device memory for a workspace; the library forgets any work plan it
    recorded for a workspace that used this address before."""
    t = torch.zeros(nbytes, dtype=torch.uint8, device=device)
    _check(lib().tk_workspace_release(_p(t)))
    return t


class tk_contract_config(ctypes.Structure):
    _fields_ = [("warps", ctypes.c_int), ("block_bytes", ctypes.c_int), ("nbuf", ctypes.c_int),
                ("ctas_per_sm", ctypes.c_int), ("row_cost", ctypes.c_int), ("tri_cost", ctypes.c_int),
                ("pieces_per_warp", ctypes.c_int), ("schedule", ctypes.c_int)]


def tk_contract_set_config(warps=0, block_bytes=0, nbuf=0, ctas_per_sm=0, row_cost=0, tri_cost=0,
                           pieces_per_warp=0, schedule=0, reset=False):
    """Process-wide launch configuration of the contraction (0 = library choice)."""
    if reset:
        _check(lib().tk_contract_set_config(None))
        return
    c = tk_contract_config(warps, block_bytes, nbuf, ctas_per_sm, row_cost, tri_cost, pieces_per_warp, schedule)
    _check(lib().tk_contract_set_config(ctypes.byref(c)))


def tk_contract_plan(m: int, n: int, off_lo: int, off_hi: int, pieces: int, row_cost: int = 256,
                     tri_cost: int = 1024) -> list[int]:
    """Row-aligned cut of [off_lo, off_hi) into `pieces` near-equal-cost pieces (host only)."""
    out = (ctypes.c_int64 * (pieces + 1))()
    _check(lib().tk_contract_plan(m, n, off_lo, off_hi, pieces, row_cost, tri_cost, out))
    return list(out)


def tk_contract_get_config(m: int, n: int, storage="f32", dual: bool = False) -> dict:
    c = tk_contract_config()
    _check(lib().tk_contract_get_config(m, n, dtype_code(storage), int(dual), ctypes.byref(c)))
    return {f: getattr(c, f) for f, _ in c._fields_}


class tk_batched_config(ctypes.Structure):
    _fields_ = [("vpl", ctypes.c_int), ("block_bytes", ctypes.c_int), ("nbuf", ctypes.c_int),
                ("slice_mult", ctypes.c_int), ("min_batch", ctypes.c_int), ("tensor_cores", ctypes.c_int)]


def tk_batched_set_config(vpl=0, block_bytes=0, nbuf=0, slice_mult=0, min_batch=0, tensor_cores=0, reset=False):
    """Process-wide launch configuration of the batched contraction (0 = library choice;
    tensor_cores: 1 = the tcgen05 pass wherever it covers the call, -1 = never)."""
    if reset:
        _check(lib().tk_batched_set_config(None))
        return
    c = tk_batched_config(vpl, block_bytes, nbuf, slice_mult, min_batch, tensor_cores)
    _check(lib().tk_batched_set_config(ctypes.byref(c)))


def tk_batched_get_config(m: int, n: int, storage="f32", dual: bool = False, B: int = 512) -> dict:
    """The batched launch a contraction of B vectors would use (vpl 0: not covered)."""
    c = tk_batched_config()
    _check(lib().tk_batched_get_config(m, n, dtype_code(storage), int(dual), B, ctypes.byref(c)))
    return {f: getattr(c, f) for f, _ in c._fields_}


def tk_check_bounded_wait(work: torch.Tensor, budget_cycles: int = 1 << 22, stream=None) -> None:
    """Run the library's bounded device wait on a barrier nothing arrives on
    (diagnostic); the status word of `work` then reads TK_ETIMEOUT."""
    _check(lib().tk_check_bounded_wait(_p(work), work.numel(), budget_cycles, _stream(stream)))


def tk_fma_probe(dtype="f32", blocks: int = 0, iters: int = 1 << 16, reps: int = 3) -> float:
    """Measured multiply-add rate of the vector units (FLOP/s) for FP32 or FP64:
    the library's probe kernel timed with CUDA events (best of `reps`)."""
    dev = torch.cuda.current_device()
    if blocks <= 0:
        blocks = 8 * torch.cuda.get_device_properties(dev).multi_processor_count
    code = dtype_code(dtype)
    out = torch.empty(blocks, dtype=_TORCH[code], device="cuda")
    st = torch.cuda.current_stream()
    _check(lib().tk_fma_probe(code, blocks, iters, _p(out), _stream(st)))  # warm-up
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        _check(lib().tk_fma_probe(code, blocks, iters, _p(out), _stream(st)))
        e1.record(st)
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1) * 1e-3)
    return 2.0 * 16 * iters * 256 * blocks / best


def tk_umma_probe(A: torch.Tensor, B: torch.Tensor, split: bool = False, stream=None) -> torch.Tensor:
    """D = A B^T for one 128 x N tile on the tensor cores (tcgen05.mma,
    kind::tf32; split=True: the 3-term TF32 split).  A: 128 x k, B: N x k FP32."""
    assert A.is_cuda and B.is_cuda and A.dtype == torch.float32 and B.dtype == torch.float32
    A, B = A.contiguous(), B.contiguous()
    k = A.shape[1]
    assert A.shape[0] == 128 and B.shape[1] == k
    D = torch.empty(128, B.shape[0], dtype=torch.float32, device=A.device)
    work = new_workspace(256, A.device)
    _check(lib().tk_umma_probe(B.shape[0], k, int(bool(split)), _p(A), _p(B), _p(D), _p(work), work.numel(),
                               _stream(stream)))
    rc = tk_status_read(work, stream)
    if rc != TK_OK:
        raise TKError(rc, "the tensor-core probe's wait on its MMAs ran out")
    return D


def tk_build_set_config(tensor_cores: int = 0) -> None:
    """Which kernel builds FP32 / BF16 storage: 0 = tensor cores where they pay,
    1 = always the tensor-core build, -1 = always the SIMT build."""
    _check(lib().tk_build_set_config(int(tensor_cores)))


def tk_build_uses_tensor_cores(d: int, storage="f32") -> bool:
    """Whether a build of d features into `storage` takes the tensor-core build."""
    return bool(lib().tk_build_path(int(d), dtype_code(storage)))


def tk_build_status(stream=None) -> int:
    """TK_ETIMEOUT if a tensor-core build's bounded wait ran out since the last read."""
    return int(lib().tk_build_status(_stream(stream)))


def tk_status_read(work: torch.Tensor, stream=None) -> int:
    return int(lib().tk_status_read(_p(work), _stream(stream)))


# ------------------------------------------------------------------ build
def tk_build_packed(X: torch.Tensor, m: int, storage="f32", feat="linear", degree: int = 1,
                    K: torch.Tensor | None = None, off_lo: int | None = None,
                    off_hi: int | None = None, stream=None) -> torch.Tensor:
    """Packed order-m tensor kernel of the rows of X (n x d, FP64, device)."""
    assert X.is_cuda and X.dtype == torch.float64 and X.dim() == 2
    X = X.contiguous()
    n, d = X.shape
    code = dtype_code(storage)
    N = tk_packed_size(m, n)
    lo = 0 if off_lo is None else off_lo
    hi = N if off_hi is None else off_hi
    if K is None:
        K = torch.empty(hi - lo, dtype=_TORCH[code], device=X.device)
    assert K.numel() >= hi - lo and K.dtype == _TORCH[code]
    f = _FEAT[feat] if isinstance(feat, str) else int(feat)
    if off_lo is None and off_hi is None:
        _check(lib().tk_build_packed(m, n, d, _p(X), f, degree, code, _p(K), _stream(stream)))
    else:
        _check(lib().tk_build_packed_range(m, n, d, _p(X), f, degree, code, lo, hi, _p(K),
                                           _stream(stream)))
    return K


# ------------------------------------------------------------------ contraction
def tk_contract(K: torch.Tensor, m: int, n: int, A: torch.Tensor, r: int | None = None,
                V: torch.Tensor | None = None, G: torch.Tensor | None = None,
                S: torch.Tensor | None = None, off_lo: int | None = None,
                off_hi: int | None = None, work: torch.Tensor | None = None, stream=None):
    """G = K[A^{m-1}] and S = K[A^m] (r = m-1), or G = K[A^{m-2}, V] (r = m-2).

    A (and V): (n,) or (B, n) FP64/FP32 device tensors.  Returns (G, S) with G
    shaped like A and S a (B,) FP64 tensor (None for r = m-2)."""
    r = m - 1 if r is None else r
    squeeze = A.dim() == 1
    A2 = A.reshape(-1, n).contiguous()
    B = A2.shape[0]
    vdt = dtype_code(A2.dtype)
    V2 = None if V is None else V.reshape(B, n).to(A2.dtype).contiguous()
    if G is None:
        G = torch.empty_like(A2)
    if S is None and r == m - 1:
        S = torch.empty(B, dtype=torch.float64, device=A.device)
    if work is None:
        work = workspace(m, n, B, A.device)
    sc = dtype_code(K.dtype)
    if off_lo is None and off_hi is None:
        rc = lib().tk_contract(m, n, sc, _p(K), B, vdt, _p(A2), r, _p(V2), _p(G), _p(S),
                               _p(work), work.numel(), _stream(stream))
    else:
        rc = lib().tk_contract_range(m, n, sc, _p(K), off_lo, off_hi, B, vdt, _p(A2), r,
                                     _p(V2), _p(G), _p(S), _p(work), work.numel(),
                                     _stream(stream))
    _check(rc)
    if squeeze:
        G = G.reshape(n)
    return G, (S if r == m - 1 else None)


def tk_objective(K: torch.Tensor, m: int, n: int, A: torch.Tensor, y: torch.Tensor,
                 lam, work: torch.Tensor | None = None, stream=None):
    """(F, grad, gnorm) of the dual objective for each row of A (FP64)."""
    A2 = A.reshape(-1, n).to(torch.float64).contiguous()
    B = A2.shape[0]
    lam_t = torch.as_tensor(lam, dtype=torch.float64, device=A.device).reshape(-1)
    if lam_t.numel() == 1 and B > 1:
        lam_t = lam_t.expand(B).contiguous()
    F = torch.empty(B, dtype=torch.float64, device=A.device)
    gn = torch.empty(B, dtype=torch.float64, device=A.device)
    grad = torch.empty_like(A2)
    if work is None:
        work = workspace(m, n, B, A.device)
    _check(lib().tk_objective(m, n, dtype_code(K.dtype), _p(K), B, _p(A2),
                              _p(y.to(torch.float64).contiguous()), _p(lam_t), _p(F), _p(grad),
                              _p(gn), _p(work), work.numel(), _stream(stream)))
    return F, grad.reshape(A.shape), gn


_host_ws: dict = {}


def tk_objective_host(K: torch.Tensor, m: int, n: int, A_host: torch.Tensor, y: torch.Tensor, lam: torch.Tensor,
                      out_host: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The dual objective of one dual vector in host memory, results in host
    memory, in one C-ABI call (host -> device copy, pass, device -> host copy,
    stream synchronisation).  A_host: (n,) FP64 CPU tensor (pinned for speed);
    y, lam: device tensors.  Returns out_host = [F, |grad F|, grad F...] ((n+2,) FP64 CPU)."""
    if A_host.device.type != "cpu" or A_host.dtype != torch.float64 or not A_host.is_contiguous():
        raise TKError(TK_EINVAL, "A_host must be a contiguous FP64 CPU tensor")
    if out_host is None:
        out_host = torch.empty(n + 2, dtype=torch.float64, pin_memory=A_host.is_pinned())
    dev = K.device
    need = int(lib().tk_objective_host_workspace_size(m, n))
    if need == 0:
        raise TKError(TK_EINVAL, lib().tk_last_error().decode())
    ws = _host_ws.get(dev.index)
    if ws is None or ws.numel() < need:
        ws = new_workspace(need, dev)
        _host_ws[dev.index] = ws
    _check(lib().tk_objective_host(m, n, dtype_code(K.dtype), _p(K), ctypes.c_void_p(A_host.data_ptr()),
                                   _p(y), _p(lam), ctypes.c_void_p(out_host.data_ptr()), _p(ws), ws.numel(),
                                   _stream(stream)))
    return out_host


def tk_dual_hvp(K: torch.Tensor, m: int, n: int, A: torch.Tensor, V: torch.Tensor, lam,
                work: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """(m-1) K[a^{m-2}, v] + lam v for each row of A and V (the dual Hessian times v), FP64."""
    A2 = A.reshape(-1, n).to(torch.float64).contiguous()
    B = A2.shape[0]
    V2 = V.reshape(B, n).to(torch.float64).contiguous()
    lam_t = torch.as_tensor(lam, dtype=torch.float64, device=A.device).reshape(-1)
    if lam_t.numel() == 1 and B > 1:
        lam_t = lam_t.expand(B).contiguous()
    HV = torch.empty_like(A2)
    if work is None:
        work = workspace(m, n, B, A.device)
    _check(lib().tk_dual_hvp(m, n, dtype_code(K.dtype), _p(K), B, _p(A2), _p(V2), _p(lam_t), _p(HV),
                             _p(work), work.numel(), _stream(stream)))
    return HV.reshape(A.shape)


def tk_assemble_objective(m: int, n: int, G: torch.Tensor, S: torch.Tensor, A: torch.Tensor,
                          y: torch.Tensor, lam, stream=None):
    """(F, grad, gnorm) from reduced contractions G = K[A^{m-1}] (B x n) and S = K[A^m] (B)."""
    G2 = G.reshape(-1, n).to(torch.float64).contiguous()
    B = G2.shape[0]
    A2 = A.reshape(B, n).to(torch.float64).contiguous()
    S2 = S.reshape(B).to(torch.float64).contiguous()
    lam_t = torch.as_tensor(lam, dtype=torch.float64, device=G.device).reshape(-1)
    if lam_t.numel() == 1 and B > 1:
        lam_t = lam_t.expand(B).contiguous()
    F = torch.empty(B, dtype=torch.float64, device=G.device)
    gn = torch.empty(B, dtype=torch.float64, device=G.device)
    grad = torch.empty_like(A2)
    _check(lib().tk_assemble_objective(m, n, B, _p(G2), _p(S2), _p(A2),
                                       _p(y.to(torch.float64).contiguous()), _p(lam_t), _p(F),
                                       _p(grad), _p(gn), _stream(stream)))
    return F, grad.reshape(A.shape), gn


def tk_contract_noalloc(K: torch.Tensor, m: int, n: int, alpha: torch.Tensor, G: torch.Tensor,
                        S: torch.Tensor | None = None, stream=None):
    """K[alpha^{m-1}] into G and K[alpha^m] into S without any device allocation by the
    library (its scratch is a static device array); G and S are caller-owned."""
    _check(lib().tk_contract_noalloc(m, n, dtype_code(K.dtype), _p(K), dtype_code(alpha.dtype),
                                     _p(alpha), _p(G), _p(S), _stream(stream)))
    return G, S


def tk_contract_noalloc_status(stream=None) -> int:
    """Read and clear the status word of tk_contract_noalloc's static scratch on the
    current device (synchronises the stream): TK_OK, TK_ETIMEOUT or TK_EINVAL."""
    return int(lib().tk_contract_noalloc_status(_stream(stream)))


class tk_problem(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int64), ("storage_dtype", ctypes.c_int),
                ("K", ctypes.c_void_p), ("y", ctypes.c_void_p), ("B", ctypes.c_int64),
                ("lam", ctypes.c_void_p), ("mask", ctypes.c_void_p), ("K_hvp", ctypes.c_void_p),
                ("hvp_storage_dtype", ctypes.c_int)]


class tk_solve_opts(ctypes.Structure):
    _fields_ = [("method", ctypes.c_int), ("tol_gradnorm", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("max_cg", ctypes.c_int), ("armijo_c", ctypes.c_double), ("tol_rel_gap", ctypes.c_double),
                ("start_on_y", ctypes.c_int)]


class tk_solve_report(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("passes", ctypes.c_int), ("gradnorm", ctypes.c_double),
                ("F", ctypes.c_double), ("status", ctypes.c_int)]


_solve_ws: dict = {}


def tk_solve_dual(K: torch.Tensor, m: int, n: int, y: torch.Tensor, lam, alpha0: torch.Tensor | None = None,
                  mask: torch.Tensor | None = None, method: str = "newton_cg", tol: float = 1e-10,
                  max_iter: int = 100, max_cg: int = 0, rel_gap: float = 0.0, K_hvp: torch.Tensor | None = None,
                  start_on_y: bool | None = None, stream=None):
    """Solve B dual problems over the packed tensor K.  Returns (alpha (B x n FP64),
    reports (list of dicts), rc) where rc is TK_OK or TK_ENOTCONV.  A problem
    stops when |grad F| <= tol or (Newton-CG, rel_gap > 0) when its Newton
    decrement estimate of F - F* is <= rel_gap * max(1, |F|).  K_hvp: an optional
    lower-precision copy of K that only the Hessian-vector passes read.  start_on_y:
    start each problem at the minimiser of F along s*y (one extra pass; the default
    for method="newton_full" when alpha0 is None)."""
    dev = K.device
    lam_t = torch.as_tensor(lam, dtype=torch.float64, device=dev).reshape(-1).contiguous()
    B = lam_t.numel()
    A = torch.zeros(B, n, dtype=torch.float64, device=dev) if alpha0 is None else \
        alpha0.reshape(B, n).to(torch.float64).clone().contiguous()
    yd = y.to(dev, torch.float64).contiguous()
    mk = None if mask is None else mask.reshape(B, n).to(dev, torch.uint8).contiguous()
    prob = tk_problem(m, n, dtype_code(K.dtype), K.data_ptr(), yd.data_ptr(), B, lam_t.data_ptr(),
                      0 if mk is None else mk.data_ptr(), 0 if K_hvp is None else K_hvp.data_ptr(),
                      0 if K_hvp is None else dtype_code(K_hvp.dtype))
    if start_on_y is None:
        start_on_y = alpha0 is None and method == "newton_full"
    opts = tk_solve_opts(_METHODS[method], tol, max_iter, max_cg, 0.0, rel_gap, int(bool(start_on_y)))
    need = int(lib().tk_solve_workspace_size_opts(ctypes.byref(prob), ctypes.byref(opts)))
    if need == 0:
        raise TKError(TK_EINVAL, lib().tk_last_error().decode())
    key = dev.index
    ws = _solve_ws.get(key)
    if ws is None or ws.numel() < need:
        ws = new_workspace(need, dev)
        _solve_ws[key] = ws
    reps = (tk_solve_report * B)()
    rc = lib().tk_solve_dual(ctypes.byref(prob), ctypes.byref(opts), _p(A), reps, _p(ws), ws.numel(),
                             _stream(stream))
    if rc not in (TK_OK, TK_ENOTCONV):
        _check(rc)
    out = [{f: getattr(r, f) for f, _ in r._fields_} for r in reps]
    return A, out, rc


_hess_ws: dict = {}


def tk_hessian(K: torch.Tensor, m: int, n: int, alpha: torch.Tensor, H: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
    """K[alpha^{m-2}] as a dense symmetric n x n FP64 matrix, from one pass over K."""
    a = alpha.reshape(n).to(torch.float64).contiguous()
    if H is None:
        H = torch.empty(n, n, dtype=torch.float64, device=a.device)
    dev = a.device
    with torch.cuda.device(dev):
        need = int(lib().tk_hessian_workspace_size(m, n))
    if need == 0:
        raise TKError(TK_EINVAL, lib().tk_last_error().decode())
    ws = _hess_ws.get(dev.index)
    if ws is None or ws.numel() < need:
        ws = new_workspace(need, dev)
        _hess_ws[dev.index] = ws
    _check(lib().tk_hessian(m, n, dtype_code(K.dtype), _p(K), _p(a), _p(H), _p(ws), ws.numel(), _stream(stream)))
    return H


def tk_primal(X: torch.Tensor, A: torch.Tensor, m: int, stream=None) -> torch.Tensor:
    """w = J_q(X^T a) for each row of A (linear tensor kernel), FP64 (B x d)."""
    X = X.to(torch.float64).contiguous()
    n, d = X.shape
    A2 = A.reshape(-1, n).to(torch.float64).contiguous()
    W = torch.empty(A2.shape[0], d, dtype=torch.float64, device=X.device)
    _check(lib().tk_primal(m, n, d, _p(X), A2.shape[0], _p(A2), _p(W), _stream(stream)))
    return W if A.dim() > 1 else W.reshape(d)


def tk_predict(Xtest: torch.Tensor, W: torch.Tensor, stream=None) -> torch.Tensor:
    """<w_b, x_j> for every test row (B x t, FP64)."""
    Xt = Xtest.to(torch.float64).contiguous()
    t, d = Xt.shape
    W2 = W.reshape(-1, d).to(torch.float64).contiguous()
    Y = torch.empty(W2.shape[0], t, dtype=torch.float64, device=Xt.device)
    _check(lib().tk_predict(t, d, _p(Xt), W2.shape[0], _p(W2), _p(Y), _stream(stream)))
    return Y if W.dim() > 1 else Y.reshape(t)


def tk_nystrom_select(N: int, n_prime: int, seed: int) -> list[int]:
    """n' of N indices, uniform without replacement, sorted (host, Section 6.1)."""
    out = (ctypes.c_int64 * max(n_prime, 1))()
    _check(lib().tk_nystrom_select(N, n_prime, ctypes.c_uint64(seed & (2**64 - 1)), out))
    return list(out)[:n_prime]


def tk_support_threshold(W: torch.Tensor, stream=None):
    """keep[b][j] = |W[b][j]| > 2 std(W[b]) (Section 6.3) for a (d,) or (B, d) FP64
    device tensor; returns (keep (uint8, shaped like W), count (B,) int64)."""
    W2 = W.reshape(-1, W.shape[-1]).to(torch.float64).contiguous()
    B, d = W2.shape
    keep = torch.empty(B, d, dtype=torch.uint8, device=W.device)
    cnt = torch.empty(B, dtype=torch.int64, device=W.device)
    _check(lib().tk_support_threshold(d, B, _p(W2), _p(keep), _p(cnt), _stream(stream)))
    return keep.reshape(W.shape), cnt


def support_threshold(w: torch.Tensor) -> list[int]:
    """Indices of the features kept by the 2 std threshold of Section 6.3 (one
    weight vector, computed on the device by tk_support_threshold)."""
    keep, _ = tk_support_threshold(w.reshape(-1))
    return torch.nonzero(keep).reshape(-1).tolist()
