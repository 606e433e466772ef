"""torch.autograd wiring of the packed contractions.

S(a) = K[a^m] (Section 4, the first term of eq. dual_tensor_kernel, times m)
  forward            : one contraction pass (tk_contract, r = m-1; S is its by-product)
  backward           : dS/da = m K[a^{m-1}]            (the same contraction kernel)
  double backward    : d(v . dS/da)/da = m(m-1) K[a^{m-2}, v]
                       (the dual-number HVP pass, tk_contract with r = m-2)
The dual objective F (eq. dual_tensor_kernel) is tk_objective; its gradient comes
from the same pass and its Hessian-vector product from tk_dual_hvp.
Only scalings by m, m(m-1) and the incoming gradients happen in PyTorch.
"""
from __future__ import annotations

import torch

import paper_2003_10482_gb300 as tk


class _Grad(torch.autograd.Function):
    """a -> m K[a^{m-1}] (B x n), differentiable once more through the HVP."""

    @staticmethod
    def forward(ctx, alpha, K, m, n):
        ctx.save_for_backward(alpha)
        ctx.K, ctx.m, ctx.n = K, m, n
        G, _ = tk.tk_contract(K, m, n, alpha.detach())
        return m * G

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, gout):
        (alpha,) = ctx.saved_tensors
        m, n = ctx.m, ctx.n
        HV, _ = tk.tk_contract(ctx.K, m, n, alpha.detach(), r=m - 2, V=gout.contiguous().to(alpha.dtype))
        return m * (m - 1) * HV, None, None, None


class TensorKernelEnergy(torch.autograd.Function):
    """S(a) = K[a^m] for a of shape (n,) or (B, n); returns shape () or (B,)."""

    @staticmethod
    def forward(ctx, alpha, K, m, n):
        ctx.save_for_backward(alpha)
        ctx.K, ctx.m, ctx.n = K, m, n
        _, S = tk.tk_contract(K, m, n, alpha.detach())
        return S.reshape(()) if alpha.dim() == 1 else S.to(alpha.dtype)

    @staticmethod
    def backward(ctx, gout):
        (alpha,) = ctx.saved_tensors
        g = _Grad.apply(alpha, ctx.K, ctx.m, ctx.n)
        if alpha.dim() == 1:
            return gout.to(g.dtype) * g, None, None, None
        return gout.to(g.dtype).reshape(-1, 1) * g, None, None, None


def energy(alpha: torch.Tensor, K: torch.Tensor, m: int) -> torch.Tensor:
    """K[a^m] with first and second derivatives from the packed kernels."""
    n = alpha.shape[-1]
    return TensorKernelEnergy.apply(alpha, K, m, n)


class _DualGrad(torch.autograd.Function):
    """a -> grad F(a), the value computed by tk_objective in the forward pass;
    its derivative is the dual Hessian, applied by tk_dual_hvp."""

    @staticmethod
    def forward(ctx, alpha, grad, K, m, n, y, lam):
        ctx.save_for_backward(alpha)
        ctx.K, ctx.m, ctx.n, ctx.y, ctx.lam = K, m, n, y, lam
        return grad

    @staticmethod
    @torch.autograd.function.once_differentiable
    def backward(ctx, gout):
        (alpha,) = ctx.saved_tensors
        HV = tk.tk_dual_hvp(ctx.K, ctx.m, ctx.n, alpha.detach(), gout.contiguous(), ctx.lam)
        return HV.to(alpha.dtype), None, None, None, None, None, None


class DualObjective(torch.autograd.Function):
    """F(a) = K[a^m]/m + (lam/2)|a|^2 - <y, a> (eq. dual_tensor_kernel, lam = 1/gamma)
    for a of shape (n,) or (B, n): the forward pass is tk_objective (F and grad F in
    FP64 in one pass over K), the backward pass returns the incoming gradient
    times grad F, and the double backward the dual Hessian-vector product."""

    @staticmethod
    def forward(ctx, alpha, K, m, n, y, lam):
        F, grad, _ = tk.tk_objective(K, m, n, alpha.detach(), y, lam)
        ctx.save_for_backward(alpha, grad)
        ctx.K, ctx.m, ctx.n, ctx.y, ctx.lam = K, m, n, y, lam
        return F.reshape(()) if alpha.dim() == 1 else F

    @staticmethod
    def backward(ctx, gout):
        alpha, grad = ctx.saved_tensors
        g = _DualGrad.apply(alpha, grad.reshape(alpha.shape).to(alpha.dtype), ctx.K, ctx.m, ctx.n, ctx.y, ctx.lam)
        if alpha.dim() == 1:
            return gout.to(g.dtype) * g, None, None, None, None, None
        return gout.to(g.dtype).reshape(-1, 1) * g, None, None, None, None, None


def dual_objective(alpha: torch.Tensor, K: torch.Tensor, m: int, y: torch.Tensor, lam) -> torch.Tensor:
    """F(a) = K[a^m]/m + (lam/2)|a|^2 - <y, a> (eq. dual_tensor_kernel, lam = 1/gamma),
    evaluated by tk_objective, with first and second derivatives from the library."""
    n = alpha.shape[-1]
    return DualObjective.apply(alpha, K, m, n, y, lam)
