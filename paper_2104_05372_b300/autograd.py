"""torch.autograd.Function wrappers over the C ABI (hand-written adjoints).

GMMObjective: forward = gmm_objective, backward = gmm_vjp with the incoming
cotangent as seed (grad f = transpose (linearize f) 1.0, Sec. 5.2). The
per-point log-joint s[k][i] is saved for the backward pass when K * N * 4 bytes
fit the memory budget; otherwise the backward pass recomputes it chunk-wise
inside gmm_vjp (a workspace of ``budget_bytes`` bounds the chunk).

ReprojResidual: forward = reproj_residual, backward = reproj_vjp (Accum scatter
into per-camera and per-point cotangents).
"""
from __future__ import annotations

import os

import torch

from . import _lib

DEFAULT_LOGJOINT_BUDGET = int(os.environ.get("GPA_LSE_BUDGET_BYTES", str(8 << 30)))


class GMMObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, alpha, mu, q, l, gamma=1.0, m=0, prec=_lib.PREC_FP32, budget_bytes=None):
        budget = DEFAULT_LOGJOINT_BUDGET if budget_bytes is None else int(budget_bytes)
        n, d = x.shape
        k = alpha.shape[0]
        x, alpha, mu, q, l = (t.contiguous() for t in (x, alpha, mu, q, l))
        store = 4 * n * k <= budget
        lse = torch.empty(n, dtype=torch.float32, device=x.device) if store else None
        lj = torch.empty(k, n, dtype=torch.float32, device=x.device) if store else None
        out = _lib.gmm_objective(x, alpha, mu, q, l, gamma, m, prec, lse_out=lse, logjoint_out=lj)
        ctx.save_for_backward(x, alpha, mu, q, l)
        ctx.lj, ctx.lse = lj, lse
        ctx.gamma, ctx.m, ctx.prec, ctx.budget = gamma, m, prec, budget
        return out[0]

    @staticmethod
    def backward(ctx, grad_out):
        x, alpha, mu, q, l = ctx.saved_tensors
        n, d = x.shape
        k = alpha.shape[0]
        # The C ABI takes the cotangent seed as a host scalar (every kernel gets
        # it as a launch argument), so it is read here: one device-to-host copy
        # of one float64 per backward pass. It waits for the stream up to the
        # objective, which the gradient kernels depend on anyway.
        seed = float(grad_out.item())
        lp = 0
        if ctx.lj is None:  # chunk size that keeps the log-joint within the budget
            lp = max(128, (ctx.budget // (4 * (k + 1))) // 128 * 128)
        da, dm, dq, dl = _lib.gmm_vjp(x, alpha, mu, q, l, ctx.gamma, ctx.m, ctx.prec, logjoint_in=ctx.lj,
                                      lse_in=ctx.lse, seed=seed, logjoint_points=lp)
        ctx.lj = ctx.lse = None
        return None, da, dm, dq, dl, None, None, None, None


def gmm_objective(x, alpha, mu, q, l, gamma=1.0, m=0, prec=_lib.PREC_FP32, budget_bytes=None):
    """Differentiable GMM log-posterior (gradients for alpha, mu, q, l)."""
    return GMMObjective.apply(x, alpha, mu, q, l, gamma, m, prec, budget_bytes)


class ReprojResidual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cams, pts, obs, tgt, strat="auto", plan=None):
        cams, pts, obs, tgt = (t.contiguous() for t in (cams, pts, obs, tgt))
        # with a plan the residual is computed in its camera-sorted order too
        # (bit-identical to the input-order kernel)
        sorted_plan = plan if plan is not None and strat in ("auto", "sort") else None
        res = _lib.reproj_residual(cams, pts, obs, tgt, plan=sorted_plan)
        ctx.save_for_backward(cams, pts, obs)
        ctx.strat, ctx.plan = strat, plan
        return res

    @staticmethod
    def backward(ctx, w):
        cams, pts, obs = ctx.saved_tensors
        dc, dp = _lib.reproj_vjp(cams, pts, obs, w.contiguous(), strat=ctx.strat, plan=ctx.plan)
        return dc, dp, None, None, None, None


def reproj_residual(cams, pts, obs, tgt, strat="auto", plan=None):
    """Differentiable reprojection residual [M, 2] (gradients for cams, pts)."""
    return ReprojResidual.apply(cams, pts, obs, tgt, strat, plan)
