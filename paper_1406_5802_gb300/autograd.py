"""torch.autograd.Function over the randomized GENP solve.

Forward: X = A^{-1} B by the method of Fact 4.1 (multiplier G, GENP of A G, X = G Y, refinement), all in
librmge.  Backward: the adjoint kernel path ``rmge_solve_backward`` reuses the saved factors of A G:
  dB = A^{-T} dX = L^{-T} U^{-T} G^T dX,   dA = -dB X^T,
with dB refined on A^T dB = dX by the same sweeps as the forward solve.
The paper has no gradients; this is the adjoint of the solve its method computes.  PyTorch provides
device memory, streams and the autograd plumbing only.
"""
from __future__ import annotations

import torch

from . import rmge


class RmgeSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, seed: int, kind: str = "gaussian", prec: str = "f64", max_iters: int = 10,
                be_tol: float = 1e-13):
        A64 = A.detach().to(torch.float64).contiguous()
        B64 = B.detach().to(torch.float64).contiguous()
        out = rmge.gesv(kind, A64, B64, seed, prec=prec, max_iters=max_iters, be_tol=be_tol)
        X64 = out["X"]
        ctx.save_for_backward(out["LU"], out["G"], X64, A64)
        ctx.kind, ctx.prec, ctx.max_iters, ctx.be_tol = kind, prec, max_iters, be_tol
        ctx.info, ctx.berr, ctx.iters = out["info"], out["berr"], out["iters"]
        return X64.to(B.dtype)

    @staticmethod
    def backward(ctx, dX):
        LU, G, X64, A64 = ctx.saved_tensors
        need_a, need_b = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        # dB = A^{-T} dX from the saved factors, refined on A^T dB = dX like the forward solve
        dB, dA, ctx.berr_bwd, ctx.iters_bwd = rmge.solve_backward(
            ctx.kind, LU, G, X64, dX.detach().to(torch.float64).contiguous(), ctx.prec, want_dA=need_a, A=A64,
            max_iters=ctx.max_iters, be_tol=ctx.be_tol)
        gA = dA.to(dX.dtype) if need_a else None
        gB = dB.to(dX.dtype) if need_b else None
        return gA, gB, None, None, None, None, None


def rmge_solve(A, B, seed: int, kind: str = "gaussian", prec: str = "f64", max_iters: int = 10,
               be_tol: float = 1e-13):
    """Differentiable X = A^{-1} B through the randomized-multiplier GENP solve."""
    return RmgeSolve.apply(A, B, seed, kind, prec, max_iters, be_tol)


_POOLS: dict = {}


def _stream_pool(count: int, device) -> list:
    """The same side streams on every call, so that a training step that uses them can be captured in a
    CUDA graph (the streams fork from and join the capturing stream)."""
    key = (torch.cuda.current_device() if device is None else device, count)
    if key not in _POOLS:
        _POOLS[key] = [torch.cuda.Stream() for _ in range(count)]
    return _POOLS[key]


def rmge_solve_batched(As, Bs, seeds, kind: str = "gaussian", prec: str = "f32", streams: int = 8, **kw):
    """A list of independent differentiable solves, spread round-robin over CUDA streams so that small
    systems overlap on the GPU.  Returns the list of X."""
    pool = _stream_pool(max(1, streams), As[0].device.index if len(As) else None)
    cur = torch.cuda.current_stream()
    outs = []
    for i, (A, B, s) in enumerate(zip(As, Bs, seeds)):
        st = pool[i % len(pool)]
        st.wait_stream(cur)
        with torch.cuda.stream(st):
            outs.append(rmge_solve(A, B, s, kind, prec, **kw))
    for st in pool:
        cur.wait_stream(st)
    return outs
