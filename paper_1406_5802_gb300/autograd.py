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


class RmgeSolveUniform(torch.autograd.Function):
    """count systems of one order n in one autograd node: the multipliers' products M_i = A_i G_i and the
    GENP factorizations run as uniform batches (one launch per kernel and step for all systems,
    rmge_apply_multiplier_batched / rmge_factor_batched), and so do the triangular solves, X_i = G_i Y_i,
    the refinement and the adjoint (rmge_solve_uniform_batched, rmge_refine_uniform_batched,
    rmge_solve_backward_uniform_batched)."""

    @staticmethod
    def forward(ctx, A, B, seeds, prec, max_iters, be_tol, streams, digits=(7, 7)):
        count, n, _ = A.shape
        A64 = A.detach().to(torch.float64).contiguous()
        B64 = B.detach().to(torch.float64).contiguous()
        G = torch.empty(count, n, n, dtype=torch.float64, device=A.device)
        for i, s in enumerate(seeds):
            rmge.make_multiplier("gaussian", n, int(s), 1, prec, G=G[i])
        ws = rmge.uniform_workspace(count, n, prec)
        opts = rmge.options(apply_digits=digits[0], factor_digits=digits[1])
        M = rmge.apply_multiplier_batched(A64, G, prec, opts=opts, ws=ws)
        info, _ = rmge.factor_batched(M, prec, ws=ws, opts=opts)
        del ws
        # the solves and sweeps with FP64 factors are uniform batches too: one launch per kernel for all
        # systems, each system stopping its refinement on its own test
        ws = rmge.uniform_solve_workspace(count, n, B64.shape[2], prec)
        X = rmge.solve_uniform_batched(M, G, B64, prec, ws=ws)
        rmge.refine_uniform_batched(A64, M, G, B64, X, prec, max_iters, be_tol, ws=ws)
        ctx.save_for_backward(M, G, X, A64)
        ctx.prec, ctx.max_iters, ctx.be_tol, ctx.streams, ctx.info = prec, max_iters, be_tol, streams, info
        return X.to(B.dtype)

    @staticmethod
    def backward(ctx, dX):
        M, G, X, A64 = ctx.saved_tensors
        count, n, _ = M.shape
        dX64 = dX.detach().to(torch.float64).contiguous()
        dB, dA, _, _ = rmge.solve_backward_uniform_batched(A64, M, G, X, dX64, ctx.prec,
                                                           want_dA=ctx.needs_input_grad[0],
                                                           max_iters=ctx.max_iters, be_tol=ctx.be_tol)
        gA = dA.to(dX.dtype) if dA is not None else None
        gB = dB.to(dX.dtype) if ctx.needs_input_grad[1] else None
        return gA, gB, None, None, None, None, None, None


def rmge_solve_batched(As, Bs, seeds, kind: str = "gaussian", prec: str = "f32", streams: int = 8, **kw):
    """A list of independent differentiable solves.  Systems of one order with the emulated-FP64 precision
    ("f64x") and dense Gaussian multipliers go through the uniform batched path (one autograd node;
    products, factorizations, solves, refinement and adjoint batched; digits=(apply, factor) sets the
    balanced base-256 digits of the emulated products, default (7, 7)); otherwise each solve is its own
    node and the solves are spread round-robin over CUDA streams so that small systems overlap on the GPU.
    Returns the list of X."""
    if (prec == "f64x" and kind == "gaussian" and len(As) > 1 and len({tuple(a.shape) for a in As}) == 1
            and len({tuple(b.shape) for b in Bs}) == 1):
        X = RmgeSolveUniform.apply(torch.stack(As), torch.stack(Bs), list(seeds), prec, kw.get("max_iters", 10),
                                   kw.get("be_tol", 1e-13), streams, tuple(kw.get("digits", (7, 7))))
        return list(X.unbind(0))
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
