"""Differentiable PC-LSQR: a torch.autograd.Function around the C ABI.

Forward: x = argmin ||A x - b|| with the global (PPN gamma) column of A set
to `a_glob` (gsr_set_values + gsr_lsqr_solve).  Backward: one call to
gsr_lsq_backward, which solves the normal equations (A^T A) q = dL/dx in
FP64 on the GPU and returns dL/db = A q and dL/dA(i, G) = r_i q_G - s_i x_G
(r = b - A x, s = A q).  Gradients are exact for the least-squares solution;
the forward must therefore be run to convergence (tight atol/btol).
"""
from __future__ import annotations

import torch


class GsrSolve(torch.autograd.Function):
    """x = GsrSolve.apply(b, a_glob, solver, itmax, atol, btol, cg_iters, cg_tol)."""

    @staticmethod
    def forward(ctx, b, a_glob, solver, itmax=20000, atol=1e-14, btol=1e-14, cg_iters=2000,
                cg_tol=1e-13):
        if not (b.is_cuda and a_glob.is_cuda):
            raise ValueError("b and a_glob must be CUDA tensors")
        b = b.detach().contiguous().to(torch.float64)
        a_glob = a_glob.detach().contiguous().to(torch.float64)
        solver.set_values(23, a_glob)
        x, _, info = solver.lsqr_solve(b, itmax, atol, btol, want_se=False)
        ctx.solver = solver
        ctx.cg = (cg_iters, cg_tol)
        ctx.info = info
        ctx.save_for_backward(b, x)
        return x

    @staticmethod
    def backward(ctx, gx):
        b, x = ctx.saved_tensors
        gx = gx.contiguous().to(torch.float64)
        need_b, need_a = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
        gb, ga, _ = ctx.solver.lsq_backward(b, x, gx, max_iter=ctx.cg[0], tol=ctx.cg[1],
                                            want_glob=need_a)
        return (gb if need_b else None), (ga if need_a else None), None, None, None, None, None, None
