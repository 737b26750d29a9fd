"""torch.autograd wrapper of the unrolled Frank-Wolfe solver (marshalling only).

FrankWolfeQP.apply(unaries, weights, y0, lattices, iters) returns y^T of
dcrf_qp_fw; its backward calls dcrf_qp_fw_backward, which recomputes the
forward with per-iteration checkpoints of y and s and runs the reverse sweep
in the library's kernels.  Gradients flow to the unaries [N, L], the kernel
weights [n_kernels] and y0.
"""
import torch

from . import _abi


class FrankWolfeQP(torch.autograd.Function):
    @staticmethod
    def forward(ctx, unaries, weights, y0, lattices, iters, compat=None):
        w = [float(v) for v in weights.detach().cpu().tolist()]
        Y = y0.detach().contiguous().clone()
        _abi.dcrf_qp_fw(unaries.detach().contiguous(), lattices, w, Y, iters, compat=compat, records=False)
        ctx.save_for_backward(unaries.detach(), y0.detach())
        ctx.weights, ctx.lattices, ctx.iters, ctx.compat = w, lattices, iters, compat
        ctx.wdev, ctx.wdtype = weights.device, weights.dtype
        return Y

    @staticmethod
    def backward(ctx, grad_y):
        unaries, y0 = ctx.saved_tensors
        dphi, dw, dy0 = _abi.dcrf_qp_fw_backward(unaries.contiguous(), ctx.lattices, ctx.weights, y0.contiguous(),
                                                 grad_y.contiguous(), ctx.iters, compat=ctx.compat,
                                                 need_dy0=ctx.needs_input_grad[2])
        dwt = torch.tensor(dw, dtype=ctx.wdtype, device=ctx.wdev)
        return dphi, dwt, dy0, None, None, None
