"""E_min as a differentiable function of (J, h) (Sec. III).

forward: tropical contraction keeping the traceback checkpoints (tn_forward).
backward: the argmax traceback kernel walks the contraction tree top-down,
recomputing intermediates that were not kept (tn_backward), and the gradient
kernel writes dE/dJ_e = -s_u s_v (Potts: -delta(s_u, s_v)) and dE/dh_i = -s_i
(tn_gradient) straight into device tensors.  The couplings are read from the
caller's CUDA tensors on the current torch stream.
"""
import torch

from . import binding as B


class TropicalEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, J, h, sg):
        if not J.is_cuda:
            raise RuntimeError("TropicalEnergy needs CUDA tensors (there is no CPU path)")
        J = J.detach().contiguous().float()
        hh = None if h is None else h.detach().contiguous().float()
        sg.set_stream(torch.cuda.current_stream(J.device).cuda_stream)
        sg.set_couplings(J, hh, on_device=True)
        E = B.tn_forward(sg.ctx)
        ctx.sg = sg
        ctx.has_h = h is not None
        ctx.device = J.device
        return torch.tensor(E, dtype=torch.float64, device=J.device)

    @staticmethod
    def backward(ctx, g):
        sg = ctx.sg
        B.tn_backward(sg.ctx, None)
        dJ = torch.empty(sg.m, dtype=torch.float32, device=ctx.device)
        dh = torch.empty(sg.n, dtype=torch.float32, device=ctx.device)
        B.tn_gradient(sg.ctx, sg.m, sg.n, dJ, dh)
        gf = g.to(torch.float32)
        return dJ * gf, (dh * gf if ctx.has_h else None), None
