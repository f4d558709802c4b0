"""torch.autograd binding of the batched target log-density.

``TargetLogProb.apply(x, target)`` returns log p(x_c) for every chain row of
x [C, D]; its backward calls the library's hand-written adjoint
(``hmc_target_vjp``), which recomputes the forward pass instead of storing
anything from it.  Both directions run in libhmc's kernels.
"""
import torch

from . import hmc


class Target:
    """A target family bound to device tensors (kept alive here)."""

    def __init__(self, kind, dim, P=None, X=None, y=None):
        dev = lambda a: None if a is None else torch.as_tensor(a).cuda().contiguous()
        self.P, self.X, self.y = dev(P), dev(X), dev(y)
        self.dim = int(dim)
        self.c = hmc.make_target(kind, dim, self.P, self.X, self.y)

    def workspace(self, nbytes):
        return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device="cuda")


class TargetLogProb(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, target):
        x = x.contiguous()
        C = x.shape[0]
        nbytes = hmc.hmc_grad_workspace_bytes(target.c, C)
        ws = target.workspace(nbytes)
        lp = torch.empty(C, dtype=torch.float32, device=x.device)
        g = torch.empty_like(x)
        hmc.hmc_target_log_prob_and_grad(target.c, C, x, lp, g, ws, nbytes)
        ctx.save_for_backward(x)
        ctx.target = target
        return lp

    @staticmethod
    def backward(ctx, grad_lp):
        (x,) = ctx.saved_tensors
        target = ctx.target
        C = x.shape[0]
        nbytes = hmc.hmc_target_vjp_workspace_bytes(target.c, C)
        ws = target.workspace(nbytes)
        dx = torch.empty_like(x)
        w = grad_lp.to(torch.float32).contiguous()
        hmc.hmc_target_vjp(target.c, C, x, w, dx, ws, nbytes)
        return dx, None


def log_prob(x, target):
    return TargetLogProb.apply(x, target)
