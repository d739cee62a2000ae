"""torch.autograd.Function over the C ABI: the Wiener estimate of the target
image after K accelerated passes (Algorithm 2, Sec. III-C-2; posterior mean,
Sec. II-A), differentiable with respect to x, a and R'.

Forward: rcscm_create (with checkpoints) + rcscm_setup + rcscm_iterate(K) +
rcscm_extract.  Backward: rcscm_backward, which recomputes the passes from the
checkpoints and runs the hand-written adjoint kernel.  Argument marshalling
only; every step runs in the library's CUDA kernels.  The initial variances
rh0, ru0 and lambda0 receive no gradient.
"""
from __future__ import annotations

import torch

from . import rcscm as R


class _WienerEstimate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, a, Rp, rh0, ru0, lambda0, n_iter, ckpt_stride, opts):
        prob = dict(x=x.detach().contiguous(), a=a.detach().contiguous(), Rp=Rp.detach().contiguous(),
                    rh0=rh0.detach().contiguous(), ru0=ru0.detach().contiguous())
        if lambda0 is not None:
            prob["lambda0"] = lambda0.detach().contiguous()
        s = R.Solver([prob], rule="accel", ckpt_stride=ckpt_stride, ckpt_max_iters=max(int(n_iter), 1), **opts)
        s.setup()
        s.iterate(int(n_iter))
        h = s.extract().view(x.shape)
        ctx.solver = s
        return h

    @staticmethod
    def backward(ctx, grad_h):
        s = ctx.solver
        ctx.solver = None
        gx, ga, gR = s.split_grads(*s.backward(grad_h.to(torch.complex64).contiguous().view(-1)))[0]
        torch.cuda.current_stream().synchronize()   # the context is freed next
        s.close()
        return gx, ga, gR, None, None, None, None, None, None


def wiener_estimate(x, a, Rp, rh0, ru0, n_iter: int, lambda0=None, ckpt_stride: int = 5, **opts):
    """h [I, J, M] (complex64) after n_iter passes from (rh0, ru0, lambda0).

    x complex64 [I, J, M], a complex128 [I, M], Rp complex128 [I, M, M], rh0 and
    ru0 float32 [I, J], lambda0 float64 [I] or None (smallest nonzero eigenvalue
    of R', held constant in the gradient), all CUDA tensors.  Gradients follow
    PyTorch's convention for complex tensors (dL/dRe + i dL/dIm)."""
    return _WienerEstimate.apply(x, a, Rp, rh0, ru0, lambda0, int(n_iter), int(ckpt_stride), dict(opts))
