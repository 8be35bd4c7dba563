"""torch.autograd wrapper of the certified solve: the anchored scaled rotations G_i = s_i R_i
(Sec. 2.2 rounding, R_0 = I, s_0 = 1) as a differentiable function of the lifted keypoints
u_e and the weights w_e.  Forward is xm_build_Q + xm_solve; backward is xm_backward, the
implicit adjoint of the certified optimum (gradients are those of the exact optimum of Eq. 17,
valid where the relaxation is tight and the optimum unique up to gauge)."""
from __future__ import annotations

import torch

from . import xm


class XMSolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, ukp, w, cam, lmk, N: int, M: int, context, opts, backward_opts):
        q = xm.xm_build_Q(context, N, M, cam, lmk, ukp.detach().contiguous(), w.detach().contiguous())
        out = xm.xm_solve(q, opts, allow_notcert=False)
        fctx.q, fctx.Y, fctx.rank = q, out["Y"], int(out["info"]["rank"])
        fctx.N, fctx.M, fctx.opts = N, M, backward_opts or opts
        fctx.info = out["info"]
        fctx.save_for_backward(ukp.detach(), w.detach(), cam, lmk)
        return out["G"]

    @staticmethod
    def backward(fctx, dG):
        ukp, w, cam, lmk = fctx.saved_tensors
        d_u, d_w, _, info, _ = xm.xm_backward(fctx.q, fctx.Y, fctx.rank, fctx.M, cam, lmk, ukp, w,
                                              dG.contiguous().to(torch.float64), fctx.opts)
        fctx.adj_info = info
        fctx.q.free()
        return d_u, d_w, None, None, None, None, None, None, None


def xm_solve_G(ukp, w, cam, lmk, N: int, M: int, context, opts=None, backward_opts=None):
    """G (N x 3 x 3) of the certified solve; differentiable in ukp (E x 3) and w (E), float64
    CUDA tensors.  Raises XmError if the solve is not certified."""
    opts = opts or xm.xm_default_opts()
    return XMSolve.apply(ukp, w, cam, lmk, N, M, context, opts, backward_opts)
