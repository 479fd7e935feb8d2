"""torch.autograd.Function around the refinement objective (Sec. V).

Forward: J(xi) of Eq. (19) for B twists about B base poses, evaluated by the
distance kernel (dock_objective_fwd).  Backward: the adjoint kernel
(dock_objective_bwd) recomputes the contact sensitivities of Eq. (24)-(28)
and returns gJ * grad J.  Tensors stay on the device; the calls are issued on
torch's current stream.
"""
import numpy as np
import torch

from . import dock


class DockObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xi, handle, obj, sw, base_poses, params):
        if not xi.is_cuda:
            raise ValueError("xi must be a CUDA tensor")
        xi_c = xi.detach().to(torch.float32).contiguous()
        B = xi_c.shape[0]
        J = torch.empty(B, dtype=torch.float32, device=xi.device)
        stream = torch.cuda.current_stream(xi.device).cuda_stream
        handle.objective_fwd(obj, sw, base_poses, xi_c.data_ptr(), B, J.data_ptr(), 0, stream, params)
        ctx.save_for_backward(xi_c)
        ctx.handle, ctx.obj, ctx.sw, ctx.base, ctx.params = handle, obj, sw, np.asarray(base_poses), params
        return J

    @staticmethod
    def backward(ctx, gJ):
        (xi_c,) = ctx.saved_tensors
        B = xi_c.shape[0]
        g = gJ.detach().to(torch.float32).contiguous()
        gxi = torch.empty_like(xi_c)
        stream = torch.cuda.current_stream(xi_c.device).cuda_stream
        ctx.handle.objective_bwd(ctx.obj, ctx.sw, ctx.base, xi_c.data_ptr(), B, g.data_ptr(), gxi.data_ptr(), stream,
                                 ctx.params)
        return gxi, None, None, None, None, None


def objective(xi, handle, obj, sw, base_poses, params=None):
    """J(xi) (B,) for twists xi (B, 6) about base_poses (B, 7)."""
    return DockObjective.apply(xi, handle, obj, sw, base_poses, params)
