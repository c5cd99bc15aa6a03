"""torch.autograd.Function over ptn_expval_grad: the trajectory-averaged
Pauli expectation F(theta) of a plan's trajectories as a differentiable
function of the rotation angles.  The forward call runs the forward and the
adjoint contractions together in the library (one ptn_expval_grad call) and
keeps dF/dtheta; backward scales it by the incoming gradient."""
import torch

from . import ptn


class TrajectoryExpval(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, plan, traj, terms):
        dev = torch.device("cuda", torch.cuda.current_device())
        th = theta.detach().to("cpu", torch.float64).contiguous()
        value = torch.empty(1, dtype=torch.float64, device=dev)
        grad = torch.empty(max(th.numel(), 1), dtype=torch.float64, device=dev)
        ptn.ptn_expval_grad(plan, traj, terms, th.numpy(), value, grad)
        ctx.save_for_backward(grad[: th.numel()])
        ctx.theta_meta = (theta.device, theta.dtype)
        return value[0].to(theta.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        (grad,) = ctx.saved_tensors
        device, dtype = ctx.theta_meta
        g = grad.to(device) * grad_out.to(device, torch.float64)
        return g.to(dtype), None, None, None


def trajectory_expval(theta, plan, traj, terms):
    """F(theta) = sum_i c_i <psi_i| O |psi_i> / sum_i c_i for O = sum_t a_t Z^{z_t}
    (terms: list of (a_t, z_mask_t)); differentiable in theta."""
    return TrajectoryExpval.apply(theta, plan, traj, terms)
