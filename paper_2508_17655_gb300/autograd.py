"""torch.autograd.Function around gsb_relaxed_energy_grad: the relaxed energy
E = -1/2 x(t_W)^T J x(t_W) after a window of W steps, differentiable with
respect to the initial positions x0, the control strengths A (per replica)
and the time step dt, through the library's hand-written adjoint kernels.
torch supplies the device buffers and the stream; every step runs in libgsb."""
from __future__ import annotations

import torch

from . import gsb


class GsbRelaxedEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, A, dt, problem, variant, M, window, c, ckpt_every, precision):
        if not (x0.is_cuda and x0.dtype == torch.float32 and x0.is_contiguous()):
            raise ValueError("x0 must be a contiguous float32 CUDA tensor (R x N)")
        R = x0.shape[0]
        dev = x0.device
        E = torch.empty(R, dtype=torch.float64, device=dev)
        gx = torch.empty_like(x0)
        gA = torch.empty(R, dtype=torch.float64, device=dev)
        gdt = torch.empty(R, dtype=torch.float64, device=dev)
        A_host = A.detach().to("cpu", torch.float32).numpy() if A.dim() else float(A)
        stream = torch.cuda.current_stream(dev)
        problem.relaxed_energy_grad(variant, M, window, x0.data_ptr(), R, A_host, float(dt), c,
                                    E.data_ptr(), gx.data_ptr(), gA.data_ptr(), gdt.data_ptr(),
                                    ckpt_every=ckpt_every, precision=precision, stream=stream)
        ctx.save_for_backward(gx, gA, gdt)
        ctx.A_shape = A.shape
        ctx.A_device = A.device
        ctx.dt_device = dt.device if torch.is_tensor(dt) else None
        ctx.dt_shape = dt.shape if torch.is_tensor(dt) else None
        return E

    @staticmethod
    def backward(ctx, gE):
        gx, gA, gdt = ctx.saved_tensors
        gE = gE.to(torch.float64)
        grad_x0 = (gE[:, None] * gx.to(torch.float64)).to(torch.float32)
        grad_A = gE * gA
        if len(ctx.A_shape) == 0:
            grad_A = grad_A.sum()
        grad_A = grad_A.to(device=ctx.A_device, dtype=torch.float32)
        grad_dt = None
        if ctx.dt_shape is not None:
            grad_dt = (gE * gdt).sum().reshape(ctx.dt_shape).to(device=ctx.dt_device,
                                                                  dtype=torch.float32)
        return grad_x0, grad_A, grad_dt, None, None, None, None, None, None, None


def relaxed_energy(x0, A, dt, problem, variant="gbsb", M=2000, window=200, c=0.5, ckpt_every=20,
                   precision="fp32"):
    """E per replica; differentiable in x0 (R x N), A (R or scalar) and dt (scalar tensor).
    precision: "fp32" (the products as FP32 SGEMMs) or "bf16x3" (on the tensor cores,
    split bf16)."""
    return GsbRelaxedEnergy.apply(x0, A, dt, problem, variant, M, window, c, ckpt_every,
                                  precision)
