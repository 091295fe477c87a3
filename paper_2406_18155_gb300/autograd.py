"""torch.autograd.Function over the library's fidelity + adjoint gradient.

forward(pulse, ham) sets the system's parameters (pulse amplitudes and
(E_J, E_C, E_L) per mode + coupling strengths, rad/ns, in the sg_get_params
order), prepares it and runs sg_fidelity_grad; backward scales the gradients the
solve already produced by the upstream gradient.  The solve runs in the CUDA
library; this class only moves arguments.
"""
import torch

_KIND = {"avg": 0, "state": 1}


class FidelityFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pulse, ham, system, T, dt, target, col_index, kind="avg", precision="mixed",
                ckpt=0):
        system.set_params(pulse=pulse.detach().cpu().double().numpy(),
                          ham=ham.detach().cpu().double().numpy())
        system.prepare()
        F, gp, gh = system.fidelity_grad(T, dt, target, col_index, kind=kind, precision=precision,
                                         ckpt=ckpt)
        ctx.save_for_backward(torch.as_tensor(gp, dtype=torch.float64),
                              torch.as_tensor(gh, dtype=torch.float64))
        ctx.devices = (pulse.device, ham.device)
        return torch.tensor(F[_KIND[kind]], dtype=torch.float64, device=pulse.device)

    @staticmethod
    def backward(ctx, gF):
        gp, gh = ctx.saved_tensors
        g = gF.detach().to("cpu", torch.float64)
        return ((g * gp).to(ctx.devices[0]), (g * gh).to(ctx.devices[1]),
                None, None, None, None, None, None, None, None)


def fidelity(system, pulse, ham, T, dt, target, col_index, kind="avg", precision="mixed", ckpt=0):
    """F(pulse, ham) as a differentiable torch scalar."""
    return FidelityFn.apply(pulse, ham, system, T, dt, target, col_index, kind, precision, ckpt)
