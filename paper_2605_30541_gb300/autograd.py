"""torch.autograd binding of the solver: velocity -> shot gathers, with the
backward pass done by libsim's adjoint-state kernels.

For a cotangent c = dL/dg of the gathers, the vector-Jacobian product J^T c is
what sim_adjoint_vjp returns: the adjoint sweep driven by c itself (no
difference g - d is formed, so a cotangent far smaller than the gathers keeps
its precision); the forward states are recomputed from checkpoints."""
import numpy as np
import torch

from . import sim_adjoint_vjp, sim_forward, sim_set_model


class _Gathers(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vel, sim, wavelet, src, rec, ckpt_fp16):
        d = sim.desc
        src = np.ascontiguousarray(np.asarray(src, np.float64).reshape(-1, d.ndim))
        rec = np.ascontiguousarray(np.asarray(rec, np.float64).reshape(-1, d.ndim))
        vel_c = vel.detach().to(sim.dtype).contiguous()
        sim_set_model(sim.handle, vel_c)
        w = wavelet.detach().to(device=vel.device, dtype=sim.dtype).contiguous()
        g = torch.empty((src.shape[0], d.nt, rec.shape[0]), dtype=sim.dtype, device=vel.device)
        sim_forward(sim.handle, src.shape[0], w, src, rec.shape[0], rec, g)
        ctx.sim, ctx.src, ctx.rec, ctx.fp16 = sim, src, rec, ckpt_fp16
        ctx.save_for_backward(vel_c, w, g)
        return g

    @staticmethod
    def backward(ctx, cot):
        vel_c, w, g = ctx.saved_tensors
        sim = ctx.sim
        sim_set_model(sim.handle, vel_c)
        c = cot.to(g.dtype).contiguous()
        grad = torch.zeros_like(vel_c)
        sim_adjoint_vjp(sim.handle, ctx.src.shape[0], w, ctx.src, ctx.rec.shape[0], ctx.rec, c, None,
                        int(ctx.fp16), grad)
        return grad.to(vel_c.dtype), None, None, None, None, None


def gathers(vel, sim, wavelet, src, rec, ckpt_fp16=False):
    """Differentiable forward modelling: returns gathers [nshots, nt, nrec]."""
    return _Gathers.apply(vel, sim, wavelet, src, rec, ckpt_fp16)
