"""torch.autograd face of the library's reverse pass (md_forward / md_backward).

`ensemble_run(eps, sigma, spec)` runs a differentiable velocity-Verlet
trajectory of every replica (all in one handle) and returns the final
(U, K, W) per replica as an (R, 3) tensor together with the final positions
and velocities ((3, N) tensors on the device of spec['x']).  Its backward
calls md_backward: d(loss)/d(eps, sigma) per replica comes from the library's
FP64 adjoint, not from autograd through the steps, for a loss on the final
energies, on the final state itself, or on both.  `ensemble_euw` is the same
run returning (U, K, W) only.  Argument marshalling only.
"""
import numpy as np
import torch

from . import md


class _Run(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, sigma, spec):
        ctx.set_materialize_grads(False)
        h = md.md_create(spec["sizes"], spec["box"], eps=eps.detach().cpu().numpy(),
                         sigma=sigma.detach().cpu().numpy(), rc_over_sigma=spec.get("rc_over_sigma", 2.5),
                         skin=spec.get("skin", 0.3), dt=spec.get("dt", 0.005),
                         precision=spec.get("precision", md.MD_FP32_FIXED))
        md.md_set_state(h, spec["x"], spec["v"])
        md.md_build_neighbors(h)
        euw = torch.zeros(len(spec["sizes"]), 3, dtype=torch.float64)
        md.md_forward(h, spec["nsteps"], spec.get("ckpt_every", 20), euw)
        xT = torch.empty_like(spec["x"])
        vT = torch.empty_like(spec["v"])
        md.md_get_state(h, xT, vT)
        ctx.h = h
        ctx.R = len(spec["sizes"])
        return euw, xT, vT

    @staticmethod
    def backward(ctx, g_euw, g_x, g_v):
        R = ctx.R
        ge = torch.zeros(R, dtype=torch.float64)
        gs = torch.zeros(R, dtype=torch.float64)
        gw = None if g_euw is None else g_euw.detach().to(torch.float64).contiguous().cpu()
        gx = None if g_x is None else g_x.detach().to(torch.float64).contiguous()
        gv = None if g_v is None else g_v.detach().to(torch.float64).contiguous()
        md.md_backward(ctx.h, gx, gv, gw, ge, gs)
        ctx.h.destroy()
        return ge, gs, None


def ensemble_run(eps, sigma, spec):
    """((U, K, W) per replica, x_T, v_T) after spec['nsteps'] steps,
    differentiable in eps, sigma.

    spec: sizes (per replica), box ((R, 3) array), x, v ((3, N) float64 device
    tensors, replicas concatenated), nsteps, ckpt_every, and optionally
    rc_over_sigma, skin, dt, precision."""
    return _Run.apply(eps, sigma, spec)


def ensemble_euw(eps, sigma, spec):
    """(U, K, W) per replica after spec['nsteps'] steps, differentiable in eps, sigma."""
    return _Run.apply(eps, sigma, spec)[0]


def mean_energy_plus_pressure(euw, sizes, boxes):
    """Loss per replica U/N + (2K + W) / (3V): the mean potential energy plus the
    virial pressure of the final state."""
    n = torch.as_tensor(np.asarray(sizes, dtype=np.float64))
    vol = torch.as_tensor(np.prod(np.asarray(boxes, dtype=np.float64), axis=1))
    return euw[:, 0] / n + (2.0 * euw[:, 1] + euw[:, 2]) / (3.0 * vol)
