"""torch.autograd binding of the differentiable rollout.

`rollout(sim, E, nu, poses, x0, ...)` loads an initial particle state into a
`Sim` (either pipeline, one environment), runs len(poses) sub-steps with the
tools following the pose stream (mpm_tape_record) and returns the final
state.  Its backward is mpm_tape_backward: the hand-written reverse mode of
the sub-step on the GPU (on the fused pipeline, block by block in the
forward pass's sorted order), with the particle state checkpointed every
`checkpoint_every` sub-steps.
Gradients flow to E, nu (0-d tensors), poses ((K, n_tools, 6) float64) and the
initial state (x0, v0, F0, C0).  The paper does not differentiate its
simulator (Sec. V names it as future work); the derivative is that of the
branches the forward pass took (contact, approaching test, friction clamp,
closest tool, walls).
"""
from __future__ import annotations

import torch

from . import mpm as M


class _Rollout(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sim, particle_volume, checkpoint_every, E, nu, poses, x0, v0, F0, C0):
        dev = x0.device
        sim.set_env_material(0, float(E), float(nu), float(sim.cfg.rho))
        sim.load(x0.detach().float().contiguous(), particle_volume,
                 None if v0 is None else v0.detach().float().contiguous(),
                 None if F0 is None else F0.detach().float().contiguous(),
                 None if C0 is None else C0.detach().float().contiguous())
        sim.tape_record(poses.detach().cpu().double().numpy(), checkpoint_every)
        n = x0.shape[0]
        out = [torch.empty((n, c), dtype=torch.float32, device=dev) for c in (3, 3, 9, 9)]
        sim.read_device(*out)
        ctx.sim = sim
        ctx.meta = (E.dtype, E.device, nu.dtype, poses.dtype, poses.device)
        ctx.has = (v0 is not None, F0 is not None, C0 is not None)
        return tuple(out)

    @staticmethod
    def backward(ctx, gx, gv, gF, gC):
        sim = ctx.sim
        want = any(ctx.needs_input_grad[6:10])
        g = sim.tape_backward(gx, gv, gF, gC, want_state=want)
        Edt, Edev, nudt, pdt, pdev = ctx.meta
        dE = torch.tensor(g["E"], dtype=Edt, device=Edev)
        dnu = torch.tensor(g["nu"], dtype=nudt, device=Edev)
        dposes = torch.as_tensor(g["poses"], dtype=pdt).to(pdev)
        st = [g.get(k) for k in ("x", "v", "F", "C")]
        hv, hF, hC = ctx.has
        return (None, None, None, dE, dnu, dposes, st[0], st[1] if hv else None, st[2] if hF else None,
                st[3] if hC else None)


def rollout(sim: "M.Sim", E: torch.Tensor, nu: torch.Tensor, poses: torch.Tensor, x0: torch.Tensor,
            particle_volume: float, v0=None, F0=None, C0=None, checkpoint_every: int = 50):
    """Final (x, v, F, C) after len(poses) sub-steps from (x0, v0, F0, C0)
    (CUDA tensors; v0, C0 default to 0 and F0 to I), differentiable with
    respect to E, nu, poses and the initial state.  The tools start where
    the sim has them (place them with Sim.set_tool before the first call);
    poses[k, t] is tool t's pose at the end of sub-step k."""
    return _Rollout.apply(sim, float(particle_volume), int(checkpoint_every), E, nu, poses, x0, v0, F0, C0)
