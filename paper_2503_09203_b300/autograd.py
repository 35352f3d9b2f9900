"""torch.autograd.Function over a T-step rollout of the batched UUV step.

Forward writes the added-mass and damping coefficients into the simulator
(M^-1 recomputed in FP64 on the GPU), runs one recorded mg_rollout from the
simulator's current state and returns per-step observations and rewards.
Backward calls mg_step_backward, the hand-written adjoint of the discrete map
(checkpoints every `ckpt_every` steps, segments recomputed on the GPU), and
returns gradients for the actions, the added mass and the damping.

The checkpoints live in the simulator, which holds one recording at a time.
Forward keeps the identity of the recording it made; backward refuses (raises)
when the simulator no longer holds that recording, for example after a second
forward on the same simulator, a step, a reset or a parameter change, instead
of differentiating another rollout.
"""
from __future__ import annotations

import torch

from . import binding as B


class RolloutFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sim: "B.Sim", actions, added_mass, d_lin, d_quad):
        T = actions.shape[0]
        stream = torch.cuda.current_stream()
        actions = actions.contiguous()
        B.mg_set_hydro(sim.handle, added_mass.contiguous(), d_lin.contiguous(), d_quad.contiguous(), stream)
        obs = torch.zeros(T, sim.n_slots, B.MG_OBS_DIM, device=actions.device)
        rew = torch.zeros(T, sim.n_slots, device=actions.device)
        B.mg_rollout(sim.handle, actions, T, obs, rew, True, stream)
        ctx.sim = sim
        ctx.rec_id = B.mg_recording(sim.handle)[1]
        ctx.save_for_backward(actions)
        return obs, rew

    @staticmethod
    def backward(ctx, g_obs, g_rew):
        (actions,) = ctx.saved_tensors
        sim = ctx.sim
        steps, rec_id = B.mg_recording(sim.handle)
        if rec_id != ctx.rec_id:
            raise RuntimeError("marinegym rollout backward: the simulator no longer holds this forward's "
                               "recording (a later forward, step, reset or parameter change replaced or "
                               "discarded it); run backward before reusing the simulator")
        T = actions.shape[0]
        stream = torch.cuda.current_stream()
        g_act = torch.zeros_like(actions)
        g_A = torch.zeros(sim.n_slots, 6, device=actions.device)
        g_D = torch.zeros(sim.n_slots, 12, device=actions.device)
        B.mg_step_backward(sim.handle, actions,
                           None if g_obs is None else g_obs.contiguous(),
                           None if g_rew is None else g_rew.contiguous(),
                           None, g_act, g_A, g_D, None, stream)
        return None, g_act, g_A, g_D[:, :6].contiguous(), g_D[:, 6:].contiguous()


def rollout(sim, actions, added_mass, d_lin, d_quad):
    """Differentiable rollout: returns (obs [T, n_slots, 13], reward [T, n_slots])."""
    return RolloutFn.apply(sim, actions, added_mass, d_lin, d_quad)
