"""Differentiable collision steps: torch.autograd.Function over the fused step with a hand-written adjoint.

The gradient is pathwise: the random stream and every discrete decision of each step (pairs, accept tests, weight
order, energy-correction passes and crossing pairs) are held fixed, and the chain rule runs backwards through the
smooth rest of each interaction in the CUDA kernel behind ``mcc_adjoint``. Gradients flow to the initial velocities,
the weights and the Coulomb logarithms (the upper-triangle entries lnL[a, b], a <= b, that the interactions use).

Checkpointing: the forward keeps the state at every ``checkpoint_every``-th step; the backward replays each segment
from its checkpoint (one interaction at a time, storing the state before every interaction of the segment), then
walks the segment backwards. Memory: checkpoint_every x interactions states of the segment, plus the checkpoints.

Recorded tapes (float64, ``tape=True``, or ``tape=None`` when the tapes fit in half the free device memory): the
forward runs every interaction through ``mcc_adjoint`` in recording mode, which keeps each cell's tape in device
memory (about 250 bytes per particle per interaction plus the energy-pair reserve), and the backward is the reverse
sweep alone, interaction by interaction from the last, with nothing recomputed. This trades memory for the
backward's two recomputations of the forward (the replay and the recomputation inside each reverse call).

Two variants, chosen by the velocity dtype: float64 runs the FP64 step forward; float32 runs the mixed-precision step
forward (float velocities, float-float sums) and, in the backward, replays each segment in FP64 from its float
checkpoint and takes the FP64 adjoint there, returning float32 velocity gradients. The FP32 variant's gradient is the
FP64 gradient at a trajectory within float rounding of the one its forward took.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import _binding as B


class _CollisionSteps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vx, vy, vz, w, lnL, cfg):
        v = [vx.detach().clone(), vy.detach().clone(), vz.detach().clone()]
        ctx.vdtype = vx.dtype
        L = lnL.detach().cpu().numpy()
        ctx.tapes = None
        if cfg["tape"]:
            # every interaction through the adjoint kernel, recording its tape
            common = (cfg["offsets"], cfg["n_cells"], cfg["S"], cfg["species"], L)
            tapes = []
            for t in range(cfg["n_steps"]):
                p = dataclasses.replace(cfg["params"], step=cfg["params"].step + t)
                for k, (a, b) in enumerate(cfg["inter"]):
                    buf = torch.empty(cfg["tape_bytes"], dtype=torch.uint8, device=vx.device)
                    out = [torch.empty_like(x) for x in v]
                    B.mcc_adjoint(*v, w.detach(), *common, a, b, k, p, cfg["max_cell"], out=out,
                                  tape=B.ADJOINT_RECORD, tape_buffer=buf)
                    tapes.append((k, a, b, p, buf))
                    v = out
            B.sync_status(vx.device)
            ctx.save_for_backward(w, lnL)
            ctx.tapes = tapes
            ctx.ckpts = []
            ctx.cfg = cfg
            return v[0], v[1], v[2]
        ckpts = []
        for t in range(cfg["n_steps"]):
            if t % cfg["every"] == 0:
                ckpts.append([x.clone() for x in v])
            p = dataclasses.replace(cfg["params"], step=cfg["params"].step + t)
            B.mcc_step_fused(*v, w.detach(), cfg["offsets"], cfg["n_cells"], cfg["S"], cfg["species"], L, p,
                             n_steps=1, max_cell=cfg["max_cell"], interactions=cfg["inter"])
        B.sync_status(vx.device)
        ctx.save_for_backward(w, lnL)
        ctx.ckpts = ckpts
        ctx.cfg = cfg
        return v[0], v[1], v[2]

    @staticmethod
    def backward(ctx, gx, gy, gz):
        w, lnL = ctx.saved_tensors
        cfg = ctx.cfg
        w = w.detach()
        L = lnL.detach().cpu().numpy()
        dev = w.device
        g = [(x if x is not None else torch.zeros_like(w)).detach().to(torch.float64).contiguous().clone()
             for x in (gx, gy, gz)]
        gw = torch.zeros_like(w)
        inter = cfg["inter"]
        glnl = torch.zeros(len(inter), dtype=torch.float64, device=dev)
        every, n_steps = cfg["every"], cfg["n_steps"]
        common = (cfg["offsets"], cfg["n_cells"], cfg["S"], cfg["species"], L)
        if ctx.tapes is not None:
            # the reverse sweep alone, from the recorded tapes (the velocities passed are not read)
            for k, a, b, p, buf in reversed(ctx.tapes):
                B.mcc_adjoint(*g, w, *common, a, b, k, p, cfg["max_cell"], grad=g, gw=gw, glnL=glnl[k:k + 1],
                              tape=B.ADJOINT_REPLAY, tape_buffer=buf)
            ctx.tapes = None
        for seg in reversed(range(len(ctx.ckpts))):
            t0, t1 = seg * every, min(seg * every + every, n_steps)
            v = [x.to(torch.float64) for x in ctx.ckpts[seg]]
            tape = []
            for t in range(t0, t1):
                p = dataclasses.replace(cfg["params"], step=cfg["params"].step + t)
                for k, (a, b) in enumerate(inter):
                    out = [torch.empty_like(x) for x in v]
                    B.mcc_adjoint(*v, w, *common, a, b, k, p, cfg["max_cell"], out=out)
                    tape.append((k, a, b, p, v))
                    v = out
            for k, a, b, p, vb in reversed(tape):
                B.mcc_adjoint(*vb, w, *common, a, b, k, p, cfg["max_cell"], grad=g, gw=gw, glnL=glnl[k:k + 1])
        B.sync_status(dev)
        gL = torch.zeros(lnL.shape, dtype=torch.float64)
        gl = glnl.cpu()
        for k, (a, b) in enumerate(inter):
            gL[a, b] += gl[k]
        gv = [x.to(ctx.vdtype) for x in g]
        return gv[0], gv[1], gv[2], gw, gL.to(lnL.device, lnL.dtype), None


def collision_steps(vx, vy, vz, w, lnL, offsets, n_cells: int, n_species: int, species, params: B.Params,
                    n_steps: int, max_cell: int | None = None, checkpoint_every: int = 10, interactions=None,
                    tape: bool | None = False):
    """n_steps collision steps (non-relativistic), differentiable with respect to vx, vy, vz, w (float64) and lnL (a
    float64 tensor of shape (S, S)). float64 velocities: the FP64 step; float32: the mixed-precision step with the
    FP64 adjoint replayed from float checkpoints. tape (float64 only): True records every interaction's tape in the
    forward so that the backward is the reverse sweep alone; None does so when the tapes take at most half the free
    device memory; False checkpoints every checkpoint_every steps. Returns the final (vx, vy, vz); the inputs are not
    modified."""
    if vx.dtype not in (torch.float64, torch.float32) or params.relativistic:
        raise ValueError("the differentiable step takes float64 or float32 velocities and is non-relativistic")
    if max_cell is None:
        max_cell = int((offsets[n_species::n_species] - offsets[:-1:n_species]).max().item()) if n_cells else 0
    inter = B.default_interactions(n_species) if interactions is None else [tuple(x) for x in interactions]
    if not torch.is_tensor(lnL):
        lnL = torch.as_tensor(np.broadcast_to(np.asarray(lnL, dtype=np.float64), (n_species, n_species)).copy())
    tape_bytes = 0
    if tape is None or tape:
        if vx.dtype != torch.float64:
            if tape:
                raise ValueError("recorded tapes take float64 velocities (the FP32 variant replays from checkpoints)")
        else:
            tape_bytes = B.adjoint_tape_bytes(vx.device, n_cells, max_cell, params.max_corr_passes)
            if tape is None:
                free, _ = torch.cuda.mem_get_info(vx.device)
                tape = tape_bytes * len(inter) * int(n_steps) <= free // 2
    cfg = dict(offsets=offsets, n_cells=int(n_cells), S=int(n_species), species=list(species), params=params,
               n_steps=int(n_steps), max_cell=int(max_cell), every=max(1, int(checkpoint_every)), inter=inter,
               tape=bool(tape) and vx.dtype == torch.float64, tape_bytes=tape_bytes)
    return _CollisionSteps.apply(vx, vy, vz, w, lnL, cfg)
