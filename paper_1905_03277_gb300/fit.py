"""Fitting the merge's tuning parameters (and the motion) by gradient descent.

The loss is the mean squared error between the merged RGB and a ground-truth image of
the base frame.  Gradients come from the hand-written adjoint (hmfsr_merge_backward via
MergeFn); PyTorch's Adam only updates the tensors.  The eight parameters are positive, so
they are optimised as logarithms.
"""
from __future__ import annotations

import math

import torch

from . import AlignParams, MergeFn, MergeParams, PARAM_NAMES, align


def fit(bursts, gts, base: MergeParams | None = None, steps: int = 200, lr: float = 0.02, motion_lr: float = 0.005,
        fit_motion: bool = True, scale=(3, 2), motions=None, log_every: int = 0):
    """Fit the eight tuning parameters (PARAM_NAMES) shared by all `bursts` (torch.uint16
    [n, H, W] on the device) to their ground truths `gts` (float32 [3, Ho, Wo], DN).

    Returns (params as a MergeParams, list of per-step mean losses, fitted motions)."""
    base = base or MergeParams()
    dev = bursts[0].device
    if motions is None:
        motions = [align(b, 0, AlignParams(tile=base.tile)) for b in bursts]
    motions = [m.detach().clone().requires_grad_(fit_motion) for m in motions]
    phi = torch.tensor([math.log(getattr(base, k)) for k in PARAM_NAMES], dtype=torch.float64, device=dev,
                       requires_grad=True)
    groups = [{"params": [phi], "lr": lr}]
    if fit_motion:
        groups.append({"params": motions, "lr": motion_lr})
    opt = torch.optim.Adam(groups)
    history = []
    for step in range(steps):
        opt.zero_grad()
        # One host read of the parameters and one of the loss per step: the bursts' forward
        # and adjoint launches queue back to back without a synchronisation between them.
        theta = torch.exp(phi).float()
        vals = theta.detach().cpu().tolist()
        total = torch.zeros((), dtype=torch.float64, device=dev)
        for b, g, m in zip(bursts, gts, motions):
            rgb = MergeFn.apply(theta, m, b, base, scale, 0, vals)
            loss = ((rgb - g) ** 2).mean() / len(bursts)
            loss.backward(retain_graph=True)
            total += loss.detach()
        history.append(float(total))
        opt.step()
        if log_every and step % log_every == 0:
            print(f"step {step}: loss {total:.4f}")
    vals = torch.exp(phi).detach().cpu().tolist()
    return MergeParams(**{**base.__dict__, **dict(zip(PARAM_NAMES, vals))}), history, [m.detach() for m in motions]
