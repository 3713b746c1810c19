"""Host-side driver of the learned sampling proposal: gathers training rays
(features and 512-sample opacity profiles) through the C-ABI, runs the
library's training step over shuffled batches, and returns the loss curve.
Orchestration only: features, profiles, the network, its gradient and the
Adam update all run in the library's kernels.
"""
from __future__ import annotations

import math

import torch

from . import (RC_PROPOSAL_FEATURES, RC_PROPOSAL_OUTPUTS, rc_camera_set, rc_profiles_generate,
               rc_proposal_features, rc_proposal_train_step)


def collect_rays(ctx, vol, cameras, params, rays_per_view, seed):
    """Features and profile targets of rays_per_view random rays (among those
    that hit the volume box) of every camera."""
    gen = torch.Generator().manual_seed(seed)
    feats, targets = [], []
    for cam in cameras:
        rc_camera_set(ctx, cam)
        n = cam["width"] * cam["height"]
        F = torch.empty((n, RC_PROPOSAL_FEATURES), device="cuda", dtype=torch.float32)
        Y = torch.empty((n, RC_PROPOSAL_OUTPUTS), device="cuda", dtype=torch.float32)
        rc_proposal_features(ctx, vol, params, F)
        rc_profiles_generate(ctx, vol, params, Y)
        hit = torch.nonzero(F[:, 3:6].abs().sum(dim=1) > 0).squeeze(1)
        k = min(rays_per_view, hit.numel())
        pick = hit[torch.randperm(hit.numel(), generator=gen)[:k].to(hit.device)]
        feats.append(F[pick])
        targets.append(Y[pick])
    return torch.cat(feats), torch.cat(targets)


def train(ctx, feat, target, epochs=20, batch=8192, lr=2e-3, lr_final=1e-4, seed=0):
    """Shuffled mini-batch Adam with a cosine learning-rate decay; returns the
    mean loss of every epoch."""
    n = feat.shape[0]
    gen = torch.Generator().manual_seed(seed)
    steps_per_epoch = math.ceil(n / batch)
    total = epochs * steps_per_epoch
    loss = torch.zeros(1, device="cuda")
    acc = torch.zeros(1, device="cuda")
    curve = []
    step = 0
    for _ in range(epochs):
        perm = torch.randperm(n, generator=gen).to("cuda")
        acc.zero_()
        for b in range(0, n, batch):
            idx = perm[b:b + batch]
            f = feat[idx].contiguous()
            t = target[idx].contiguous()
            cur = lr_final + 0.5 * (lr - lr_final) * (1 + math.cos(math.pi * step / max(1, total - 1)))
            rc_proposal_train_step(ctx, f, t, idx.numel(), cur, loss)
            acc += loss * idx.numel()
            step += 1
        curve.append(float(acc.item()) / n)
    return curve
