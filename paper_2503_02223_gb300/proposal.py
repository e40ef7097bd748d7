"""Learned quadric proposal: labels, training loop and proposals through the library.

The network (dqo_mlp_*) maps up to 8 views of a quadric (box + camera, 128 features) to its
canonical parameters.  Training pairs come from the plain multi-view fit (Eq. 1
initialisation + Eq. 12 refinement over all of a quadric's views, dqo_quadric_fit) in
canonical form (dqo_quadric_canonical); each epoch the network sees a random number of
each quadric's views (2..8), so it learns to propose from few views what the full fit
finds.  The proposal then starts dqo_quadric_fit's refinement.  This module only
orchestrates library calls: features, products, the optimiser and the fit all run in the
library's kernels.
"""
from __future__ import annotations

import torch

from . import dqo

FIT_ITERS = 100
FIT_LR = 1e-2


def fit(ctx, d: dict, iters: int = FIT_ITERS, start=None, stream=None) -> dict:
    """Plain fit (start=None) or refinement from `start` of every quadric in a CSR set."""
    nq = d["q_ptr"].shape[0] - 1
    dev = d["q_ptr"].device
    out = dict(init=torch.zeros(nq, 9, device=dev), params=torch.zeros(nq, 9, device=dev),
               loss=torch.zeros(nq, device=dev), ok=torch.zeros(nq, dtype=torch.uint8, device=dev))
    dqo.dqo_quadric_fit(ctx, d["P"], d["q_ptr"], d["pair_v"], d["obs_bbox"], iters, FIT_LR, out["init"],
                        out["params"], out["loss"], out["ok"], stream, start=start)
    return out


def make_labels(ctx, d: dict) -> tuple[torch.Tensor, torch.Tensor]:
    """Canonical parameters of the plain fit over all views, and its ok flags."""
    f = fit(ctx, d)
    return dqo.dqo_quadric_canonical(f["params"]), f["ok"]


def features(d: dict, counts: torch.Tensor | None, X=None, XT=None, length_scale: float = 1.0):
    return dqo.dqo_mlp_features(d["P"], d["q_ptr"], d["pair_v"], d["obs_bbox"], counts, length_scale, X, XT)


class Trainer:
    """Adam training of the proposal network on a fixed sample set: per epoch, the features
    for freshly drawn view counts (one launch) and every batch's step (one launch of
    `dqo_mlp_train_steps`)."""

    def __init__(self, ctx, state: dqo.MlpState, d: dict, labels: torch.Tensor, batch: int = 4096,
                 epochs: int = 30, seed: int = 0, length_scale: float = 1.0, min_views: int = 2,
                 max_views: int = 8, **hp):
        n = labels.shape[0] // batch * batch
        if n == 0:
            raise ValueError("fewer samples than one batch")
        self.ctx, self.state, self.d, self.batch, self.n = ctx, state, d, batch, n
        self.labels = labels
        self.gen = torch.Generator(device=labels.device)   # view counts are drawn on the device
        self.gen.manual_seed(seed)
        self.min_views, self.max_views = min_views, max_views
        dev = labels.device
        nq = d["q_ptr"].shape[0] - 1
        self.nq = nq
        self.X = torch.empty(nq, dqo.MLP_FEATURES, dtype=torch.bfloat16, device=dev)
        self.counts = torch.empty(nq, dtype=torch.int32, device=dev)
        self.steps = n // batch
        self.loss = torch.zeros(self.steps, device=dev)
        self.hp = dqo.mlp_hparams(total_steps=epochs * self.steps, **hp)
        self.length_scale = length_scale

    def epoch_async(self) -> torch.Tensor:
        """One pass over the samples with freshly drawn view counts, without waiting for it;
        returns the mean batch loss as a device scalar."""
        torch.randint(self.min_views, self.max_views + 1, (self.nq,), generator=self.gen, device=self.counts.device,
                      dtype=torch.int32, out=self.counts)
        features(self.d, self.counts, self.X, None, self.length_scale)
        dqo.dqo_mlp_train_steps(self.ctx, self.state, self.hp, self.X[:self.n], self.labels[:self.n], self.batch,
                                self.loss)
        return self.loss.mean()

    def epoch(self) -> float:
        """One pass over the samples with freshly drawn view counts; returns the mean batch loss."""
        return float(self.epoch_async().item())


def propose(ctx, state: dqo.MlpState, d: dict, counts: torch.Tensor | None = None, length_scale: float = 1.0):
    """Network proposal [nq, 9] (canonical parameters) from each quadric's first views."""
    X = features(d, counts, length_scale=length_scale)
    return dqo.dqo_mlp_forward(ctx, state, X)
