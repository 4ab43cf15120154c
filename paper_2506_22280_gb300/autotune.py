"""Autotuner of the launch shape of ``digs_step``.

Three knobs change how the library's kernels cover the work, not what they compute (results agree to
rounding): the raster tile edge (8, 16 or 32 pixels: tile-list length against binning cost), the lanes
that share one (projection, Gaussian) pair in the backward raster (16 or 32, i.e. two Gaussians or one
per warp), and the projections per step (one launch per stage covers all of them).  Each candidate runs
a few steps on a fresh copy of the caller's reconstruction state, timed with CUDA events on the
launching stream, and the fastest in projections per second is kept.  Results may be cached in a JSON
file keyed by the problem's signature.
"""
from __future__ import annotations

import json
import os
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

import torch

Batch = Tuple[torch.Tensor, Sequence[int], Sequence[Dict]]


def _time_candidate(make_rec: Callable[[int, int], "object"], make_batch: Callable[[int, int], Batch], tile: int,
                    lanes: int, B: int, steps: int, warmup: int) -> float:
    """Projections per second of `steps` timed steps (after `warmup`) with this launch shape."""
    rec = make_rec(tile, lanes)
    for s in range(warmup):
        rec.step(*make_batch(B, s))
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for s in range(steps):
        M, ids, views = make_batch(B, warmup + s)
        ev[s][0].record()
        rec.step(M, ids, views)
        ev[s][1].record()
    torch.cuda.synchronize()
    if rec.status() != 0:
        return 0.0
    ms = sum(a.elapsed_time(b) for a, b in ev)
    del rec
    return steps * B / (ms / 1e3)


def tune(make_rec: Callable[[int, int], "object"], make_batch: Callable[[int, int], Batch],
         tiles: Iterable[int] = (8, 16, 32), lanes: Iterable[int] = (16, 32),
         batch_sizes: Iterable[int] = (16,), steps: int = 3, warmup: int = 1,
         cache: Optional[str] = None, key: Optional[str] = None) -> Dict:
    """Pick (tile, bwd_lanes, projections per step) for the caller's problem.

    make_rec(tile, lanes) returns a fresh Reconstruction on the problem's initial parameters;
    make_batch(B, s) returns step s's (measured projections, projection ids, views) with B projections.
    Tile and lanes are searched jointly at the first batch size, then the batch sizes at the best pair.
    Returns {"tile", "bwd_lanes", "batch", "proj_per_s", "trials": [...]}."""
    if cache and key and os.path.exists(cache):
        try:
            hit = json.load(open(cache)).get(key)
            if hit:
                return dict(hit, cached=True)
        except (OSError, ValueError):
            pass
    batch_sizes = list(batch_sizes)
    trials: List[Dict] = []
    best = None
    for t in tiles:
        for l in lanes:
            r = _time_candidate(make_rec, make_batch, t, l, batch_sizes[0], steps, warmup)
            trials.append(dict(tile=t, bwd_lanes=l, batch=batch_sizes[0], proj_per_s=r))
            if best is None or r > best["proj_per_s"]:
                best = trials[-1]
    for B in batch_sizes[1:]:
        r = _time_candidate(make_rec, make_batch, best["tile"], best["bwd_lanes"], B, steps, warmup)
        trials.append(dict(tile=best["tile"], bwd_lanes=best["bwd_lanes"], batch=B, proj_per_s=r))
        if r > best["proj_per_s"]:
            best = trials[-1]
    out = dict(best, trials=trials, cached=False)
    if cache and key:
        try:
            data = json.load(open(cache)) if os.path.exists(cache) else {}
        except (OSError, ValueError):
            data = {}
        data[key] = {k: v for k, v in out.items() if k != "cached"}
        os.makedirs(os.path.dirname(os.path.abspath(cache)), exist_ok=True)
        json.dump(data, open(cache, "w"), indent=1)
    return out
