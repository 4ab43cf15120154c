"""FP64 CPU oracle of adaptive density control.  TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may import or run this module; it shares no code with the CUDA path.

The paper (Sec. 4.2) densifies the Gaussian cloud during the optimisation with a gradient threshold of
5e-8 and takes every other setting from the R2-Gaussian method it builds on, whose values are not
given.  The readings implemented here (each a parameter of the library call):

* statistic: for every Gaussian, the sum over the projections rendered since the last densification
  of the norm of dL/dmu'_{b,n}, the gradient of the step's loss (mean over the batch's pixels of the
  squared residual) with respect to the Gaussian's deformed mean in projection b (Eq. 7), the deformed
  covariance held fixed; its mean over those projections is the quantity compared with the threshold
  (a Gaussian that projection b does not see contributes 0 for it);
* plan: a Gaussian is pruned if its density rho is below rho_min; otherwise it is densified if its
  mean gradient norm reaches the threshold -- split if its largest scale exceeds s_split, else cloned
  -- and kept unchanged otherwise.  The decision compares float32 values: grad_sum >= float32(tau *
  n_projections), max scale > float32(s_split), rho < float32(rho_min);
* clone: two copies with half the density each (line integrals add, so the total attenuation is
  unchanged);
* split: two children at mu + R diag(s) z_i (z_1, z_2 ~ N(0, I), drawn by the caller), scales s / 1.6,
  the same rotation, and density rho 1.6^3 / 2, so that the children's integrated mass
  rho (2 pi)^(3/2) s_1 s_2 s_3 adds up to the parent's;
* output order: the kept and new Gaussians in the order of their parents (a prefix sum of 0 / 1 / 2
  outputs per parent), the clone's original first; optimiser moments of new rows start at zero.

Pins: ``tests/test_oracle_density.py`` (the rules on hand-made cases, mass conservation, the split
children's positions, and the statistic against central finite differences of the loss).
"""
from __future__ import annotations

from typing import Dict, Sequence

import numpy as np
import torch

from oracle import digs_oracle as O

SPLIT_SHRINK = 1.6
PRUNE, KEEP, CLONE, SPLIT = -1, 0, 1, 2


def density_grad_sums(gauss: Dict, lattice: Dict, phi, w, views: Sequence[Dict], meas,
                      cutoff: float = 3.5) -> np.ndarray:
    """sum_b ||dL/dmu'_{b,n}|| per Gaussian for one batch (rows of w and views in batch order), with
    L = mean over every pixel of the batch of (I - M)^2 and the deformed covariances held fixed."""
    T = O._inputs(gauss, phi, w)
    M = O._t(meas)
    count = float(M.numel())
    with torch.no_grad():
        sigma0 = O.covariance(T["scale"], T["quat"])
        U, dU = O.ffd_eval(T["phi"], lattice, T["mu0"])
    out = torch.zeros(T["mu0"].shape[0], dtype=O.DT)
    for b, view in enumerate(views):
        v = O.view_tensors(view)
        with torch.no_grad():
            mu, sigma, K = O.deform(T["mu0"], sigma0, U, dU, T["w"][b])
            P = torch.linalg.inv(sigma)
            alive = O.alive_mask(v, mu, P, K, cutoff)
        mu_l = mu.clone().requires_grad_(True)
        img = O.render_view_bbox(v, mu_l, sigma, P, T["rho"], alive, cutoff)
        L = ((img.reshape(v["nv"], v["nu"]) - M[b]) ** 2).sum() / count
        L.backward()
        out += mu_l.grad.norm(dim=1)
    return out.numpy()


def densify_plan(grad_sum, n_projections: int, scale, rho, tau: float, s_split: float, rho_min: float):
    """(action [n] in PRUNE / KEEP / CLONE / SPLIT, first output row [n], number of output rows)."""
    g = np.asarray(grad_sum, dtype=np.float32)
    s = np.asarray(scale, dtype=np.float32)
    r = np.asarray(rho, dtype=np.float32)
    prune = r < np.float32(rho_min)
    dens = ~prune & (g >= np.float32(float(np.float32(tau)) * n_projections))  # tau as the library's float
    split = dens & (s.max(axis=1) > np.float32(s_split))
    action = np.where(prune, PRUNE, np.where(split, SPLIT, np.where(dens, CLONE, KEEP)))
    size = np.where(action == PRUNE, 0, np.where(action == KEEP, 1, 2))
    dst = np.concatenate([[0], np.cumsum(size)[:-1]]).astype(np.int64) if len(size) else np.zeros(0, np.int64)
    return action, dst, int(size.sum())


def densify_apply(gauss: Dict, action, dst, n_out: int, z) -> Dict[str, np.ndarray]:
    """The new cloud (mu0, scale, quat, rho), each output row's parent (src) and whether it is new."""
    mu0 = np.asarray(gauss["mu0"], np.float64)
    scale = np.asarray(gauss["scale"], np.float64)
    quat = np.asarray(gauss["quat"], np.float64)
    rho = np.asarray(gauss["rho"], np.float64)
    z = np.asarray(z, np.float64).reshape(len(mu0), 2, 3)
    out = dict(mu0=np.zeros((n_out, 3)), scale=np.zeros((n_out, 3)), quat=np.zeros((n_out, 4)),
               rho=np.zeros(n_out), src=np.zeros(n_out, np.int64), new=np.zeros(n_out, np.int64))
    R = O.quat_to_rotmat(torch.as_tensor(quat / np.linalg.norm(quat, axis=1, keepdims=True))).numpy()
    for n in range(len(mu0)):
        a, d = int(action[n]), int(dst[n])
        if a == PRUNE:
            continue
        rows = [d] if a == KEEP else [d, d + 1]
        for i, j in enumerate(rows):
            out["src"][j] = n
            out["quat"][j] = quat[n]
            if a == SPLIT:
                out["mu0"][j] = mu0[n] + R[n] @ (scale[n] * z[n, i])
                out["scale"][j] = scale[n] / SPLIT_SHRINK
                out["rho"][j] = rho[n] * SPLIT_SHRINK ** 3 / 2.0
                out["new"][j] = 1
            else:
                out["mu0"][j] = mu0[n]
                out["scale"][j] = scale[n]
                out["rho"][j] = rho[n] / 2.0 if a == CLONE else rho[n]
                out["new"][j] = 1 if (a == CLONE and i == 1) else 0
    return out


def gather_rows(src, new, rows) -> np.ndarray:
    """Per-Gaussian rows (e.g. optimiser moments) of the new cloud: the parent's row, zero for new rows."""
    rows = np.asarray(rows)
    out = rows[np.asarray(src)].copy()
    out[np.asarray(new).astype(bool)] = 0
    return out
