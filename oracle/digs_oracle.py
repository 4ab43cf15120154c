"""FP64 CPU oracle for the DIGS hot path.  TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` may import or run this module.  It shares no code with the CUDA path: it is a plain,
slow, obviously checkable statement of what the path computes, in float64 PyTorch CPU ops, with
PyTorch autograd giving the gradient of the same definition.

What it follows (paper sections / equations):

* Sec. 3.1, Eq. 2 and the sentence after it: Gaussian kernels with covariance Sigma = R S S^T R^T,
  S diagonal (the scales), R the rotation of a quaternion (w, x, y, z) that is normalised first.
* Sec. 3.3, Eq. 9-11: D(x, t) = x + sum_r w_r u_r(x); u_r interpolated from the 4x4x4 control points
  around x with cubic B-spline weights (the uniform cubic basis of the cited FFD work), node indices
  floor(p) - 1 + l; K = I + sum_r w_r grad u_r.  grad is taken with respect to world coordinates, so each
  derivative carries 1 / spacing.  Control points outside the lattice read as zero.
* Sec. 3.2, Eq. 7-8: mu_t = D(mu_0, t), Sigma_t = K Sigma_0 K^T, density unchanged.
* Sec. 3.1, Eq. 4 and the X-ray transform F (Eq. 1, 3): the projection of a Gaussian is its line
  integral along each detector ray.  Along a ray x = o + s d (unit d) with m = o - mu and P = Sigma^-1,
  a = d^T P d, b = d^T P m, c = m^T P m, the integral over the whole line is
  rho sqrt(2 pi / a) exp(-E / 2) with E = c - b^2 / a (the squared Mahalanobis distance from the ray to mu).
  The paper's 2D-Gaussian approximation with the integration-bias factor equals this exactly for
  parallel rays; this oracle uses the exact integral for cone beams too.
* A pair (ray, Gaussian) contributes iff E <= cutoff^2 (cutoff 3.5 by default, inclusive).  Gaussians
  whose deformation folds (det K <= 1e-6) are dropped; for cone beams so are Gaussians whose mean is
  not in front of the source or whose cutoff ellipsoid contains the source.
* Sec. 4.2: L2 loss in projection space, read as the mean of squared residuals.
* Sec. 4.2: Adam on the reference Gaussians and the B-spline grids, with linearly decaying learning rates.

Geometry: pixel (i, j) of a view has centre det_c + (i - (nu-1)/2 + off_u) du e_u +
(j - (nv-1)/2 + off_v) dv e_v; a cone-beam ray runs from the source through that centre; a parallel
ray runs through it along the unit vector from src to det_c.  Projections are stored [P][nv][nu].

Two evaluation modes: ``brute`` sums every ray against every Gaussian; ``bbox`` only visits the pixels
inside the detector image of the axis-aligned box that holds each Gaussian's cutoff ellipsoid (half
extents cutoff * sqrt(Sigma_ii)).  Every ray with E <= cutoff^2 meets that box, so both modes select the
same pairs; the tests check this.

Parity pins: every function here is checked in ``tests/test_oracle_*.py`` against closed forms,
invariants, textbook special cases or brute force.  Where no pin exists the docstring says
"parity unpinned".
"""
from __future__ import annotations

import math
from typing import Dict, List, Optional, Sequence

import numpy as np
import torch

DT = torch.float64
FOLD_EPS = 1e-6


def _t(x) -> torch.Tensor:
    if isinstance(x, torch.Tensor):
        return x.to(DT)
    return torch.as_tensor(np.asarray(x), dtype=DT)


# ----------------------------------------------------------------------------- Sec. 3.1
def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of the quaternion (w, x, y, z), normalised first (Sec. 3.1: R parameterised
    by a quaternion)."""
    q = q / q.norm(dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    rows = [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
            2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
            2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]
    return torch.stack(rows, -1).reshape(q.shape[:-1] + (3, 3))


def covariance(scale: torch.Tensor, quat: torch.Tensor) -> torch.Tensor:
    """Sigma = R S S^T R^T with S = diag(scale) (Sec. 3.1, after Eq. 2)."""
    R = quat_to_rotmat(quat)
    return R @ torch.diag_embed(scale * scale) @ R.transpose(-1, -2)


# ----------------------------------------------------------------------------- Sec. 3.3
def bspline(u: torch.Tensor, deriv: int = 0) -> torch.Tensor:
    """Uniform cubic B-spline basis B_0..B_3 at local coordinate u in [0, 1) (Eq. 10; the basis of the
    cited FFD registration work), stacked on the last axis; ``deriv`` = 1 or 2 gives d/du, d2/du2."""
    if deriv == 0:
        return torch.stack([(1 - u) ** 3 / 6, (3 * u ** 3 - 6 * u ** 2 + 4) / 6,
                            (-3 * u ** 3 + 3 * u ** 2 + 3 * u + 1) / 6, u ** 3 / 6], -1)
    if deriv == 1:
        return torch.stack([-(1 - u) ** 2 / 2, (3 * u ** 2 - 4 * u) / 2,
                            (-3 * u ** 2 + 2 * u + 1) / 2, u ** 2 / 2], -1)
    if deriv == 2:
        return torch.stack([1 - u, 3 * u - 2, 1 - 3 * u, u], -1)
    raise ValueError(deriv)


def temporal_weights(ctrl, t_step: float, rows) -> torch.Tensor:
    """Weights w[rows][R] from temporal control points ctrl[n_ctrl][R] (Sec. 4.2: a cubic B-spline over
    the time axis, control points every t_step time points, with the basis of Eq. 10): projection p sits
    at tau = p / t_step + 1 control-point units; with f = floor(tau) - 1 and u = tau - floor(tau),
    w(p) = sum_l B_l(u) ctrl[f + l]; control points outside [0, n_ctrl) read as zero.  Differentiable in
    ctrl (torch input)."""
    c = ctrl if isinstance(ctrl, torch.Tensor) else torch.as_tensor(np.asarray(ctrl), dtype=DT)
    out = []
    for p in rows:
        tau = float(p) / float(t_step) + 1.0
        fl = math.floor(tau)
        B = bspline(torch.tensor(tau - fl, dtype=DT))
        acc = torch.zeros(c.shape[1], dtype=DT)
        for l in range(4):
            j = fl - 1 + l
            if 0 <= j < c.shape[0]:
                acc = acc + B[l] * c[j]
        out.append(acc)
    return torch.stack(out, 0)


def lattice_coords(lattice: Dict, x: torch.Tensor):
    """p = (x - origin) / spacing, its floor and fractional part (Eq. 10)."""
    origin = _t(lattice["origin"])
    spacing = _t(lattice["spacing"])
    p = (x - origin) / spacing
    f = torch.floor(p)
    return p, f, p - f


def ffd_eval(phi: torch.Tensor, lattice: Dict, x: torch.Tensor):
    """u_r(x) and grad u_r(x) for every rank (Eq. 10 and the gradient in Eq. 11).

    phi: [R][nz][ny][nx][3]; x: [N][3].  Returns U [N][R][3] and dU [N][R][3][3] with
    dU[n, r, i, j] = d u_{r,i} / d x_j in world units.  Node indices i = floor(p_1) - 1 + l (x),
    j = floor(p_2) - 1 + m (y), k = floor(p_3) - 1 + n (z); nodes outside the lattice contribute zero.
    """
    nx, ny, nz, R = lattice["nx"], lattice["ny"], lattice["nz"], lattice["R"]
    spacing = _t(lattice["spacing"])
    _, f, u = lattice_coords(lattice, x)
    B = [bspline(u[:, a]) for a in range(3)]          # each [N][4]
    dB = [bspline(u[:, a], 1) / spacing[a] for a in range(3)]
    fi = f.to(torch.long)
    N = x.shape[0]
    U = torch.zeros(N, R, 3, dtype=DT)
    dU = torch.zeros(N, R, 3, 3, dtype=DT)
    phi_flat = phi.reshape(R, nz * ny * nx, 3)
    for n3 in range(4):
        k = fi[:, 2] - 1 + n3
        for m in range(4):
            j = fi[:, 1] - 1 + m
            for l in range(4):
                i = fi[:, 0] - 1 + l
                valid = (i >= 0) & (i < nx) & (j >= 0) & (j < ny) & (k >= 0) & (k < nz)
                flat = torch.where(valid, (k * ny + j) * nx + i, torch.zeros_like(i))
                d = phi_flat[:, flat, :] * valid.to(DT)[None, :, None]      # [R][N][3]
                d = d.permute(1, 0, 2)                                          # [N][R][3]
                wgt = B[0][:, l] * B[1][:, m] * B[2][:, n3]
                g = torch.stack([dB[0][:, l] * B[1][:, m] * B[2][:, n3],
                                 B[0][:, l] * dB[1][:, m] * B[2][:, n3],
                                 B[0][:, l] * B[1][:, m] * dB[2][:, n3]], -1)   # [N][3]
                U = U + wgt[:, None, None] * d
                dU = dU + d[:, :, :, None] * g[:, None, None, :]
    return U, dU


# ----------------------------------------------------------------------------- Sec. 3.2
def deform(mu0: torch.Tensor, sigma0: torch.Tensor, U: torch.Tensor, dU: torch.Tensor, w_b: torch.Tensor):
    """Deformation-informed warp for one time point (Eq. 7-9, 11):
    mu' = mu0 + sum_r w_r u_r(mu0), K = I + sum_r w_r grad u_r(mu0), Sigma' = K Sigma0 K^T."""
    mu = mu0 + torch.einsum("r,nri->ni", w_b, U)
    K = torch.eye(3, dtype=DT)[None] + torch.einsum("r,nrij->nij", w_b, dU)
    sigma = K @ sigma0 @ K.transpose(-1, -2)
    return mu, sigma, K


# ----------------------------------------------------------------------------- volumes (evaluation)
def grid_centres(grid: Dict) -> torch.Tensor:
    """Voxel centres [nz][ny][nx][3] of a grid: origin + (i, j, k) * spacing, i (x) fastest."""
    o, h = _t(grid["origin"]), _t(grid["spacing"])
    k, j, i = torch.meshgrid(torch.arange(grid["nz"], dtype=DT), torch.arange(grid["ny"], dtype=DT),
                             torch.arange(grid["nx"], dtype=DT), indexing="ij")
    return torch.stack([o[0] + i * h[0], o[1] + j * h[1], o[2] + k * h[2]], -1)


def voxelize(gauss: Dict, lattice: Dict, phi, w_row, grid: Dict, cutoff: Optional[float] = 3.5) -> np.ndarray:
    """Attenuation volume of the cloud deformed with weights w_row [R] (Eq. 3 with the warp of Eq. 7-8):
    vol[k][j][i] = sum_n rho_n exp(-E_n / 2), E_n = (x - mu'_n)^T Sigma'_n^-1 (x - mu'_n), at the voxel
    centres, each Gaussian taken where E_n <= cutoff^2 (all of it when cutoff is None); folded Gaussians
    (det K <= 1e-6) are dropped as in the projector."""
    with torch.no_grad():
        T = _inputs(gauss, phi, np.asarray(w_row)[None])
        sigma0 = covariance(T["scale"], T["quat"])
        U, dU = ffd_eval(T["phi"], lattice, T["mu0"])
        mu, sigma, K = deform(T["mu0"], sigma0, U, dU, T["w"][0])
        P = torch.linalg.inv(sigma)
        keep = torch.linalg.det(K) > FOLD_EPS
        X = grid_centres(grid).reshape(-1, 3)
        vol = torch.zeros(X.shape[0], dtype=DT)
        for n in torch.nonzero(keep).flatten().tolist():
            d = X - mu[n]
            E = torch.einsum("vi,ij,vj->v", d, P[n], d)
            val = T["rho"][n] * torch.exp(-0.5 * E)
            if cutoff is not None:
                val = torch.where(E <= cutoff * cutoff, val, torch.zeros_like(val))
            vol += val
        return vol.reshape(grid["nz"], grid["ny"], grid["nx"]).numpy()


def dvf(lattice: Dict, phi, w_row, grid: Dict) -> np.ndarray:
    """Displacement D(x, t) - x = sum_r w_r u_r(x) at the voxel centres, [nz][ny][nx][3] (Eq. 9-10)."""
    with torch.no_grad():
        X = grid_centres(grid).reshape(-1, 3)
        U, _ = ffd_eval(_t(phi), lattice, X)
        d = torch.einsum("r,nri->ni", _t(w_row), U)
        return d.reshape(grid["nz"], grid["ny"], grid["nx"], 3).numpy()


# ----------------------------------------------------------------------------- geometry
def view_tensors(view: Dict):
    v = {k: _t(view[k]) for k in ("src", "det_c", "e_u", "e_v")}
    n_d = torch.linalg.cross(v["e_u"], v["e_v"])
    n_d = n_d / n_d.norm()
    if torch.dot(n_d, v["det_c"] - v["src"]) < 0:
        n_d = -n_d
    v["n_d"] = n_d
    for k in ("du", "dv", "off_u", "off_v"):
        v[k] = float(view[k])
    v["nu"], v["nv"] = int(view["nu"]), int(view["nv"])
    v["parallel"] = bool(view.get("parallel", False))
    return v


def pixel_centres(v) -> torch.Tensor:
    """Centres of all pixels, [nv * nu][3], pixel (i, j) at flat index j * nu + i."""
    i = torch.arange(v["nu"], dtype=DT)
    j = torch.arange(v["nv"], dtype=DT)
    uu = (i - (v["nu"] - 1) / 2 + v["off_u"]) * v["du"]
    vv = (j - (v["nv"] - 1) / 2 + v["off_v"]) * v["dv"]
    X = (v["det_c"][None, None, :] + uu[None, :, None] * v["e_u"][None, None, :]
         + vv[:, None, None] * v["e_v"][None, None, :])
    return X.reshape(-1, 3)


def ray_directions(v, X: torch.Tensor) -> torch.Tensor:
    if v["parallel"]:
        d = v["det_c"] - v["src"]
        return (d / d.norm()).expand_as(X)
    d = X - v["src"][None]
    return d / d.norm(dim=-1, keepdim=True)


def project_to_pixel(v, pts: torch.Tensor) -> torch.Tensor:
    """Detector pixel coordinates (i, j) of the ray through each point (cone: from the source)."""
    if v["parallel"]:
        d = v["det_c"] - v["src"]
        d = d / d.norm()
        t = ((v["det_c"][None] - pts) @ v["n_d"]) / torch.dot(d, v["n_d"])
        X = pts + t[:, None] * d[None]
    else:
        s = v["src"]
        t = torch.dot(v["det_c"] - s, v["n_d"]) / ((pts - s[None]) @ v["n_d"])
        X = s[None] + t[:, None] * (pts - s[None])
    rel = X - v["det_c"][None]
    ii = (rel @ v["e_u"]) / v["du"] + (v["nu"] - 1) / 2 - v["off_u"]
    jj = (rel @ v["e_v"]) / v["dv"] + (v["nv"] - 1) / 2 - v["off_v"]
    return torch.stack([ii, jj], -1)


# ----------------------------------------------------------------------------- Eq. 4 / X-ray transform
def alive_mask(v, mu: torch.Tensor, P: torch.Tensor, K: torch.Tensor, cutoff: Optional[float]) -> torch.Tensor:
    alive = torch.linalg.det(K) > FOLD_EPS
    if not v["parallel"]:
        alive = alive & (((mu - v["src"][None]) @ v["n_d"]) > 0)
        if cutoff is not None:
            m = v["src"][None] - mu
            c_src = torch.einsum("ni,nij,nj->n", m, P, m)
            alive = alive & (c_src > cutoff * cutoff)
    return alive


def pair_values(a, b, c, rho, cutoff: Optional[float]):
    """V = rho sqrt(2 pi / a) exp(-E/2), E = c - b^2/a, and the cutoff mask E <= cutoff^2."""
    E = c - b * b / a
    V = rho * torch.sqrt(2 * math.pi / a) * torch.exp(-0.5 * E)
    mask = torch.ones_like(E, dtype=torch.bool) if cutoff is None else (E <= cutoff * cutoff)
    return V, mask, E


def render_view_brute(v, mu, P, rho, alive, cutoff, chunk: int = 512) -> torch.Tensor:
    """Every ray against every Gaussian; returns the flat image [nv * nu]."""
    X = pixel_centres(v)
    d = ray_directions(v, X)
    npix = X.shape[0]
    img = torch.zeros(npix, dtype=DT)
    idx = torch.nonzero(alive).flatten()
    for s0 in range(0, idx.numel(), chunk):
        sel = idx[s0:s0 + chunk]
        mu_c, P_c, rho_c = mu[sel], P[sel], rho[sel]
        Pflat = P_c.reshape(-1, 9)
        if v["parallel"]:
            dd = d[0]
            a = (torch.outer(dd, dd).reshape(1, 9) @ Pflat.T).expand(npix, -1)
            Pd = P_c @ dd
            b = X @ Pd.T - (mu_c * Pd).sum(-1)[None]
            XX = (X[:, :, None] * X[:, None, :]).reshape(npix, 9)
            Pmu = torch.einsum("nij,nj->ni", P_c, mu_c)
            c = XX @ Pflat.T - 2 * X @ Pmu.T + (mu_c * Pmu).sum(-1)[None]
        else:
            m = v["src"][None] - mu_c
            Pm = torch.einsum("nij,nj->ni", P_c, m)
            dd = (d[:, :, None] * d[:, None, :]).reshape(npix, 9)
            a = dd @ Pflat.T
            b = d @ Pm.T
            c = (m * Pm).sum(-1)[None].expand(npix, -1)
        V, mask, _ = pair_values(a, b, c, rho_c[None], cutoff)
        img = img + (V * mask.to(DT)).sum(1)
    return img


def bbox_pixels(v, mu: torch.Tensor, sigma: torch.Tensor, cutoff: float):
    """Pixel rectangle [i0, i1] x [j0, j1] (inclusive) of the detector image of the axis-aligned box
    with half extents cutoff * sqrt(Sigma_ii) around each mean."""
    h = cutoff * torch.sqrt(torch.diagonal(sigma, dim1=-2, dim2=-1))
    signs = torch.tensor([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], dtype=DT)
    corners = mu[:, None, :] + signs[None] * h[:, None, :]                      # [N][8][3]
    pix = project_to_pixel(v, corners.reshape(-1, 3)).reshape(-1, 8, 2)
    lo = torch.ceil(pix.min(1).values - 1e-9)
    hi = torch.floor(pix.max(1).values + 1e-9)
    lo[:, 0].clamp_(min=0)
    lo[:, 1].clamp_(min=0)
    hi[:, 0].clamp_(max=v["nu"] - 1)
    hi[:, 1].clamp_(max=v["nv"] - 1)
    return lo.to(torch.long), hi.to(torch.long)


def bbox_pairs(v, mu, sigma, alive, cutoff):
    """(pixel flat index, Gaussian index) for every pixel inside each alive Gaussian's rectangle."""
    with torch.no_grad():
        if not v["parallel"]:
            h = cutoff * torch.sqrt(torch.diagonal(sigma, dim1=-2, dim2=-1))
            # every box corner must lie in front of the source for the rectangle to be conservative
            signs = torch.tensor([[sx, sy, sz] for sx in (-1, 1) for sy in (-1, 1) for sz in (-1, 1)], dtype=DT)
            corners = mu[:, None, :] + signs[None] * h[:, None, :]
            depth = (corners - v["src"]) @ v["n_d"]
            if bool(((depth <= 0).any(1) & alive).any()):
                raise ValueError("a cutoff box reaches behind the source; use mode='brute'")
        lo, hi = bbox_pixels(v, mu, sigma, cutoff)
        w = (hi[:, 0] - lo[:, 0] + 1).clamp(min=0)
        hgt = (hi[:, 1] - lo[:, 1] + 1).clamp(min=0)
        cnt = torch.where(alive, w * hgt, torch.zeros_like(w))
        g = torch.repeat_interleave(torch.arange(mu.shape[0]), cnt)
        start = torch.cumsum(cnt, 0) - cnt
        k = torch.arange(g.numel()) - start[g]
        ii = lo[g, 0] + k % w[g]
        jj = lo[g, 1] + k // w[g]
        return jj * v["nu"] + ii, g


def render_view_bbox(v, mu, sigma, P, rho, alive, cutoff) -> torch.Tensor:
    pix, g = bbox_pairs(v, mu, sigma, alive, cutoff)
    X = pixel_centres(v)[pix]
    d = ray_directions(v, X)
    mu_g, P_g = mu[g], P[g]
    m = (X if v["parallel"] else v["src"][None]) - mu_g
    Pd = torch.einsum("nij,nj->ni", P_g, d)
    a = (d * Pd).sum(-1)
    b = (m * Pd).sum(-1)
    c = torch.einsum("ni,nij,nj->n", m, P_g, m)
    V, mask, _ = pair_values(a, b, c, rho[g], cutoff)
    img = torch.zeros(v["nu"] * v["nv"], dtype=DT)
    return img.index_add(0, pix, V * mask.to(DT))


def cutoff_margin(gauss: Dict, lattice: Dict, phi, w, views: Sequence[Dict], cutoff: float = 3.5) -> np.ndarray:
    """Per Gaussian, the smallest |E - cutoff^2| / cutoff^2 over its (pixel, view) pairs, E the squared
    Mahalanobis distance from the pixel ray to the deformed mean (Eq. 4 with the deformation of Eq. 7-11),
    in float64 (inf for a Gaussian without pairs).  A pair whose margin is at the level of FP32 rounding
    (~1e-7) is decided by rounding: a float32 evaluation of the same E may include it or not, so parity
    tests that compare gradients element by element leave such Gaussians out.  Pairs are taken from the
    box of the 1.05 x cutoff ellipsoid, so that near misses just outside the cutoff count too."""
    T = _inputs(gauss, phi, w)
    with torch.no_grad():
        sigma0 = covariance(T["scale"], T["quat"])
        U, dU = ffd_eval(T["phi"], lattice, T["mu0"])
        n = T["mu0"].shape[0]
        out = torch.full((n,), float("inf"), dtype=DT)
        c2 = cutoff * cutoff
        for b, view in enumerate(views):
            v = view_tensors(view)
            mu, sigma, K = deform(T["mu0"], sigma0, U, dU, T["w"][b])
            P = torch.linalg.inv(sigma)
            alive = alive_mask(v, mu, P, K, cutoff)
            pix, g = bbox_pairs(v, mu, sigma, alive, 1.05 * cutoff)  # also the near misses just outside
            if g.numel() == 0:
                continue
            X = pixel_centres(v)[pix]
            d = ray_directions(v, X)
            m = (X if v["parallel"] else v["src"][None]) - mu[g]
            Pd = torch.einsum("nij,nj->ni", P[g], d)
            a = (d * Pd).sum(-1)
            bb = (m * Pd).sum(-1)
            c = torch.einsum("ni,nij,nj->n", m, P[g], m)
            _, _, E = pair_values(a, bb, c, T["rho"][g], cutoff)
            out = out.scatter_reduce(0, g, (E - c2).abs() / c2, reduce="amin")
    return out.numpy()


def _inputs(gauss: Dict, phi, w):
    return dict(mu0=_t(gauss["mu0"]), scale=_t(gauss["scale"]), quat=_t(gauss["quat"]), rho=_t(gauss["rho"]),
                phi=_t(phi), w=_t(w))


def render_tensors(T: Dict, lattice: Dict, views: Sequence[Dict], cutoff: Optional[float] = 3.5,
                   mode: str = "bbox") -> torch.Tensor:
    """Projections [P][nv][nu] of the deformed Gaussians (Eq. 1, 3, 4, 7-11) from float64 tensors
    (``T`` holds mu0, scale, quat, rho, phi, w; autograd flows through all of them)."""
    sigma0 = covariance(T["scale"], T["quat"])
    U, dU = ffd_eval(T["phi"], lattice, T["mu0"])
    out = []
    for b, view in enumerate(views):
        v = view_tensors(view)
        mu, sigma, K = deform(T["mu0"], sigma0, U, dU, T["w"][b])
        P = torch.linalg.inv(sigma)
        alive = alive_mask(v, mu.detach(), P.detach(), K.detach(), cutoff)
        if mode == "brute" or cutoff is None:
            img = render_view_brute(v, mu, P, T["rho"], alive, cutoff)
        elif mode == "bbox":
            img = render_view_bbox(v, mu, sigma, P, T["rho"], alive, cutoff)
        else:
            raise ValueError(mode)
        out.append(img.reshape(v["nv"], v["nu"]))
    return torch.stack(out) if out else torch.zeros(0, dtype=DT)


def ewa_view(v, mu: torch.Tensor, sigma: torch.Tensor, rho: torch.Tensor, keep: torch.Tensor,
             cutoff: Optional[float], chunk: int = 256) -> torch.Tensor:
    """The paper's 2D-Gaussian model of one cone-beam view (Sec. 3.1, Eq. 4), brute force over every pixel:
    each Gaussian becomes rho~ exp(-1/2 Delta^T Sig2^-1 Delta) around its projected mean, where
    Sig2 = J Sigma' J^T with J the 2 x 3 Jacobian of the world-to-pixel perspective map at mu' (the EWA
    covariance with its depth row and column dropped), and rho~ = rho sqrt(2 pi) |det J3| sqrt(det Sigma'
    / det Sig2) with J3 = [J; d^T / |d|], d = mu' - src: the integration bias factor that makes the
    ray-space Gaussian's integral along the ray the line integral.  A pair contributes where
    Delta^T Sig2^-1 Delta <= cutoff^2."""
    s, n = v["src"], v["n_d"]
    sdd = torch.dot(v["det_c"] - s, n)
    d = mu - s[None]
    dn = d @ n
    sc = sdd / dn
    Ju = sc[:, None] / v["du"] * (v["e_u"][None] - ((d @ v["e_u"]) / dn)[:, None] * n[None])
    Jv = sc[:, None] / v["dv"] * (v["e_v"][None] - ((d @ v["e_v"]) / dn)[:, None] * n[None])
    J = torch.stack([Ju, Jv], 1)                                            # [N][2][3]
    sig2 = J @ sigma @ J.transpose(-1, -2)
    J3 = torch.cat([J, (d / d.norm(dim=1, keepdim=True))[:, None, :]], 1)
    amp = rho * math.sqrt(2 * math.pi) * torch.linalg.det(J3).abs() * torch.sqrt(
        torch.linalg.det(sigma) / torch.linalg.det(sig2))
    mpix = project_to_pixel(v, mu)
    jj, ii = torch.meshgrid(torch.arange(v["nv"], dtype=DT), torch.arange(v["nu"], dtype=DT), indexing="ij")
    pix = torch.stack([ii.reshape(-1), jj.reshape(-1)], -1)                 # [npix][2]
    out = torch.zeros(pix.shape[0], dtype=DT)
    inv2 = torch.linalg.inv(sig2)
    for a in range(0, mu.shape[0], chunk):
        sl = slice(a, a + chunk)
        D = pix[None] - mpix[sl, None, :]                                   # [c][npix][2]
        E = torch.einsum("cpi,cij,cpj->cp", D, inv2[sl], D)
        val = amp[sl, None] * torch.exp(-0.5 * E)
        mask = keep[sl, None] & (dn[sl, None] > 0)
        if cutoff is not None:
            mask = mask & (E <= cutoff * cutoff)
        out = out + torch.where(mask, val, torch.zeros_like(val)).sum(0)
    return out


def render_ewa(gauss: Dict, lattice: Dict, phi, w, views: Sequence[Dict], cutoff: Optional[float] = 3.5,
               grad: bool = False):
    """Projections [P][nv][nu] with the 2D-Gaussian model for cone-beam views (parallel views are the
    exact model, which the 2D Gaussian equals there).  With grad=True returns the float64 tensors' graph
    inputs and output for autograd."""
    T = _inputs(gauss, phi, w)
    if grad:
        for k in T:
            T[k].requires_grad_(True)
    sigma0 = covariance(T["scale"], T["quat"])
    U, dU = ffd_eval(T["phi"], lattice, T["mu0"])
    out = []
    for b, view in enumerate(views):
        v = view_tensors(view)
        mu, sigma, K = deform(T["mu0"], sigma0, U, dU, T["w"][b])
        keep = torch.linalg.det(K).detach() > FOLD_EPS
        if v["parallel"]:
            P = torch.linalg.inv(sigma)
            alive = alive_mask(v, mu.detach(), P.detach(), K.detach(), cutoff)
            img = render_view_brute(v, mu, P, T["rho"], alive, cutoff)
        else:
            img = ewa_view(v, mu, sigma, T["rho"], keep, cutoff)
        out.append(img.reshape(v["nv"], v["nu"]))
    I = torch.stack(out)
    return (T, I) if grad else I.detach().numpy()


def project_vjp_ewa(gauss: Dict, lattice: Dict, phi, w, views: Sequence[Dict], grad_proj,
                    cutoff: Optional[float] = 3.5) -> Dict[str, np.ndarray]:
    """Gradients of sum(grad_proj * render_ewa) with respect to every input (autograd)."""
    T, I = render_ewa(gauss, lattice, phi, w, views, cutoff, grad=True)
    (I * _t(grad_proj)).sum().backward()
    return {k: T[k].grad.numpy() for k in ("mu0", "scale", "quat", "rho", "phi", "w")}


def render(gauss: Dict, lattice: Dict, phi, w, views: Sequence[Dict], cutoff: Optional[float] = 3.5,
           mode: str = "bbox") -> np.ndarray:
    """Projections [P][nv][nu] as float64 numpy.  ``gauss`` holds mu0, scale, quat, rho."""
    with torch.no_grad():
        return render_tensors(_inputs(gauss, phi, w), lattice, views, cutoff, mode).numpy()


def project_vjp(gauss: Dict, lattice: Dict, phi, w, views: Sequence[Dict], grad_proj,
                cutoff: Optional[float] = 3.5, mode: str = "bbox") -> Dict[str, np.ndarray]:
    """Gradient of sum(grad_proj * I) with respect to mu0, scale, quat, rho, phi and w (autograd of the
    definition above; the cutoff mask is held fixed, i.e. the truncated sum is differentiated almost
    everywhere)."""
    T = {k: t.clone().requires_grad_(True) for k, t in _inputs(gauss, phi, w).items()}
    I = render_tensors(T, lattice, views, cutoff, mode)
    (I * _t(grad_proj)).sum().backward()
    return {k: t.grad.numpy().copy() if t.grad is not None else np.zeros(t.shape) for k, t in T.items()}


def render_pixels(gauss: Dict, lattice: Dict, phi, w, view: Dict, w_row, pix_ij: np.ndarray,
                  cutoff: float = 3.5) -> np.ndarray:
    """Values of chosen pixels (i, j) of one view, each summed over every Gaussian (for sampled checks
    at full size)."""
    with torch.no_grad():
        T = _inputs(gauss, phi, w_row[None])
        sigma0 = covariance(T["scale"], T["quat"])
        U, dU = ffd_eval(T["phi"], lattice, T["mu0"])
        v = view_tensors(view)
        mu, sigma, K = deform(T["mu0"], sigma0, U, dU, T["w"][0])
        P = torch.linalg.inv(sigma)
        alive = alive_mask(v, mu, P, K, cutoff)
        X_all = pixel_centres(v)
        pix_ij = np.asarray(pix_ij)
        flat = torch.as_tensor(pix_ij[:, 1] * v["nu"] + pix_ij[:, 0])
        X = X_all[flat]
        d = ray_directions(v, X)
        idx = torch.nonzero(alive).flatten()
        out = torch.zeros(X.shape[0], dtype=DT)
        for s0 in range(0, idx.numel(), 4096):
            sel = idx[s0:s0 + 4096]
            mu_c, P_c = mu[sel], P[sel]
            m = (X[:, None, :] if v["parallel"] else v["src"][None, None, :]) - mu_c[None]   # [Q][n][3]
            Pd = torch.einsum("nij,qj->qni", P_c, d)
            a = (d[:, None, :] * Pd).sum(-1)
            b = (m * Pd).sum(-1)
            c = torch.einsum("qni,nij,qnj->qn", m, P_c, m)
            V, mask, _ = pair_values(a, b, c, T["rho"][sel][None], cutoff)
            out += (V * mask.to(DT)).sum(1)
        return out.numpy()


def pair_count(gauss: Dict, lattice: Dict, phi, w, views: Sequence[Dict], cutoff: float = 3.5) -> int:
    """Number of (ray, Gaussian) pairs with E <= cutoff^2 (bbox enumeration)."""
    with torch.no_grad():
        T = _inputs(gauss, phi, w)
        sigma0 = covariance(T["scale"], T["quat"])
        U, dU = ffd_eval(T["phi"], lattice, T["mu0"])
        total = 0
        for b, view in enumerate(views):
            v = view_tensors(view)
            mu, sigma, K = deform(T["mu0"], sigma0, U, dU, T["w"][b])
            P = torch.linalg.inv(sigma)
            alive = alive_mask(v, mu, P, K, cutoff)
            pix, g = bbox_pairs(v, mu, sigma, alive, cutoff)
            X = pixel_centres(v)[pix]
            d = ray_directions(v, X)
            m = (X if v["parallel"] else v["src"][None]) - mu[g]
            Pd = torch.einsum("nij,nj->ni", P[g], d)
            a = (d * Pd).sum(-1)
            b_ = (m * Pd).sum(-1)
            c = torch.einsum("ni,nij,nj->n", m, P[g], m)
            _, mask, _ = pair_values(a, b_, c, T["rho"][g], cutoff)
            total += int(mask.sum())
        return total


# ----------------------------------------------------------------------------- Sec. 4.2
def mse_loss(proj, meas) -> float:
    """L2 loss in projection space read as mean((I - M)^2) over all pixels of all projections."""
    return float(torch.mean((_t(proj) - _t(meas)) ** 2))


def lr_at(lr0: float, lr1: float, it: int, total: int) -> float:
    """Linear decay from lr0 at iteration 0 to lr1 at the final iteration (Sec. 4.2)."""
    if total <= 1:
        return lr0
    a = min(max(it / (total - 1), 0.0), 1.0)
    return lr0 + (lr1 - lr0) * a


def adam_update(param, grad, m, v, step: int, lr: float, beta1: float, beta2: float, eps: float):
    """One Adam step (Kingma & Ba) on float64 arrays; ``step`` counts from 1.  Returns new (param, m, v).
    Pinned by the first-step closed form (update = lr g / (|g| + eps)) and a scalar trajectory."""
    param, grad, m, v = (np.asarray(a, dtype=np.float64) for a in (param, grad, m, v))
    m = beta1 * m + (1 - beta1) * grad
    v = beta2 * v + (1 - beta2) * grad * grad
    mhat = m / (1 - beta1 ** step)
    vhat = v / (1 - beta2 ** step)
    return param - lr * mhat / (np.sqrt(vhat) + eps), m, v


def adam_update_reparam(param, grad, m, v, step: int, lr: float, beta1: float, beta2: float, eps: float,
                        kind: str = "plain"):
    """Adam on a re-parameterisation of a positive physical parameter: kind 'log' optimises
    theta = log(param), kind 'softplus' optimises theta with param = log(1 + exp(theta)); 'plain' is
    :func:`adam_update`.  ``grad`` is dL/dparam; the chain rule gives dL/dtheta.  Returns the new physical
    parameter and the moments (which live in theta space)."""
    param = np.asarray(param, dtype=np.float64)
    grad = np.asarray(grad, dtype=np.float64)
    if kind == "plain":
        return adam_update(param, grad, m, v, step, lr, beta1, beta2, eps)
    if kind == "log":
        theta, dtheta = np.log(param), param                       # d param / d theta = exp(theta)
    elif kind == "softplus":
        theta = np.log(np.expm1(param))
        dtheta = 1.0 / (1.0 + np.exp(-theta))                     # sigmoid(theta)
    else:
        raise ValueError(kind)
    theta, m, v = adam_update(theta, grad * dtheta, m, v, step, lr, beta1, beta2, eps)
    new = np.exp(theta) if kind == "log" else np.log1p(np.exp(theta))
    return new, m, v
