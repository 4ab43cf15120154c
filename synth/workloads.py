"""Seeded synthetic workloads (input recipes only; no method arithmetic).

Every array is float64 numpy; the GPU path casts to float32 itself.  Layouts:

* ``mu0[N][3]`` mm, ``scale[N][3]`` mm (>0), ``quat[N][4]`` as (w, x, y, z), not necessarily unit,
  ``rho[N]`` mm^-1 -- the reference Gaussians of Sec. 3.1 (Eq. 2, Sigma = R S S^T R^T).
* ``phi[R][nz][ny][nx][3]`` mm -- control-point displacements d^r_ijk of the low-rank FFD (Sec. 3.3,
  Eq. 10), x index fastest; node (i, j, k) sits at ``origin + (i, j, k) * spacing``.
* ``w[P][R]`` -- temporal weights omega_r(t) at each projection's time (Eq. 9).
* ``views`` -- one dict per projection: source point, detector centre, detector axes e_u / e_v (unit,
  orthogonal), pixel pitch du / dv (mm), detector offsets off_u / off_v (pixels), nu x nv pixels and a
  ``parallel`` flag.  Circular cone-beam scans rotate about the world z axis.

The recipes follow the scan set-up of Sec. 4.1 (SAD 1000 mm, SDD about 1.5 m, full-circle scans,
breathing-driven low-rank motion with cycle-to-cycle variation and drift) at the sizes of the
benchmark configurations: a tiny 2,000-Gaussian cloud, a 100k-Gaussian thorax phantom with 680
projections of 256x256, four uneven thorax scans for batching, and a 500k / 512x512 scale case.
The paper's own datasets (XCAT, 4DLung) are not available; these stand in for them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np


@dataclasses.dataclass
class Workload:
    name: str
    mu0: np.ndarray
    scale: np.ndarray
    quat: np.ndarray
    rho: np.ndarray
    lattice: Dict
    phi: np.ndarray
    w: np.ndarray
    views: List[Dict]
    times: np.ndarray
    angles: np.ndarray
    extra: Dict = dataclasses.field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.mu0.shape[0])

    @property
    def R(self) -> int:
        return int(self.lattice["R"])

    def subset(self, idx) -> "Workload":
        """Same workload restricted to Gaussians ``idx`` (lattice, weights, views unchanged)."""
        idx = np.asarray(idx, dtype=np.int64)
        return dataclasses.replace(self, mu0=self.mu0[idx], scale=self.scale[idx], quat=self.quat[idx],
                                   rho=self.rho[idx], extra=dict(self.extra))

    def select_views(self, ids) -> "Workload":
        ids = list(ids)
        return dataclasses.replace(self, w=self.w[ids], views=[self.views[i] for i in ids],
                                   times=self.times[ids], angles=self.angles[ids], extra=dict(self.extra))


def circular_views(angles, sad: float, sdd: float, nu: int, nv: int, du: float, dv: float,
                   off_u: float = 0.0, off_v: float = 0.0, parallel: bool = False) -> List[Dict]:
    """Circular scan about the world z axis: source at SAD*(cos a, sin a, 0), detector centre at
    -(SDD-SAD)*(cos a, sin a, 0), e_u = (-sin a, cos a, 0), e_v = (0, 0, 1)."""
    out = []
    for a in np.asarray(angles, dtype=np.float64):
        c, s = math.cos(a), math.sin(a)
        out.append(dict(src=np.array([sad * c, sad * s, 0.0]),
                        det_c=np.array([-(sdd - sad) * c, -(sdd - sad) * s, 0.0]),
                        e_u=np.array([-s, c, 0.0]), e_v=np.array([0.0, 0.0, 1.0]),
                        du=float(du), dv=float(dv), off_u=float(off_u), off_v=float(off_v),
                        nu=int(nu), nv=int(nv), parallel=bool(parallel)))
    return out


def _uniform_in_ellipsoid(rng, n, semi, centre=(0.0, 0.0, 0.0)):
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = rng.uniform(size=(n, 1)) ** (1.0 / 3.0)
    return np.asarray(centre) + d * r * np.asarray(semi)


def _random_quats(rng, n):
    q = rng.normal(size=(n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _lattice(nodes, spacing, origin, R):
    return dict(nx=int(nodes[0]), ny=int(nodes[1]), nz=int(nodes[2]), R=int(R),
                origin=np.asarray(origin, dtype=np.float64), spacing=np.asarray(spacing, dtype=np.float64))


def _node_coords(lat):
    xs = lat["origin"][0] + lat["spacing"][0] * np.arange(lat["nx"])
    ys = lat["origin"][1] + lat["spacing"][1] * np.arange(lat["ny"])
    zs = lat["origin"][2] + lat["spacing"][2] * np.arange(lat["nz"])
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return X, Y, Z  # each [nz][ny][nx]


def tiny(seed: int = 0, n: int = 2000, n_proj: int = 16, nu: int = 64, nv: int = 64,
         du: float = 1.6, dv: float = 1.6, motion_seed: Optional[int] = None) -> Workload:
    """2,000 Gaussians uniform in the ellipsoid inscribed in a 64^3 mm box; log-normal scales
    (median 2 mm, sigma_log 0.4); uniform random rotations; densities U[0.005, 0.03] mm^-1;
    8^3 control lattice at 10 mm (origin -35 mm) with R=2 ranks of N(0, 1 mm) displacements;
    16 cone-beam projections (SAD 1000, SDD 1500) of a 64x64 detector with 1.6 mm pixels over 360 deg;
    sinusoidal breathing weights w1 = sin(2 pi t / 4 s), w2 = 0.5 cos(2 pi t / 4 s), t_p = 3.75 p s.
    ``motion_seed`` redraws phi (and shifts the weights) for a second, 'measured' state."""
    rng = np.random.default_rng(seed)
    mu0 = _uniform_in_ellipsoid(rng, n, (32.0, 32.0, 32.0))
    scale = np.exp(np.log(2.0) + 0.4 * rng.normal(size=(n, 3)))
    quat = _random_quats(rng, n)
    rho = rng.uniform(0.005, 0.03, size=n)
    lat = _lattice((8, 8, 8), (10.0, 10.0, 10.0), (-35.0, -35.0, -35.0), 2)
    mrng = np.random.default_rng(seed + 1000 if motion_seed is None else motion_seed)
    phi = mrng.normal(0.0, 1.0, size=(2, 8, 8, 8, 3))
    times = 3.75 * np.arange(n_proj)
    shift = 0.0 if motion_seed is None else 0.3
    w = np.stack([np.sin(2 * math.pi * times / 4.0 + shift), 0.5 * np.cos(2 * math.pi * times / 4.0 + shift)], 1)
    angles = 2 * math.pi * np.arange(n_proj) / n_proj
    views = circular_views(angles, 1000.0, 1500.0, nu, nv, du, dv)
    return Workload("tiny", mu0, scale, quat, rho, lat, phi, w, views, times, angles, dict(seed=seed))


# ---------------------------------------------------------------- thorax phantom
BODY_SEMI = np.array([120.0, 85.0, 120.0])
LUNG_CENTRES = np.array([[55.0, 0.0, 20.0], [-55.0, 0.0, 20.0]])
LUNG_SEMI = np.array([40.0, 55.0, 80.0])
TUMOUR_CENTRE = np.array([-55.0, 0.0, 30.0])
TUMOUR_RADIUS = 7.5
MU_BODY, MU_LUNG, MU_TUMOUR = 0.02, 0.004, 0.02


def thorax_attenuation(x: np.ndarray) -> np.ndarray:
    """Piecewise-constant phantom: body ellipsoid 0.02/mm, lungs 0.004/mm (replacing body), a 15 mm
    tumour sphere 0.02/mm in the right lung, 0 outside the body."""
    x = np.asarray(x, dtype=np.float64)
    mu = np.where(np.sum((x / BODY_SEMI) ** 2, -1) <= 1.0, MU_BODY, 0.0)
    for c in LUNG_CENTRES:
        mu = np.where(np.sum(((x - c) / LUNG_SEMI) ** 2, -1) <= 1.0, MU_LUNG, mu)
    mu = np.where(np.sum((x - TUMOUR_CENTRE) ** 2, -1) <= TUMOUR_RADIUS ** 2, MU_TUMOUR, mu)
    return mu


def _lung_mask(X, Y, Z):
    m = np.zeros_like(X)
    for c in LUNG_CENTRES:
        m += np.exp(-0.5 * (((X - c[0]) / LUNG_SEMI[0]) ** 2 + ((Y - c[1]) / LUNG_SEMI[1]) ** 2
                            + ((Z - c[2]) / LUNG_SEMI[2]) ** 2))
    return np.clip(m, 0.0, 1.0)


def breathing_surrogate(times: np.ndarray, R: int = 3, phase0: float = 0.0) -> np.ndarray:
    """Irregular breathing: period T(t) = 4.25 + 0.75 sin(2 pi t / 47 s) in [3.5, 5] s, phase
    psi = 2 pi int dt / T, SI amplitude A(t) = 12.5 + 7.5 sin(2 pi t / 61 s) in [5, 20] mm;
    w1 = A (1 - cos psi) / 2, w2 = 0.3 A sin(psi) / 2 (hysteresis), w3 = 2 sin(2 pi t / 90 s) (drift),
    w4 = 0.5 sin(2 pi t / 0.9 s) (a fast small component, scale case only)."""
    t = np.asarray(times, dtype=np.float64)
    fine = np.linspace(0.0, max(float(t.max()), 1e-9), 20001)
    period = 4.25 + 0.75 * np.sin(2 * math.pi * fine / 47.0)
    dpsi = 2 * math.pi / period
    psi_f = np.concatenate([[0.0], np.cumsum(0.5 * (dpsi[1:] + dpsi[:-1]) * np.diff(fine))])
    psi = np.interp(t, fine, psi_f) + phase0
    amp = 12.5 + 7.5 * np.sin(2 * math.pi * t / 61.0)
    cols = [amp * (1 - np.cos(psi)) / 2, 0.3 * amp * np.sin(psi) / 2, 2.0 * np.sin(2 * math.pi * t / 90.0),
            0.5 * np.sin(2 * math.pi * t / 0.9)]
    return np.stack(cols[:R], 1)


def thorax(seed: int = 1, n: int = 100_000, n_proj: int = 680, nu: int = 256, nv: int = 256,
           du: float = 1.6, dv: float = 1.6, spacing: float = 16.0, R: int = 3, scan_s: float = 60.0,
           phase0: float = 0.0) -> Workload:
    """Synthetic thorax scan.  Ground truth: ``n`` means uniform in the body ellipsoid, log-normal
    scales (median 2.5 mm, sigma_log 0.25), random rotations, rho_n = mu(mu_n) / (nbar (2 pi)^1.5 E[s1 s2 s3])
    so that the mixture's mean attenuation follows the phantom; motion with R ranks on a lattice over
    256^3 mm (span/spacing + 3 nodes per axis, origin -128 - spacing): r1 superior-inferior lung field
    (1 mm per unit weight), r2 the same field anterior-posterior, r3 a broad left-right drift field,
    r4 (R=4) a small anterior-posterior field; weights from :func:`breathing_surrogate`.  680 projections
    over 360 deg in a 60 s scan.  The returned workload is the reconstruction's initial state
    (GT means + N(0, 1 mm), scales x1.2, rho x U[0.5, 1.5], phi ~ N(0, 0.1 mm), w ~ N(0, 0.1));
    the ground truth sits in ``extra['gt']``."""
    rng = np.random.default_rng(seed)
    mu_gt = _uniform_in_ellipsoid(rng, n, BODY_SEMI)
    med, sl = 2.5, 0.25
    scale_gt = np.exp(np.log(med) + sl * rng.normal(size=(n, 3)))
    quat_gt = _random_quats(rng, n)
    vol = 4.0 / 3.0 * math.pi * np.prod(BODY_SEMI)
    nbar = n / vol
    e_s3 = (med * math.exp(sl * sl / 2)) ** 3
    rho_gt = thorax_attenuation(mu_gt) / (nbar * (2 * math.pi) ** 1.5 * e_s3)
    nodes = int(round(256.0 / spacing)) + 3
    origin = -128.0 - spacing
    lat = _lattice((nodes, nodes, nodes), (spacing,) * 3, (origin,) * 3, R)
    X, Y, Z = _node_coords(lat)
    lung = _lung_mask(X, Y, Z)
    broad = np.exp(-0.5 * ((X / 150.0) ** 2 + (Y / 150.0) ** 2 + (Z / 150.0) ** 2))
    phi_gt = np.zeros((R, lat["nz"], lat["ny"], lat["nx"], 3))
    phi_gt[0, ..., 2] = lung
    if R > 1:
        phi_gt[1, ..., 1] = lung
    if R > 2:
        phi_gt[2, ..., 0] = broad
    if R > 3:
        phi_gt[3, ..., 1] = 0.5 * broad
    times = scan_s * np.arange(n_proj) / n_proj
    angles = 2 * math.pi * np.arange(n_proj) / n_proj
    w_gt = breathing_surrogate(times, R, phase0)
    views = circular_views(angles, 1000.0, 1500.0, nu, nv, du, dv)
    irng = np.random.default_rng(seed + 7)
    mu0 = mu_gt + irng.normal(0.0, 1.0, size=mu_gt.shape)
    scale0 = scale_gt * 1.2
    rho0 = rho_gt * irng.uniform(0.5, 1.5, size=n)
    phi0 = irng.normal(0.0, 0.1, size=phi_gt.shape)
    w0 = irng.normal(0.0, 0.1, size=w_gt.shape)
    # Store the cloud in lattice-cell order (z, y, x) of the starting means: the order of the Gaussians is
    # free for the method, and spatial order keeps the FFD neighbourhoods of neighbouring Gaussians together.
    cell = np.floor((mu0 - lat["origin"]) / lat["spacing"]).astype(np.int64)
    order = np.lexsort((cell[:, 0], cell[:, 1], cell[:, 2]))
    mu0, scale0, rho0 = mu0[order], scale0[order], rho0[order]
    mu_gt, scale_gt, quat_gt, rho_gt = mu_gt[order], scale_gt[order], quat_gt[order], rho_gt[order]
    gt = dict(mu0=mu_gt, scale=scale_gt, quat=quat_gt.copy(), rho=rho_gt, phi=phi_gt, w=w_gt)
    return Workload("thorax", mu0, scale0, quat_gt.copy(), rho0, lat, phi0, w0, views, times, angles,
                    dict(seed=seed, gt=gt))


def thorax_batch(seed: int = 11, counts=(30_000, 60_000, 120_000, 200_000), n_proj: int = 680,
                 nu: int = 256, nv: int = 256) -> List[Workload]:
    """Four independent thorax scans with uneven Gaussian counts and their own surrogates."""
    return [thorax(seed=seed + 17 * i, n=c, n_proj=n_proj, nu=nu, nv=nv, phase0=0.9 * i)
            for i, c in enumerate(counts)]


def scale(seed: int = 5, n: int = 500_000, n_proj: int = 680) -> Workload:
    """500k Gaussians, 512x512 detector of 0.8 mm pixels, control lattice at 8 mm, R=4."""
    return thorax(seed=seed, n=n, n_proj=n_proj, nu=512, nv=512, du=0.8, dv=0.8, spacing=8.0, R=4)


def random_grad_proj(n_proj: int, nv: int, nu: int, seed: int = 3) -> np.ndarray:
    """A seeded upstream gradient dL/dI for testing the backward pass on its own."""
    return np.random.default_rng(seed).normal(size=(n_proj, nv, nu))
