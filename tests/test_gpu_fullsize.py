"""Parity at the benchmark sizes, in the launch configuration the bench times.

* Thorax, 100k Gaussians, 16 projections of 256x256, tile 16, 16 lanes per pair: projections on sampled
  pixels (the oracle sums every Gaussian for each chosen pixel) and, for one of the projections, every
  gradient against the oracle's full backward.
* Scale, 500k Gaussians, 512x512 detector of 0.8 mm pixels, lattice at 8 mm, R = 4: projections on
  sampled pixels; gradients on a seeded 1,000-Gaussian subset at that detector size and lattice.
* The largest call: 128 projections (DIGS_MAX_VIEWS) of the tiny cloud.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import digs_oracle as O

pytestmark = pytest.mark.gpu


def relL2(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def T(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()


def _sampled(wl, I, ids, n=96, seed=0):
    """Compare n pixels of each of three projections, half of them drawn where the image is bright."""
    rng = np.random.default_rng(seed)
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    got, ref = [], []
    for k in (0, len(ids) // 2, len(ids) - 1):
        img = I[k].cpu().numpy()
        nv, nu = img.shape
        bright = np.argwhere(img > 0.5 * img.max())
        pick = bright[rng.choice(len(bright), n // 2, replace=False)][:, ::-1]
        anyp = np.stack([rng.integers(0, nu, n // 2), rng.integers(0, nv, n // 2)], 1)
        pix = np.concatenate([pick, anyp], 0)
        ref.append(O.render_pixels(g, wl.lattice, wl.phi, wl.w, wl.views[ids[k]], wl.w[ids[k]], pix))
        got.append(img[pix[:, 1], pix[:, 0]])
    return np.concatenate(got), np.concatenate(ref)


def test_thorax_100k_projections_and_gradients():
    import paper_2506_22280_gb300 as pkg
    wl = synth.thorax(seed=1, n=100_000)
    ids = [int((j * 42) % 680) for j in range(16)]
    views = [wl.views[i] for i in ids]
    ins = [T(wl.mu0), T(wl.scale), T(wl.quat), T(wl.rho), T(wl.phi), T(wl.w[ids])]
    pj = pkg.Projector(wl.lattice, views, tile=16, bwd_lanes=16)
    I = pj.forward(*ins)
    assert pj.status() == 0
    got, ref = _sampled(wl, I, ids)
    assert relL2(got, ref) < 1e-5
    # one projection's full backward against the oracle (about a minute of FP64 CPU work at most)
    one = wl.select_views([ids[3]])
    p1 = pkg.Projector(wl.lattice, one.views, tile=16, bwd_lanes=16)
    gp = synth.random_grad_proj(1, 256, 256, seed=4)
    g = p1.backward(T(wl.mu0), T(wl.scale), T(wl.quat), T(wl.rho), T(wl.phi), T(one.w), T(gp))
    assert p1.status() == 0
    gref = O.project_vjp(dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho), wl.lattice, wl.phi, one.w,
                         one.views, gp)
    for k in ("mu0", "scale", "quat", "rho", "phi", "w"):
        assert relL2(g[k].cpu().numpy(), gref[k]) < 1e-4, (k, relL2(g[k].cpu().numpy(), gref[k]))


def test_scale_500k_512_projections_and_subset_gradients():
    import paper_2506_22280_gb300 as pkg
    wl = synth.scale()
    ids = [0, 170, 340, 510]
    views = [wl.views[i] for i in ids]
    pj = pkg.Projector(wl.lattice, views, tile=16)
    I = pj.forward(T(wl.mu0), T(wl.scale), T(wl.quat), T(wl.rho), T(wl.phi), T(wl.w[ids]))
    assert pj.status() == 0
    got, ref = _sampled(wl, I, ids, n=64)
    assert relL2(got, ref) < 1e-5
    sub = wl.subset(np.random.default_rng(7).choice(wl.n, 1000, replace=False)).select_views([ids[1], ids[2]])
    ps = pkg.Projector(sub.lattice, sub.views, tile=16)
    gp = synth.random_grad_proj(2, 512, 512, seed=6)
    g = ps.backward(T(sub.mu0), T(sub.scale), T(sub.quat), T(sub.rho), T(sub.phi), T(sub.w), T(gp))
    gref = O.project_vjp(dict(mu0=sub.mu0, scale=sub.scale, quat=sub.quat, rho=sub.rho), sub.lattice, sub.phi,
                         sub.w, sub.views, gp)
    for k in ("mu0", "scale", "quat", "rho", "phi", "w"):
        assert relL2(g[k].cpu().numpy(), gref[k]) < 1e-4, (k, relL2(g[k].cpu().numpy(), gref[k]))


def test_largest_call_128_projections():
    import paper_2506_22280_gb300 as pkg
    from paper_2506_22280_gb300 import digs as D
    wl = synth.tiny(n=500, n_proj=D.DIGS_MAX_VIEWS)
    pj = pkg.Projector(wl.lattice, wl.views)
    I = pj.forward(T(wl.mu0), T(wl.scale), T(wl.quat), T(wl.rho), T(wl.phi), T(wl.w))
    ref = O.render(dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho), wl.lattice, wl.phi, wl.w, wl.views)
    assert relL2(I.cpu().numpy(), ref) < 1e-5
