"""Pins of the oracle's Gaussian, deformation and X-ray projection (Sec. 3.1-3.2, Eq. 2-4, 7-8).

Checks against closed forms and invariants: quaternion rotations, covariance spectrum, the line
integral of one Gaussian against numerical quadrature and textbook special cases, mass conservation
for parallel rays, brute force vs box enumeration, equivariance under rotation about the scan axis,
detector offsets, identity at zero weights, translation by a constant field, the push-forward of an
affine map, and the rank-scaling symmetry of the low-rank model.
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import digs_oracle as O

DT = torch.float64


def _one(mu, scale, quat, rho):
    return dict(mu0=np.atleast_2d(mu).astype(float), scale=np.atleast_2d(scale).astype(float),
                quat=np.atleast_2d(quat).astype(float), rho=np.atleast_1d(rho).astype(float))


def _static_lattice(R=1):
    return dict(nx=4, ny=4, nz=4, R=R, origin=np.array([-15.0] * 3), spacing=np.array([10.0] * 3))


def _zero_motion(R=1, P=1):
    return np.zeros((R, 4, 4, 4, 3)), np.zeros((P, R))


def test_quaternion_rotation_textbook():
    th = 0.7
    q = torch.tensor([[math.cos(th / 2), 0.0, 0.0, math.sin(th / 2)]], dtype=DT) * 3.0  # unnormalised
    R = O.quat_to_rotmat(q)[0].numpy()
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    assert np.allclose(R, Rz, atol=1e-15)
    qs = torch.tensor(np.random.default_rng(0).normal(size=(20, 4)))
    Rs = O.quat_to_rotmat(qs)
    assert torch.allclose(Rs @ Rs.transpose(-1, -2), torch.eye(3, dtype=DT).expand(20, 3, 3), atol=1e-14)
    assert torch.allclose(torch.linalg.det(Rs), torch.ones(20, dtype=DT), atol=1e-14)


def test_covariance_spectrum():
    rng = np.random.default_rng(1)
    s = torch.tensor(rng.uniform(0.5, 3.0, size=(10, 3)))
    q = torch.tensor(rng.normal(size=(10, 4)))
    ev = torch.linalg.eigvalsh(O.covariance(s, q))
    assert torch.allclose(ev, torch.sort(s * s, -1).values, atol=1e-12)


def _quad_line_integral(mu, sigma, rho, o, d, half=60.0, n=200001):
    """Simpson quadrature of rho exp(-1/2 (x-mu)^T Sigma^-1 (x-mu)) along x = o + s d around the
    point of the line nearest to mu."""
    P = np.linalg.inv(sigma)
    s0 = float(np.dot(mu - o, d))
    s = np.linspace(s0 - half, s0 + half, n)
    x = o[None] + s[:, None] * d[None]
    r = x - mu[None]
    f = rho * np.exp(-0.5 * np.einsum("ni,ij,nj->n", r, P, r))
    h = s[1] - s[0]
    return h / 3 * (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum())


def test_line_integral_matches_quadrature():
    """Cone-beam pixel values of single anisotropic Gaussians equal quadrature along the pixel ray."""
    rng = np.random.default_rng(2)
    views = synth.circular_views([0.4], 1000.0, 1500.0, 9, 7, 1.6, 1.6)
    v = O.view_tensors(views[0])
    X = O.pixel_centres(v).numpy()
    phi, w = _zero_motion()
    for trial in range(4):
        g = _one(rng.normal(0, 2.0, 3), rng.uniform(1.0, 3.0, 3), rng.normal(size=4), rng.uniform(0.01, 0.03))
        img = O.render(g, _static_lattice(), phi, w, views, cutoff=None, mode="brute")[0].ravel()
        sigma = O.covariance(torch.tensor(g["scale"]), torch.tensor(g["quat"]))[0].numpy()
        src = views[0]["src"]
        for p in rng.choice(X.shape[0], 6, replace=False):
            d = (X[p] - src) / np.linalg.norm(X[p] - src)
            ref = _quad_line_integral(g["mu0"][0], sigma, g["rho"][0], src, d)
            assert abs(img[p] - ref) <= 1e-10 * max(1.0, abs(ref)), (trial, p, img[p], ref)


def test_isotropic_and_principal_axis_closed_forms():
    sig, rho = 2.0, 0.02
    views = synth.circular_views([1.1], 1000.0, 1500.0, 33, 33, 0.5, 0.5)
    phi, w = _zero_motion()
    g = _one([0.0, 0.0, 0.0], [sig] * 3, [1, 0, 0, 0], rho)
    img = O.render(g, _static_lattice(), phi, w, views, cutoff=None, mode="brute")[0]
    # central pixel ray passes through the isocentre: rho sigma sqrt(2 pi)
    assert abs(img[16, 16] - rho * sig * math.sqrt(2 * math.pi)) < 1e-9 * rho * sig
    # any other pixel: distance delta from the centre to the ray, rho sigma sqrt(2 pi) exp(-delta^2 / 2 sigma^2)
    v = O.view_tensors(views[0])
    X = O.pixel_centres(v).numpy().reshape(33, 33, 3)
    s = views[0]["src"]
    for (j, i) in [(0, 0), (5, 20), (16, 30), (32, 1)]:
        dvec = (X[j, i] - s) / np.linalg.norm(X[j, i] - s)
        delta = np.linalg.norm(np.cross(-s, dvec))
        ref = rho * sig * math.sqrt(2 * math.pi) * math.exp(-delta ** 2 / (2 * sig ** 2))
        # E = c - b^2/a cancels two numbers of size (1000 mm / sigma)^2 ~ 2.5e5: ~1e-11 relative in FP64
        assert abs(img[j, i] - ref) < 1e-14 + 1e-9 * ref
    # anisotropic Gaussian whose principal axis k lies along the central ray: rho s_k sqrt(2 pi)
    ang = 1.1
    axis = np.array([math.cos(ang), math.sin(ang), 0.0])
    # rotate the x axis onto the ray direction: rotation about z by ang
    q = [math.cos(ang / 2), 0, 0, math.sin(ang / 2)]
    g2 = _one([0.0, 0.0, 0.0], [3.0, 1.0, 0.5], q, rho)
    img2 = O.render(g2, _static_lattice(), phi, w, views, cutoff=None, mode="brute")[0]
    assert abs(img2[16, 16] - rho * 3.0 * math.sqrt(2 * math.pi)) < 1e-9 * rho
    assert np.allclose(O.quat_to_rotmat(torch.tensor([q], dtype=DT))[0].numpy()[:, 0], axis)


def test_parallel_beam_mass_conservation():
    """Sum_pixels I du dv = integral of the Gaussian = rho (2 pi)^1.5 s1 s2 s3 (cutoff off); with the
    3.5-sigma cutoff the 2-D mass inside Mahalanobis radius 3.5 is the fraction 1 - exp(-12.25 / 2)."""
    du = 0.1
    views = synth.circular_views([0.3], 1000.0, 1500.0, 241, 241, du, du, parallel=True)
    phi, w = _zero_motion()
    s = np.array([2.0, 1.2, 1.5])
    g = _one([0.3, -0.2, 0.1], s, [0.9, 0.2, -0.3, 0.1], 0.02)
    total = 0.02 * (2 * math.pi) ** 1.5 * np.prod(s)
    img = O.render(g, _static_lattice(), phi, w, views, cutoff=None, mode="brute")[0]
    assert abs(img.sum() * du * du / total - 1) < 1e-9
    img_c = O.render(g, _static_lattice(), phi, w, views, cutoff=3.5, mode="bbox")[0]
    assert abs(img_c.sum() * du * du / (total * (1 - math.exp(-12.25 / 2))) - 1) < 2e-3


def test_brute_equals_bbox_on_tiny():
    wl = synth.tiny().subset(np.arange(300)).select_views([0, 5, 11])
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    a = O.render(g, wl.lattice, wl.phi, wl.w, wl.views, mode="brute")
    b = O.render(g, wl.lattice, wl.phi, wl.w, wl.views, mode="bbox")
    # equal up to FP64 rounding of E = c - b^2/a (the two modes contract in different orders)
    assert np.allclose(a, b, rtol=1e-9, atol=1e-15)
    # the same pairs contribute: counting pairs per Gaussian individually
    for n in (0, 17, 123):
        wn = wl.subset([n])
        gn = dict(mu0=wn.mu0, scale=wn.scale, quat=wn.quat, rho=wn.rho)
        an = O.render(gn, wl.lattice, wl.phi, wl.w, wl.views, mode="brute")
        bn = O.render(gn, wl.lattice, wl.phi, wl.w, wl.views, mode="bbox")
        assert np.array_equal(an > 0, bn > 0)


def test_cone_equivariance_under_rotation_about_scan_axis():
    """Rotating the cloud by alpha about z is the same as moving the gantry back by alpha."""
    wl = synth.tiny().subset(np.arange(200))
    alpha = 0.37
    c, s = math.cos(alpha), math.sin(alpha)
    Rz = np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])
    qa = np.array([math.cos(alpha / 2), 0, 0, math.sin(alpha / 2)])
    q = wl.quat
    # Hamilton product qa * q
    w1, x1, y1, z1 = qa
    w2, x2, y2, z2 = q.T
    qr = np.stack([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                   w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2], 1)
    phi, w = _zero_motion(P=1)
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    g_rot = dict(mu0=wl.mu0 @ Rz.T, scale=wl.scale, quat=qr, rho=wl.rho)
    th = 0.9
    # cutoff off: a pair sitting on E = 12.25 could otherwise flip under FP64 rounding
    a = O.render(g_rot, _static_lattice(), phi, w, synth.circular_views([th], 1000, 1500, 48, 40, 1.6, 1.6),
                 cutoff=None)
    b = O.render(g, _static_lattice(), phi, w, synth.circular_views([th - alpha], 1000, 1500, 48, 40, 1.6, 1.6),
                 cutoff=None)
    assert np.allclose(a, b, rtol=1e-9, atol=1e-13)


def test_linearity_in_density_and_detector_offset():
    wl = synth.tiny().subset(np.arange(150)).select_views([3])
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    a = O.render(g, wl.lattice, wl.phi, wl.w, wl.views)
    g2 = dict(g, rho=2.5 * wl.rho)
    assert np.allclose(O.render(g2, wl.lattice, wl.phi, wl.w, wl.views), 2.5 * a, rtol=1e-13, atol=0)
    vo = [dict(wl.views[0], off_u=3.0, off_v=-2.0)]
    b = O.render(g, wl.lattice, wl.phi, wl.w, vo)
    # pixel (i, j) of the offset detector sits where pixel (i + 3, j - 2) sits without offset
    assert np.allclose(b[0, 2:, :-3], a[0, :-2, 3:], rtol=1e-9, atol=1e-14)


def test_zero_weights_is_identity_and_constant_field_translates():
    wl = synth.tiny().subset(np.arange(120)).select_views([2, 9])
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    static = O.render(g, _static_lattice(2), np.zeros((2, 4, 4, 4, 3)), np.zeros((2, 2)), wl.views)
    a = O.render(g, wl.lattice, wl.phi, np.zeros_like(wl.w), wl.views)
    assert np.allclose(a, static, rtol=1e-13, atol=1e-16)
    # constant control displacements t_r on a lattice wide enough that every Gaussian is interior
    lat = dict(nx=12, ny=12, nz=12, R=2, origin=np.array([-60.0] * 3), spacing=np.array([11.0] * 3))
    t = np.array([[1.5, -0.5, 2.0], [0.3, 0.7, -1.1]])
    phi = np.broadcast_to(t[:, None, None, None, :], (2, 12, 12, 12, 3)).copy()
    b = O.render(g, lat, phi, wl.w, wl.views, cutoff=None, mode="brute")
    for p in range(2):
        shift = wl.w[p] @ t
        gp = dict(g, mu0=wl.mu0 + shift)
        ref = O.render(gp, _static_lattice(2), np.zeros((2, 4, 4, 4, 3)), np.zeros((1, 2)), [wl.views[p]],
                       cutoff=None, mode="brute")
        assert np.allclose(b[p], ref[0], rtol=1e-9, atol=1e-14)


def test_affine_field_pushes_gaussian_forward():
    """For an affine FFD D(x) = K x + t the warped Gaussian is the push-forward of the reference one:
    the covariance of mapped samples converges to the oracle's K Sigma0 K^T and the mean to mu'."""
    rng = np.random.default_rng(7)
    lat = dict(nx=10, ny=10, nz=10, R=1, origin=np.array([-45.0] * 3), spacing=np.array([10.0] * 3))
    xs = lat["origin"][0] + 10.0 * np.arange(10)
    Z, Y, X = np.meshgrid(xs, xs, xs, indexing="ij")
    nodes = np.stack([X, Y, Z], -1)
    A = np.array([[0.1, 0.05, 0.0], [-0.02, 0.2, 0.03], [0.01, 0.0, -0.15]])
    tt = np.array([1.0, -2.0, 0.5])
    phi = (nodes @ A.T + tt)[None]
    mu0 = np.array([[1.0, 2.0, -3.0]])
    s = np.array([[2.0, 1.0, 0.7]])
    q = np.array([[0.8, 0.3, -0.2, 0.4]])
    w_b = torch.tensor([0.8], dtype=DT)
    U, dU = O.ffd_eval(torch.tensor(phi), lat, torch.tensor(mu0))
    sig0 = O.covariance(torch.tensor(s), torch.tensor(q))
    mu, sigma, K = O.deform(torch.tensor(mu0), sig0, U, dU, w_b)
    L = np.linalg.cholesky(sig0[0].numpy())
    smp = mu0[0] + rng.normal(size=(400000, 3)) @ L.T
    mapped = smp + 0.8 * (smp @ A.T + tt)
    assert np.allclose(mapped.mean(0), mu[0].numpy(), atol=0.02)
    assert np.allclose(np.cov(mapped.T), sigma[0].numpy(), atol=0.03 * np.abs(sigma[0].numpy()).max())
    assert np.allclose(K[0].numpy(), np.eye(3) + 0.8 * A, atol=1e-13)


def test_rank_scaling_symmetry():
    """(w_r, phi_r) -> (alpha w_r, phi_r / alpha) leaves every projection unchanged (Eq. 9)."""
    wl = synth.tiny().subset(np.arange(150)).select_views([1, 7])
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    a = O.render(g, wl.lattice, wl.phi, wl.w, wl.views, cutoff=None, mode="brute")
    phi2 = wl.phi.copy()
    w2 = wl.w.copy()
    phi2[1] /= 2.5
    w2[:, 1] *= 2.5
    b = O.render(g, wl.lattice, phi2, w2, wl.views, cutoff=None, mode="brute")
    assert np.allclose(a, b, rtol=1e-9, atol=1e-15)


def test_render_pixels_matches_full_render():
    wl = synth.tiny().subset(np.arange(200)).select_views([4])
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    full = O.render(g, wl.lattice, wl.phi, wl.w, wl.views)[0]
    ij = np.array([[0, 0], [31, 32], [40, 10], [63, 63], [12, 50]])
    vals = O.render_pixels(g, wl.lattice, wl.phi, wl.w, wl.views[0], wl.w[0], ij)
    assert np.allclose(vals, full[ij[:, 1], ij[:, 0]], rtol=1e-9, atol=1e-15)


def test_mse_loss_is_the_mean_over_every_pixel_of_every_projection():
    # two 1 x 2 projections, residuals 1, 0, -2, 0: the mean of the squares over the four pixels is 5 / 4
    # (the sum would give 5, per-projection means summed 2.5, the root of the mean 1.118)
    I = np.array([[[1.0, 2.0]], [[3.0, 4.0]]])
    M = np.array([[[0.0, 2.0]], [[5.0, 4.0]]])
    assert O.mse_loss(I, M) == 1.25
    assert O.mse_loss(M, M) == 0.0


def test_gaussians_behind_the_source_or_around_it_are_dropped():
    views = synth.circular_views([0.4], 1000.0, 1500.0, 17, 17, 4.0, 4.0)
    v = O.view_tensors(views[0])
    src = np.asarray(views[0]["src"], dtype=float)
    phi, w = _zero_motion()
    lat = _static_lattice()
    # behind the source: the whole line through the source and a pixel would meet it, but it lies on the
    # far side of the source from the detector
    behind = _one(1.2 * src, [5.0] * 3, [1, 0, 0, 0], 0.02)
    front = _one(0.2 * src, [5.0] * 3, [1, 0, 0, 0], 0.02)
    for cut in (3.5, None):
        assert np.abs(O.render(behind, lat, phi, w, views, cutoff=cut, mode="brute")).max() == 0.0
        assert O.render(front, lat, phi, w, views, cutoff=cut, mode="brute").max() > 0.0
    # a Gaussian whose cutoff ellipsoid holds the source (Mahalanobis distance of the source
    # 1000 / 400 = 2.5 < 3.5) is dropped with the cutoff on; at 1000 / 250 = 4 > 3.5 it is kept
    wide = _one([0.0, 0.0, 0.0], [400.0] * 3, [1, 0, 0, 0], 1e-4)
    kept = _one([0.0, 0.0, 0.0], [250.0] * 3, [1, 0, 0, 0], 1e-4)
    assert np.abs(O.render(wide, lat, phi, w, views, cutoff=3.5, mode="brute")).max() == 0.0
    assert O.render(wide, lat, phi, w, views, cutoff=None, mode="brute").max() > 0.0
    assert O.render(kept, lat, phi, w, views, cutoff=3.5, mode="brute").max() > 0.0
    # the mask itself on the three cases
    mu = torch.tensor(np.stack([1.2 * src, 0.2 * src, np.zeros(3)]), dtype=DT)
    sig = torch.tensor([5.0, 5.0, 400.0], dtype=DT)
    P = torch.diag_embed((1.0 / sig ** 2)[:, None].expand(3, 3))
    K = torch.eye(3, dtype=DT).expand(3, 3, 3)
    assert O.alive_mask(v, mu, P, K, 3.5).tolist() == [False, True, False]
    assert O.alive_mask(v, mu, P, K, None).tolist() == [False, True, True]


def test_cutoff_margin_of_an_isotropic_gaussian():
    # isotropic sigma at the isocentre: E of a pixel ray is (distance from the ray to the centre / sigma)^2
    sig = 2.0
    views = synth.circular_views([0.7, 2.1], 1000.0, 1500.0, 31, 29, 0.5, 0.5)
    phi, w = _zero_motion(P=2)
    g = _one([0.0, 0.0, 0.0], [sig] * 3, [1, 0, 0, 0], 0.02)
    got = O.cutoff_margin(g, _static_lattice(), phi, w, views)[0]
    best = np.inf
    for view in views:
        v = O.view_tensors(view)
        X = O.pixel_centres(v).numpy()
        s = np.asarray(view["src"], dtype=float)
        d = (X - s) / np.linalg.norm(X - s, axis=1, keepdims=True)
        dist = np.linalg.norm(np.cross(-s[None], d), axis=1)
        E = (dist / sig) ** 2
        near = E <= (1.05 * 3.5) ** 2
        best = min(best, float(np.min(np.abs(E[near] - 12.25) / 12.25)))
    assert abs(got - best) <= 1e-9 * max(best, 1e-12) + 1e-12, (got, best)
