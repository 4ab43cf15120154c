"""Pins of the oracle's 2D-Gaussian (EWA) projection model: for a Gaussian on the central ray the
bias-corrected amplitude is the exact line integral through it; with a distant source the model tends
to the exact projection (the paper's statement that they coincide for parallel rays); it is linear in
the density; and its gradient matches central differences."""
import math

import numpy as np

import synth
from oracle import digs_oracle as O


def _single(mu, scale, quat=(1.0, 0.0, 0.0, 0.0), rho=0.02):
    return dict(mu0=np.array([mu], float), scale=np.array([scale], float), quat=np.array([quat], float),
                rho=np.array([rho]))


def _static():
    lat = dict(nx=4, ny=4, nz=4, R=1, origin=[-30.0, -30.0, -30.0], spacing=[20.0, 20.0, 20.0])
    return lat, np.zeros((1, 4, 4, 4, 3)), np.zeros((1, 1))


def test_central_isotropic_gaussian_amplitude_is_the_line_integral():
    lat, phi, w = _static()
    v = synth.circular_views([0.3], 1000.0, 1500.0, 33, 33, 1.0, 1.0)
    g = _single([0.0, 0.0, 0.0], [2.0, 2.0, 2.0])
    ewa = O.render_ewa(g, lat, phi, w, v)
    exact = O.render(g, lat, phi, w, v, mode="brute")
    assert np.isclose(ewa[0, 16, 16], 0.02 * 2.0 * math.sqrt(2 * math.pi), rtol=1e-12)
    assert np.isclose(ewa[0, 16, 16], exact[0, 16, 16], rtol=1e-9)


def test_distant_source_tends_to_the_exact_projection():
    lat, phi, w = _static()
    g = _single([3.0, -2.0, 4.0], [2.5, 1.5, 3.0], quat=(0.9, 0.2, -0.3, 0.25))
    errs = []
    for sad in (1e3, 1e5):
        v = synth.circular_views([0.7], sad, 1.5 * sad, 48, 48, 0.8 * 1.5, 0.8 * 1.5)   # magnification 1.5
        ewa = O.render_ewa(g, lat, phi, w, v, cutoff=None)
        exact = O.render(g, lat, phi, w, v, cutoff=None, mode="brute")
        errs.append(np.abs(ewa - exact).max() / exact.max())
    assert errs[1] < 1e-4 and errs[1] < 0.05 * errs[0], errs


def test_linear_in_density_and_gradient_matches_differences():
    wl = synth.tiny(n=6).select_views([2])
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    I1 = O.render_ewa(g, wl.lattice, wl.phi, wl.w, wl.views, cutoff=None)
    I2 = O.render_ewa(dict(g, rho=2 * wl.rho), wl.lattice, wl.phi, wl.w, wl.views, cutoff=None)
    assert np.allclose(I2, 2 * I1, rtol=1e-12)
    gp = np.random.default_rng(0).normal(size=I1.shape)
    grads = O.project_vjp_ewa(g, wl.lattice, wl.phi, wl.w, wl.views, gp, cutoff=None)
    f = lambda gg, phi=wl.phi, w=wl.w: float((O.render_ewa(gg, wl.lattice, phi, w, wl.views, cutoff=None) * gp).sum())
    h = 1e-5
    for key, idx in (("mu0", (2, 1)), ("scale", (4, 0)), ("quat", (1, 2)), ("rho", (3,))):
        a, b = {k: v.copy() for k, v in g.items()}, {k: v.copy() for k, v in g.items()}
        a[key][idx] += h
        b[key][idx] -= h
        fd = (f(a) - f(b)) / (2 * h)
        assert abs(fd - grads[key][idx]) <= 1e-5 * max(1.0, abs(fd)), (key, fd, grads[key][idx])
