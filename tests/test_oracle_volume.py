"""Pins of the oracle's evaluation volumes: the voxelised mass of one Gaussian against its closed form
(with the chi-square-3 mass fraction inside the cutoff), the peak value at the mean, zero weights leave
the cloud undeformed, a constant control field moves the volume rigidly, and the DVF of affine control
points is the affine field itself."""
import math

import numpy as np
from scipy.special import gammainc

import synth
from oracle import digs_oracle as O


def _one(mu, scale, rho=0.02):
    return dict(mu0=np.array([mu]), scale=np.array([scale]), quat=np.array([[1.0, 0.2, -0.3, 0.1]]),
                rho=np.array([rho]))


def test_voxelised_mass_and_peak():
    lat = dict(nx=4, ny=4, nz=4, R=1, origin=[-30.0, -30.0, -30.0], spacing=[20.0, 20.0, 20.0])
    phi = np.zeros((1, 4, 4, 4, 3))
    grid = dict(nx=41, ny=41, nz=41, origin=[-10.0, -10.0, -10.0], spacing=[0.5, 0.5, 0.5])
    g = _one([0.0, 0.0, 0.0], [1.5, 2.0, 1.2])
    vol = O.voxelize(g, lat, phi, [0.0], grid, cutoff=3.5)
    mass = vol.sum() * 0.5 ** 3
    full = 0.02 * (2 * math.pi) ** 1.5 * 1.5 * 2.0 * 1.2
    frac = gammainc(1.5, 12.25 / 2)               # P(chi2_3 <= 3.5^2)
    assert abs(mass / (full * frac) - 1) < 2e-3
    assert np.isclose(vol[20, 20, 20], 0.02)      # the mean sits on a voxel centre
    nocut = O.voxelize(g, lat, phi, [0.0], grid, cutoff=None)
    assert abs(nocut.sum() * 0.5 ** 3 / full - 1) < 2e-3


def test_zero_weights_and_rigid_translation():
    wl = synth.tiny(n=40)
    grid = dict(nx=16, ny=16, nz=16, origin=[-30.0, -30.0, -30.0], spacing=[4.0, 4.0, 4.0])
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    zero = O.voxelize(g, wl.lattice, wl.phi, [0.0, 0.0], grid)
    undeformed = O.voxelize(g, wl.lattice, np.zeros_like(wl.phi), [1.0, -0.5], grid)
    assert np.allclose(zero, undeformed, atol=1e-15)
    # a constant displacement of 4 mm in x on every node (inside the lattice) shifts the volume by one voxel
    lat = dict(nx=8, ny=8, nz=8, R=1, origin=[-70.0, -70.0, -70.0], spacing=[20.0, 20.0, 20.0])
    phi = np.zeros((1, 8, 8, 8, 3))
    phi[..., 0] = 4.0
    base = O.voxelize(g, lat, np.zeros_like(phi), [0.0], grid)
    moved = O.voxelize(g, lat, phi, [1.0], grid)
    assert np.allclose(moved[:, :, 1:], base[:, :, :-1], atol=1e-12)


def test_dvf_of_affine_control_points():
    lat = dict(nx=8, ny=8, nz=8, R=2, origin=[-35.0, -35.0, -35.0], spacing=[10.0, 10.0, 10.0])
    A = np.array([[0.01, 0.02, 0.0], [0.0, -0.03, 0.01], [0.02, 0.0, 0.01]])
    t = np.array([0.5, -1.0, 2.0])
    k, j, i = np.meshgrid(np.arange(8), np.arange(8), np.arange(8), indexing="ij")
    nodes = np.stack([-35 + 10 * i, -35 + 10 * j, -35 + 10 * k], -1).astype(float)
    phi = np.zeros((2, 8, 8, 8, 3))
    phi[0] = nodes @ A.T + t
    phi[1] = 2.0 * (nodes @ A.T + t)
    grid = dict(nx=5, ny=5, nz=5, origin=[-10.0, -10.0, -10.0], spacing=[5.0, 5.0, 5.0])
    d = O.dvf(lat, phi, [0.5, 0.25], grid)
    X = O.grid_centres(grid).numpy()
    assert np.allclose(d, 1.0 * (X @ A.T + t), atol=1e-10)
