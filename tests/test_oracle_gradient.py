"""Pins of the oracle's gradient (autograd of the FP64 definition) and of its Adam step.

* Central finite differences of the FP64 forward with the cutoff off (a smooth function) against the
  oracle's gradient for every input group (means, scales, quaternions, densities, phi, w).
* Identities the gradient must satisfy whatever the input: q . dL/dq = 0 (normalised quaternions),
  sum_n rho_n dL/drho_n = sum_pix I dL/dI (linearity in rho), and for each rank
  sum_t w_tr dL/dw_tr = sum_k phi_rk . dL/dphi_rk (the rank-scaling symmetry of Eq. 9).
* Adam: the first step moves every element by lr g / (|g| + eps), and a scalar trajectory against
  the textbook recurrences evaluated by hand.
"""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import digs_oracle as O


def _small_case(seed=0, n=10, cutoff=None):
    wl = synth.tiny(seed=seed, n=n, n_proj=2, nu=14, nv=12, du=4.0, dv=4.0)
    lat = dict(nx=5, ny=5, nz=5, R=2, origin=np.array([-40.0] * 3), spacing=np.array([20.0] * 3))
    rng = np.random.default_rng(seed + 5)
    phi = rng.normal(0, 1.5, size=(2, 5, 5, 5, 3))
    return wl, lat, phi


def _loss(wl, lat, inputs, grad_proj, cutoff):
    g = dict(mu0=inputs["mu0"], scale=inputs["scale"], quat=inputs["quat"], rho=inputs["rho"])
    I = O.render(g, lat, inputs["phi"], inputs["w"], wl.views, cutoff=cutoff, mode="brute")
    return float(np.sum(I * grad_proj))


@pytest.mark.parametrize("key", ["mu0", "scale", "quat", "rho", "phi", "w"])
def test_gradient_matches_central_differences(key):
    wl, lat, phi = _small_case()
    inputs = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho, phi=phi, w=wl.w)
    gp = synth.random_grad_proj(2, 12, 14, seed=9)
    grads = O.project_vjp(dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho), lat, phi, wl.w,
                          wl.views, gp, cutoff=None, mode="brute")
    x = inputs[key]
    flat = x.ravel()
    rng = np.random.default_rng(1)
    idx = rng.choice(flat.size, min(flat.size, 12), replace=False)
    for i in idx:
        # FP64 rounding of E = c - b^2/a leaves ~1e-11 relative noise in the loss, so a small step is
        # noise-bound; a Richardson-extrapolated central difference at h = 4e-3 keeps both the noise
        # (~1e-9) and the O(h^4) truncation error far below the bound
        h = 4e-3 * max(1.0, abs(flat[i]))

        def central(hh):
            xp, xm = flat.copy(), flat.copy()
            xp[i] += hh
            xm[i] -= hh
            fp = _loss(wl, lat, dict(inputs, **{key: xp.reshape(x.shape)}), gp, None)
            fm = _loss(wl, lat, dict(inputs, **{key: xm.reshape(x.shape)}), gp, None)
            return (fp - fm) / (2 * hh)

        fd = (4 * central(h / 2) - central(h)) / 3
        an = grads[key].ravel()[i]
        scale_ = np.abs(grads[key]).max()
        assert abs(fd - an) <= 1e-6 * scale_ + 1e-6 * abs(an), (key, i, fd, an)


def test_gradient_identities_with_cutoff():
    wl = synth.tiny().subset(np.arange(150)).select_views([0, 6, 13])
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    gp = synth.random_grad_proj(3, 64, 64, seed=4)
    grads = O.project_vjp(g, wl.lattice, wl.phi, wl.w, wl.views, gp)
    I = O.render(g, wl.lattice, wl.phi, wl.w, wl.views)
    # quaternions are normalised inside: the gradient is orthogonal to q
    qdot = np.sum(grads["quat"] * wl.quat, 1)
    assert np.abs(qdot).max() <= 1e-10 * np.abs(grads["quat"]).max() * np.abs(wl.quat).max()
    # linearity in rho
    lhs = np.sum(wl.rho * grads["rho"])
    rhs = np.sum(I * gp)
    assert abs(lhs - rhs) <= 1e-10 * np.sum(np.abs(I * gp))
    # rank-scaling symmetry: d/dalpha of I(alpha w_r, phi_r / alpha) = 0
    for r in range(wl.R):
        a = np.sum(wl.w[:, r] * grads["w"][:, r])
        b = np.sum(wl.phi[r] * grads["phi"][r])
        assert abs(a - b) <= 1e-9 * (abs(a) + abs(b) + 1e-30), (r, a, b)


def test_adam_first_step_and_scalar_trajectory():
    rng = np.random.default_rng(2)
    g = rng.normal(size=50)
    p0 = rng.normal(size=50)
    lr, b1, b2, eps = 0.01, 0.9, 0.999, 1e-15
    p1, m1, v1 = O.adam_update(p0, g, np.zeros(50), np.zeros(50), 1, lr, b1, b2, eps)
    assert np.allclose(p1, p0 - lr * g / (np.abs(g) + eps), rtol=0, atol=1e-15)
    # scalar: gradients 1, -2, 0.5 over three steps, recurrences expanded by hand
    p, m, v = 0.3, 0.0, 0.0
    for t, gt in enumerate([1.0, -2.0, 0.5], start=1):
        p, m, v = O.adam_update(p, gt, m, v, t, 0.1, 0.9, 0.99, 1e-8)
    m3 = 0.1 * 0.9 ** 2 * 1.0 + 0.1 * 0.9 * -2.0 + 0.1 * 0.5
    v3 = 0.01 * 0.99 ** 2 * 1.0 + 0.01 * 0.99 * 4.0 + 0.01 * 0.25
    assert abs(float(m) - m3) < 1e-15 and abs(float(v) - v3) < 1e-15
    assert O.lr_at(1e-2, 1e-3, 0, 100) == 1e-2 and abs(O.lr_at(1e-2, 1e-3, 99, 100) - 1e-3) < 1e-18


def test_reparameterised_adam():
    """Log and softplus re-parameterisations: the first step moves theta by -lr sign(g) exactly, so the
    physical parameter moves by the closed forms exp(-+lr) and the softplus of theta -+ lr; the chain-rule
    factor never changes a sign, so the move follows -sign(dL/dparam)."""
    rng = np.random.default_rng(4)
    s = rng.uniform(0.5, 3.0, 30)
    g = rng.normal(size=30)
    lr = 0.05
    s1, _, _ = O.adam_update_reparam(s, g, np.zeros(30), np.zeros(30), 1, lr, 0.9, 0.999, 1e-15, "log")
    assert np.allclose(s1, s * np.exp(-lr * np.sign(g)), rtol=1e-12)
    rho = rng.uniform(0.001, 0.05, 30)
    r1, _, _ = O.adam_update_reparam(rho, g, np.zeros(30), np.zeros(30), 1, lr, 0.9, 0.999, 1e-15, "softplus")
    theta = np.log(np.exp(rho) - 1)
    assert np.allclose(r1, np.log(1 + np.exp(theta - lr * np.sign(g))), rtol=1e-10)
    assert np.all(np.sign(r1 - rho) == -np.sign(g))
