"""Pins of the density-control oracle: the plan's rules on hand-made Gaussians, mass conservation of
clone and split, the split children's positions, the output order, and the gradient statistic against
central finite differences of the loss in the deformed means."""
import numpy as np
import torch

import synth
from oracle import density_oracle as DO
from oracle import digs_oracle as O


def test_plan_rules_and_order():
    scale = np.array([[1, 1, 1], [3, 1, 1], [1, 1, 1], [1, 4, 1], [1, 1, 1.0]])
    rho = np.array([0.01, 0.01, 1e-9, 0.02, 0.01])
    g = np.array([5.0, 5.0, 5.0, 5.0, 0.1])            # tau * n = 1
    action, dst, n_out = DO.densify_plan(g, 10, scale, rho, tau=0.1, s_split=2.0, rho_min=1e-6)
    assert list(action) == [DO.CLONE, DO.SPLIT, DO.PRUNE, DO.SPLIT, DO.KEEP]
    assert list(dst) == [0, 2, 4, 4, 6] and n_out == 7
    # exactly at the threshold counts as reaching it; just below does not
    a2, _, _ = DO.densify_plan([1.0, np.nextafter(np.float32(1.0), np.float32(0))], 10, scale[:2], rho[:2],
                               tau=0.1, s_split=10.0, rho_min=0.0)
    assert list(a2) == [DO.CLONE, DO.KEEP]


def test_apply_conserves_mass_and_places_children():
    rng = np.random.default_rng(0)
    n = 6
    q = rng.normal(size=(n, 4))
    g = dict(mu0=rng.normal(size=(n, 3)) * 10, scale=rng.uniform(0.5, 3, size=(n, 3)), quat=q,
             rho=rng.uniform(0.01, 0.03, size=n))
    action = np.array([DO.KEEP, DO.CLONE, DO.SPLIT, DO.PRUNE, DO.SPLIT, DO.CLONE])
    size = np.array([1, 2, 2, 0, 2, 2])
    dst = np.concatenate([[0], np.cumsum(size)[:-1]])
    z = rng.normal(size=(n, 2, 3))
    out = DO.densify_apply(g, action, dst, int(size.sum()), z)
    mass = lambda r, s: r * np.prod(s, axis=1)
    kept = action != DO.PRUNE
    assert np.isclose(mass(out["rho"], out["scale"]).sum(), mass(g["rho"], g["scale"])[kept].sum(), rtol=1e-12)
    assert list(out["src"]) == [0, 1, 1, 2, 2, 4, 4, 5, 5] and list(out["new"]) == [0, 0, 1, 1, 1, 1, 1, 0, 1]
    # a split child sits at mu + R diag(s) z: its Mahalanobis offset from the parent is |z|
    Rm = O.quat_to_rotmat(torch.as_tensor(q / np.linalg.norm(q, axis=1, keepdims=True))).numpy()
    for j, (n_, i) in zip((3, 4), ((2, 0), (2, 1))):
        off = Rm[n_].T @ (out["mu0"][j] - g["mu0"][n_]) / g["scale"][n_]
        assert np.allclose(off, z[n_, i], atol=1e-12)
    assert np.allclose(out["scale"][3], g["scale"][2] / 1.6) and np.allclose(out["quat"][5], q[4])
    rows = rng.normal(size=(n, 3))
    gr = DO.gather_rows(out["src"], out["new"], rows)
    assert np.array_equal(gr[0], rows[0]) and np.all(gr[2] == 0) and np.array_equal(gr[7], rows[5])


def test_gradient_statistic_matches_finite_differences():
    wl = synth.tiny(n=60, n_proj=2)
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    meas = O.render(dict(g, mu0=wl.mu0 + 0.4), wl.lattice, wl.phi, wl.w, wl.views)
    got = DO.density_grad_sums(g, wl.lattice, wl.phi, wl.w, wl.views, meas)
    # reference: the same per-projection gradient by central differences of the loss in mu'_{b,n}
    T = O._inputs(g, wl.phi, wl.w)
    sigma0 = O.covariance(T["scale"], T["quat"])
    U, dU = O.ffd_eval(T["phi"], wl.lattice, T["mu0"])
    M = torch.as_tensor(meas)
    ref = np.zeros(len(wl.mu0))
    for b, view in enumerate(wl.views):
        v = O.view_tensors(view)
        mu, sigma, K = O.deform(T["mu0"], sigma0, U, dU, T["w"][b])
        P = torch.linalg.inv(sigma)
        alive = O.alive_mask(v, mu, P, K, 3.5)

        def loss(mu_):
            img = O.render_view_brute(v, mu_, P, T["rho"], alive, 3.5)
            return float(((img.reshape(v["nv"], v["nu"]) - M[b]) ** 2).sum() / M.numel())

        for n in range(0, len(wl.mu0), 7):
            grad = np.zeros(3)
            for c in range(3):
                h = 1e-4
                mp, mm = mu.clone(), mu.clone()
                mp[n, c] += h
                mm[n, c] -= h
                grad[c] = (loss(mp) - loss(mm)) / (2 * h)
            ref[n] += np.linalg.norm(grad)
    sel = np.arange(0, len(wl.mu0), 7)
    assert np.allclose(got[sel], ref[sel], rtol=2e-3, atol=1e-12 + 1e-3 * np.abs(ref[sel]).max())
    assert (got > 0).sum() > len(got) // 2
