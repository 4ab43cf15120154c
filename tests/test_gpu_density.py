"""Adaptive density control through the C-ABI against its FP64 oracle: the statistic digs_step
accumulates, the plan (bit for bit on the same inputs), the new cloud and the carried-over rows, and a
reconstruction that densifies and keeps stepping."""
import numpy as np
import pytest
import torch

import synth
from oracle import density_oracle as DO
from oracle import digs_oracle as O

pytestmark = pytest.mark.gpu

LR0 = [0.02, 0.005, 0.002, 0.01, 0.02, 0.01]


def relL2(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def T(a, dtype=torch.float32):
    return torch.as_tensor(np.asarray(a), dtype=dtype, device="cuda").contiguous()


def _rec(wl, total=100):
    from paper_2506_22280_gb300 import digs as D
    import paper_2506_22280_gb300 as pkg
    return pkg.Reconstruction(wl.mu0, wl.scale, wl.quat, wl.rho, wl.phi, wl.w, wl.lattice,
                              D.adam_config(LR0, [x / 10 for x in LR0], total))


def test_statistic_matches_oracle():
    wl = synth.tiny(n=600, n_proj=6)
    meas = O.render(dict(mu0=wl.mu0 + 0.3, scale=wl.scale, quat=wl.quat, rho=wl.rho * 1.1), wl.lattice, wl.phi,
                    wl.w, wl.views)
    rec = _rec(wl)
    rec.enable_density_stats()
    ids = [1, 4, 5]
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    ref = DO.density_grad_sums(g, wl.lattice, wl.phi, wl.w[ids], [wl.views[i] for i in ids], meas[ids])
    rec.step(T(meas[ids]), ids, [wl.views[i] for i in ids])
    got = rec.dens_grad.cpu().numpy()
    assert rec.status() == 0 and rec.dens_projections == 3
    assert relL2(got, ref) < 1e-4
    # a second step adds its own sums
    ref2 = DO.density_grad_sums(dict(mu0=rec.mu0.cpu().numpy(), scale=rec.scale.cpu().numpy(),
                                     quat=rec.quat.cpu().numpy(), rho=rec.rho.cpu().numpy()),
                                wl.lattice, rec.phi.cpu().numpy(), rec.w[[0, 2]].cpu().numpy(),
                                [wl.views[0], wl.views[2]], meas[[0, 2]])
    rec.step(T(meas[[0, 2]]), [0, 2], [wl.views[0], wl.views[2]])
    assert relL2(rec.dens_grad.cpu().numpy(), got + ref2) < 1e-4


def _random_cloud(n, seed):
    rng = np.random.default_rng(seed)
    return dict(mu0=rng.normal(size=(n, 3)) * 20, scale=rng.uniform(0.5, 6, size=(n, 3)),
                quat=rng.normal(size=(n, 4)), rho=rng.uniform(0.0, 0.03, size=n))


@pytest.mark.parametrize("n", [0, 1, 1000, 5000])
def test_plan_apply_gather_match_oracle(n):
    from paper_2506_22280_gb300 import digs as D
    g = {k: v.astype(np.float32) for k, v in _random_cloud(n, seed=n).items()}
    rng = np.random.default_rng(n + 1)
    grad = rng.uniform(0, 2, size=n).astype(np.float32)
    tau, n_proj, s_split, rho_min = 0.0625, 16, 4.0, 0.003     # threshold on the sum: 1.0
    grad[: n // 10] = np.float32(1.0)                            # exactly at the threshold
    action, dst = D.densify_plan(T(grad), T(g["scale"]), T(g["rho"]), tau, n_proj, s_split, rho_min)
    a_ref, d_ref, n_ref = DO.densify_plan(grad, n_proj, g["scale"], g["rho"], tau, s_split, rho_min)
    assert np.array_equal(action.cpu().numpy(), a_ref)
    assert np.array_equal(dst.cpu().numpy()[:n], d_ref) and int(dst[n].item()) == n_ref
    z = rng.normal(size=(n, 2, 3)).astype(np.float32)
    out = D.densify_apply(T(g["mu0"]), T(g["scale"]), T(g["quat"]), T(g["rho"]), action, dst, T(z), n_ref)
    ref = DO.densify_apply(g, a_ref, d_ref, n_ref, z)
    assert np.array_equal(out["src"].cpu().numpy(), ref["src"]) and np.array_equal(out["new"].cpu().numpy(), ref["new"])
    for k in ("mu0", "scale", "quat", "rho"):
        if n_ref:
            assert relL2(out[k].cpu().numpy(), ref[k]) < 1e-6, k
    rows = rng.normal(size=(n, 3)).astype(np.float32)
    if n_ref:
        got = D.gather_rows(out["src"], out["new"], T(rows)).cpu().numpy()
        assert np.array_equal(got, DO.gather_rows(ref["src"], ref["new"], rows).astype(np.float32))


def test_reconstruction_densifies_and_keeps_stepping():
    wl = synth.tiny(n=800, n_proj=8)
    meas = O.render(dict(mu0=wl.mu0 + 0.3, scale=wl.scale, quat=wl.quat, rho=wl.rho * 1.1), wl.lattice, wl.phi,
                    wl.w, wl.views)
    rec = _rec(wl)
    rec.enable_density_stats()
    plan = [[0, 3, 6], [1, 4, 7], [2, 5, 0]]
    for ids in plan:
        rec.step(T(meas[ids]), ids, [wl.views[i] for i in ids])
    n0 = int(rec.mu0.shape[0])
    stat = rec.dens_grad.cpu().numpy() / rec.dens_projections
    tau = float(np.quantile(stat, 0.9))                          # about a tenth of the cloud densifies
    m_before = rec.m.cpu().numpy().copy()
    rho0, s0 = rec.rho.cpu().numpy(), rec.scale.cpu().numpy()
    rho_min = float(np.quantile(rho0, 0.02))
    info = rec.densify(tau=tau, s_split=2.5, rho_min=rho_min, generator=torch.Generator(device="cuda").manual_seed(0))
    n1 = int(rec.mu0.shape[0])
    assert info["cloned"] + info["split"] > 0 and info["pruned"] > 0
    assert n1 == n0 - info["pruned"] + info["cloned"] + info["split"] == info["n_after"]
    # the integrated mass of everything that was not pruned is conserved
    kept = rho0 >= np.float32(rho_min)
    mass = lambda r, s: (r.astype(np.float64) * s.astype(np.float64).prod(1)).sum()
    assert abs(mass(rec.rho.cpu().numpy(), rec.scale.cpu().numpy()) - mass(rho0[kept], s0[kept])) < 1e-5 * mass(rho0, s0)
    # the moments of kept rows carried over, new rows zero; the control-point and weight moments unchanged
    m_after = rec.m.cpu().numpy()
    assert np.array_equal(m_after[11 * n1:], m_before[11 * n0:])
    # and the reconstruction keeps stepping
    for ids in plan:
        loss = float(rec.step(T(meas[ids]), ids, [wl.views[i] for i in ids]).item())
        assert np.isfinite(loss)
    assert rec.status() == 0 and rec.dens_projections == 9 and rec.dens_grad.shape[0] == n1
