"""Parity at the batch shapes the benchmark runs: more projections per call than the per-Gaussian chain's
eight projection slots, so every slot takes several projections and adds their adjoints into its
shared-memory column (the chain rule through Eq. 7-11 of Sec. 3.2-3.3, summed over the batch).

* ``digs_project_bwd`` on the tiny cloud with P = 16 (two full slot groups) and P = 17 (a ragged third
  group holding one projection), all six gradients against the FP64 oracle.
* ``digs_step`` with B = 16, B = 17 and B = 128 (the benchmark's projections per step: 16 per slot):
  loss, the six in-step gradients and the first Adam update.
* One step over three scans of uneven Gaussian counts with B = 26 items (11 / 9 / 6 per scan).
* The 100k-Gaussian thorax with 16 and with the benchmark's 128 projections, tile 16 and 16 lanes per record: the
  gradients of a seeded 1,000-Gaussian subset against the oracle run on that subset with the same
  dL/dI (a Gaussian's own gradient depends only on its parameters, the motion model and dL/dI), plus
  three identities that hold at any size: q . dL/dq = 0 per Gaussian (the quaternion is normalised
  inside), sum_n rho_n dL/drho_n = sum_pix I dL/dI (I is linear in every rho_n) and, per rank,
  sum_b w_br dL/dw_br = sum_k phi_rk . dL/dphi_rk (the projections do not change under
  (w_r, phi_r) -> (a w_r, phi_r / a)).

Tolerances: rel-L2 over the whole tensor, projections and losses <= 1e-5, gradients <= 1e-4.  Gaussians
with a (pixel, view) pair within FP32 rounding of the cutoff (conftest.unambiguous) are left out of the
clouds, since the float32 kernels and the float64 oracle may decide such a pair differently.
"""
import numpy as np
import pytest
import torch

import synth
from conftest import unambiguous
from oracle import digs_oracle as O

pytestmark = pytest.mark.gpu

LR0 = [0.02, 0.005, 0.002, 0.01, 0.02, 0.01]
LR1 = [x / 10 for x in LR0]
KINDS = ["plain", "log", "plain", "softplus", "plain", "plain"]
GROUPS = ("mu0", "scale", "quat", "rho", "phi", "w")


def relL2(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def T(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()


def gauss(wl):
    return dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)


@pytest.fixture(scope="module")
def pkg():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2506_22280_gb300 as P
    P.lib()
    return P


@pytest.mark.parametrize("n_views", [16, 17])
def test_project_bwd_more_views_than_slots(pkg, n_views):
    wl = synth.tiny(n_proj=n_views)
    wl = wl.subset(unambiguous(wl, wl.w, wl.views))
    gp = synth.random_grad_proj(n_views, 64, 64, seed=11)
    pj = pkg.Projector(wl.lattice, wl.views, tile=16, bwd_lanes=16)
    ins = [T(wl.mu0), T(wl.scale), T(wl.quat), T(wl.rho), T(wl.phi), T(wl.w)]
    g = pj.backward(*ins, T(gp))
    assert pj.status() == 0
    ref = O.project_vjp(gauss(wl), wl.lattice, wl.phi, wl.w, wl.views, gp)
    for k in GROUPS:
        e = relL2(g[k].cpu().numpy(), ref[k])
        assert e < 1e-4, (n_views, k, e)
    # the same gradients when the backward reuses the forward's records
    pj.forward(*ins)
    g2 = pj.backward(*ins, T(gp), reuse=True)
    for k in GROUPS:
        assert relL2(g2[k].cpu().numpy(), ref[k]) < 1e-4, (n_views, k, "reuse")


def _split_grad(grad, n, nphi):
    return {"mu0": grad[:3 * n], "scale": grad[3 * n:6 * n], "quat": grad[6 * n:10 * n],
            "rho": grad[10 * n:11 * n], "phi": grad[11 * n:11 * n + nphi], "w": grad[11 * n + nphi:]}


@pytest.mark.parametrize("B", [16, 17, 128])
def test_step_batch_beyond_slots(pkg, B):
    from paper_2506_22280_gb300 import digs as D
    n_proj, n = (24, 2000) if B <= 17 else (136, 1000)
    wl = synth.tiny(n=n, n_proj=n_proj)
    ref_state = synth.tiny(n=n, n_proj=n_proj, motion_seed=77)
    g_meas = dict(mu0=ref_state.mu0 + 0.3, scale=ref_state.scale, quat=ref_state.quat, rho=ref_state.rho * 1.1)
    meas = O.render(g_meas, ref_state.lattice, ref_state.phi, ref_state.w, ref_state.views)
    ids = sorted(np.random.default_rng(B).choice(n_proj, B, replace=False).tolist())
    views = [wl.views[i] for i in ids]
    wl = wl.subset(unambiguous(wl, wl.w[ids], views))
    rec = pkg.Reconstruction(wl.mu0, wl.scale, wl.quat, wl.rho, wl.phi, wl.w, wl.lattice,
                             D.adam_config(LR0, LR1, 100))
    loss = float(rec.step(T(meas[ids]), ids, views).item())
    assert rec.status() == 0
    g = gauss(wl)
    I = O.render(g, wl.lattice, wl.phi, wl.w[ids], views)
    L = O.mse_loss(I, meas[ids])
    assert abs(loss - L) / L < 1e-5, (loss, L)
    ref = O.project_vjp(g, wl.lattice, wl.phi, wl.w[ids], views, 2.0 * (I - meas[ids]) / I.size)
    parts = _split_grad(rec.grad.cpu().numpy().astype(np.float64), wl.n, wl.phi.size)
    ref_w = np.zeros_like(wl.w)
    ref_w[ids] = ref["w"]
    refs = {k: ref[k].ravel() for k in GROUPS[:5]}
    refs["w"] = ref_w.ravel()
    for k in GROUPS:
        assert relL2(parts[k], refs[k]) < 1e-4, (B, k, relL2(parts[k], refs[k]))
    # first Adam step of every group with a clearly non-zero gradient
    olds = {"mu0": wl.mu0, "scale": wl.scale, "quat": wl.quat, "rho": wl.rho, "phi": wl.phi, "w": wl.w}
    news = {"mu0": rec.mu0, "scale": rec.scale, "quat": rec.quat, "rho": rec.rho, "phi": rec.phi, "w": rec.w}
    for gi, k in enumerate(GROUPS):
        old = olds[k].ravel()
        gr = refs[k]
        expect, _, _ = O.adam_update_reparam(old, gr, np.zeros_like(old), np.zeros_like(old), 1, LR0[gi], 0.9, 0.999,
                                             1e-15, KINDS[gi])
        got = news[k].detach().cpu().numpy().astype(np.float64).ravel()
        big = np.abs(gr) > 1e-3 * np.abs(gr).max()
        tol = 1e-5 * (np.abs(old[big]) + LR0[gi]) + 1e-7
        assert (np.abs(got[big] - expect[big]) <= tol).mean() > 0.999, k
        assert np.allclose(got[gr == 0], old[gr == 0])


def test_multiscan_step_26_items(pkg):
    from paper_2506_22280_gb300 import digs as D
    scans = []
    for s, n in enumerate((2000, 1100, 600)):
        wl = synth.tiny(seed=20 + s, n=n)
        ref = synth.tiny(seed=20 + s, n=n, motion_seed=400 + s)
        g_meas = dict(mu0=ref.mu0 + 0.3, scale=ref.scale, quat=ref.quat, rho=ref.rho * 1.1)
        scans.append((wl, O.render(g_meas, ref.lattice, ref.phi, ref.w, ref.views)))
    per_scan = {0: [0, 1, 3, 4, 6, 7, 9, 10, 12, 13, 15], 1: [0, 2, 5, 6, 8, 9, 11, 14, 15], 2: [1, 4, 7, 8, 11, 14]}
    scans = [(wl.subset(unambiguous(wl, wl.w[per_scan[s]], [wl.views[i] for i in per_scan[s]])), meas)
             for s, (wl, meas) in enumerate(scans)]
    cat = lambda k: np.concatenate([getattr(wl, k) for wl, _ in scans], 0)
    rec = pkg.Reconstruction(cat("mu0"), cat("scale"), cat("quat"), cat("rho"), np.stack([wl.phi for wl, _ in scans]),
                             np.concatenate([wl.w for wl, _ in scans]), scans[0][0].lattice,
                             D.adam_config(LR0, LR1, 100), scan_sizes=[wl.n for wl, _ in scans])
    batch = []
    for k in range(11):  # interleaved: scan 0, 1, 2, 0, 1, 2, ...
        for s in range(3):
            if k < len(per_scan[s]):
                batch.append((s, per_scan[s][k]))
    assert len(batch) == 26
    n_proj = 16
    views = [dict(scans[s][0].views[p], scan=s) for s, p in batch]
    rows = [n_proj * s + p for s, p in batch]
    M = np.stack([scans[s][1][p] for s, p in batch])
    loss = float(rec.step(T(M), rows, views).item())
    assert rec.status() == 0
    grad = rec.grad.cpu().numpy().astype(np.float64)
    N = sum(wl.n for wl, _ in scans)
    nphi = scans[0][0].phi.size
    npix = float(M.size)
    sq = 0.0
    g_w_ref = np.zeros((3 * n_proj, 2))
    for s, (wl, meas) in enumerate(scans):
        ids = [p for ss, p in batch if ss == s]
        vs = [wl.views[i] for i in ids]
        I = O.render(gauss(wl), wl.lattice, wl.phi, wl.w[ids], vs)
        sq += float(((I - meas[ids]) ** 2).sum())
        ref = O.project_vjp(gauss(wl), wl.lattice, wl.phi, wl.w[ids], vs, 2.0 * (I - meas[ids]) / npix)
        a, b = rec.scan_off[s], rec.scan_off[s + 1]
        got = {"mu0": grad[3 * a:3 * b], "scale": grad[3 * N + 3 * a:3 * N + 3 * b],
               "quat": grad[6 * N + 4 * a:6 * N + 4 * b], "rho": grad[10 * N + a:10 * N + b],
               "phi": grad[11 * N + s * nphi:11 * N + (s + 1) * nphi]}
        for k in got:
            assert relL2(got[k], ref[k].ravel()) < 1e-4, (s, k, relL2(got[k], ref[k].ravel()))
        for j, i in enumerate(ids):
            g_w_ref[n_proj * s + i] += ref["w"][j]
    assert abs(loss - sq / npix) / (sq / npix) < 1e-5, (loss, sq / npix)
    assert relL2(grad[11 * N + 3 * nphi:].reshape(-1, 2), g_w_ref) < 1e-4


@pytest.mark.parametrize("n_views", [16, 128])
def test_thorax_100k_subset_gradients_and_identities(pkg, n_views):
    wl = synth.thorax(seed=1, n=100_000)
    ids = [int((j * (680 // n_views)) % 680) for j in range(n_views)]
    one = wl.select_views(ids)
    gp = synth.random_grad_proj(n_views, 256, 256, seed=9)
    pj = pkg.Projector(wl.lattice, one.views, tile=16, bwd_lanes=16)
    ins = [T(wl.mu0), T(wl.scale), T(wl.quat), T(wl.rho), T(wl.phi), T(one.w)]
    I = pj.forward(*ins)
    g = pj.backward(*ins, T(gp), reuse=True)
    assert pj.status() == 0
    got = {k: g[k].cpu().numpy().astype(np.float64) for k in GROUPS}
    # a seeded 1,000-Gaussian subset against the oracle with the same dL/dI
    idx = np.sort(np.random.default_rng(7).choice(wl.n, 1000 if n_views <= 16 else 300, replace=False))
    idx = idx[unambiguous(one.subset(idx), one.w, one.views)]
    sub = one.subset(idx)
    ref = O.project_vjp(gauss(sub), sub.lattice, sub.phi, sub.w, sub.views, gp)
    for k in ("mu0", "scale", "quat", "rho"):
        e = relL2(got[k][idx], ref[k])
        assert e < 1e-4, (k, e)
    # q . dL/dq = 0 for every Gaussian
    q = wl.quat / np.linalg.norm(wl.quat, axis=1, keepdims=True)
    dots = np.abs((q * got["quat"]).sum(1))
    assert dots.max() <= 1e-4 * np.abs(got["quat"]).max() + 1e-12
    # sum_n rho_n dL/drho_n = sum_pix I dL/dI
    lhs = float((wl.rho * got["rho"]).sum())
    Ih = I.cpu().numpy().astype(np.float64)
    rhs = float((Ih * gp).sum())
    assert abs(lhs - rhs) <= 1e-4 * float(np.abs(Ih * gp).sum()), (lhs, rhs)
    # per rank: sum_b w_br dL/dw_br = sum_k phi_rk . dL/dphi_rk
    R = wl.R
    gw, gphi = got["w"].reshape(n_views, R), got["phi"].reshape(R, -1)
    phi = wl.phi.reshape(R, -1)
    for r in range(R):
        a = float((one.w[:, r] * gw[:, r]).sum())
        b = float((phi[r] * gphi[r]).sum())
        scale = float(np.abs(one.w[:, r] * gw[:, r]).sum() + np.abs(phi[r] * gphi[r]).sum())
        assert abs(a - b) <= 1e-3 * scale, (r, a, b)
