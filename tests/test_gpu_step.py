"""digs_step (render a batch, L2 loss, backward, fused Adam) against the FP64 oracle, and a short
reconstruction that must reduce the projection loss."""
import numpy as np
import pytest
import torch

import synth
from oracle import digs_oracle as O

pytestmark = pytest.mark.gpu

LR0 = [0.02, 0.005, 0.002, 0.01, 0.02, 0.01]
LR1 = [x / 10 for x in LR0]
KINDS = ["plain", "log", "plain", "softplus", "plain", "plain"]


def relL2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.fixture(scope="module")
def P():
    assert torch.cuda.is_available()
    import paper_2506_22280_gb300 as pkg
    pkg.lib()
    return pkg


def _setup(P, total=100):
    wl = synth.tiny()
    ref_state = synth.tiny(motion_seed=77)
    g_meas = dict(mu0=ref_state.mu0 + 0.3, scale=ref_state.scale, quat=ref_state.quat, rho=ref_state.rho * 1.1)
    meas = O.render(g_meas, ref_state.lattice, ref_state.phi, ref_state.w, ref_state.views)
    from paper_2506_22280_gb300 import digs as D
    rec = P.Reconstruction(wl.mu0, wl.scale, wl.quat, wl.rho, wl.phi, wl.w, wl.lattice,
                           D.adam_config(LR0, LR1, total))
    return wl, meas, rec


def test_step_loss_gradients_and_adam_update(P):
    wl, meas, rec = _setup(P)
    ids = [0, 5, 9, 13]
    views = [wl.views[i] for i in ids]
    M = torch.as_tensor(meas[ids], dtype=torch.float32, device="cuda").contiguous()
    loss = float(rec.step(M, ids, views).item())
    assert rec.status() == 0
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    I = O.render(g, wl.lattice, wl.phi, wl.w[ids], views)
    L = O.mse_loss(I, meas[ids])
    assert abs(loss - L) / L < 1e-5, (loss, L)
    gp = 2.0 * (I - meas[ids]) / I.size
    ref = O.project_vjp(g, wl.lattice, wl.phi, wl.w[ids], views, gp)
    n = wl.n
    nphi = wl.phi.size
    grad = rec.grad.cpu().numpy().astype(np.float64)
    parts = {"mu0": grad[:3 * n], "scale": grad[3 * n:6 * n], "quat": grad[6 * n:10 * n], "rho": grad[10 * n:11 * n],
             "phi": grad[11 * n:11 * n + nphi], "w": grad[11 * n + nphi:]}
    ref_w = np.zeros_like(wl.w)
    ref_w[ids] = ref["w"]
    refs = {"mu0": ref["mu0"].ravel(), "scale": ref["scale"].ravel(), "quat": ref["quat"].ravel(),
            "rho": ref["rho"].ravel(), "phi": ref["phi"].ravel(), "w": ref_w.ravel()}
    for k in parts:
        assert relL2(parts[k], refs[k]) < 1e-4, k
    # Adam, first step: every element with a clearly non-zero gradient moves as the oracle's update
    olds = {"mu0": wl.mu0, "scale": wl.scale, "quat": wl.quat, "rho": wl.rho, "phi": wl.phi, "w": wl.w}
    news = {"mu0": rec.mu0, "scale": rec.scale, "quat": rec.quat, "rho": rec.rho, "phi": rec.phi, "w": rec.w}
    for gi, k in enumerate(["mu0", "scale", "quat", "rho", "phi", "w"]):
        old = olds[k].ravel()
        gr = refs[k]
        expect, _, _ = O.adam_update_reparam(old, gr, np.zeros_like(old), np.zeros_like(old), 1, LR0[gi], 0.9, 0.999,
                                             1e-15, KINDS[gi])
        got = news[k].detach().cpu().numpy().astype(np.float64).ravel()
        big = np.abs(gr) > 1e-3 * np.abs(gr).max()
        tol = 1e-5 * (np.abs(old[big]) + LR0[gi]) + 1e-7
        ok = np.abs(got[big] - expect[big]) <= tol
        assert ok.mean() > 0.999, (k, ok.mean())
        assert np.allclose(got[gr == 0], old[gr == 0])


def test_short_reconstruction_reduces_loss(P):
    wl, meas, rec = _setup(P, total=60)
    losses = []
    rng = np.random.default_rng(0)
    for it in range(60):
        ids = sorted(rng.choice(16, 4, replace=False).tolist())
        M = torch.as_tensor(meas[ids], dtype=torch.float32, device="cuda").contiguous()
        losses.append(float(rec.step(M, ids, [wl.views[i] for i in ids]).item()))
    assert rec.status() == 0
    assert np.mean(losses[-5:]) < 0.5 * np.mean(losses[:5]), (losses[:5], losses[-5:])
