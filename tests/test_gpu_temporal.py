"""digs_step with the weights given by temporal B-spline control points (Sec. 4.2): loss and the
gradient of the control points against the FP64 oracle (the oracle's temporal B-spline, differentiated
by autograd through its own projection), and the Adam update of the control points."""
import numpy as np
import pytest
import torch

import synth
from oracle import digs_oracle as O

pytestmark = pytest.mark.gpu

LR0 = [0.02, 0.005, 0.002, 0.01, 0.02, 0.01]
LR1 = [x / 10 for x in LR0]


def relL2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def test_step_with_temporal_control_points():
    import paper_2506_22280_gb300 as pkg
    from paper_2506_22280_gb300 import digs as D
    wl = synth.tiny()
    ref = synth.tiny(motion_seed=77)
    meas = O.render(dict(mu0=ref.mu0 + 0.3, scale=ref.scale, quat=ref.quat, rho=ref.rho * 1.1), ref.lattice, ref.phi,
                    ref.w, ref.views)
    t_step = 4.0
    n_ctrl = int(np.floor((len(wl.views) - 1) / t_step)) + 4
    ctrl = np.random.default_rng(3).normal(0, 0.8, size=(n_ctrl, 2))
    rec = pkg.Reconstruction(wl.mu0, wl.scale, wl.quat, wl.rho, wl.phi, np.zeros_like(wl.w), wl.lattice,
                             D.adam_config(LR0, LR1, 100), w_ctrl=ctrl, t_step=t_step)
    ids = [0, 5, 9, 13, 5]   # a repeated projection: its row's gradient counts once per occurrence
    views = [wl.views[i] for i in ids]
    M = torch.as_tensor(meas[ids], dtype=torch.float32, device="cuda").contiguous()
    loss = float(rec.step(M, ids, views).item())
    assert rec.status() == 0
    g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
    c = torch.tensor(ctrl, dtype=torch.float64, requires_grad=True)
    w_rows = O.temporal_weights(c, t_step, ids)
    I = O.render(g, wl.lattice, wl.phi, w_rows.detach().numpy(), views)
    L = O.mse_loss(I, meas[ids])
    assert abs(loss - L) / L < 1e-5, (loss, L)
    gp = 2.0 * (I - meas[ids]) / I.size
    gw = O.project_vjp(g, wl.lattice, wl.phi, w_rows.detach().numpy(), views, gp)["w"]
    (w_rows * torch.as_tensor(gw)).sum().backward()
    n, nphi = wl.n, wl.phi.size
    got = rec.grad.cpu().numpy().astype(np.float64)[11 * n + nphi:]
    assert got.size == n_ctrl * 2
    assert relL2(got, c.grad.numpy().ravel()) < 1e-4
    # the evaluated rows of w and the first Adam step of the control points
    assert np.allclose(rec.w[ids].cpu().numpy(), w_rows.detach().numpy(), rtol=1e-5, atol=1e-6)
    moved = rec.w_ctrl.cpu().numpy().astype(np.float64) - ctrl
    big = np.abs(c.grad.numpy()) > 1e-3 * np.abs(c.grad.numpy()).max()
    assert np.allclose(moved[big], -LR0[5] * np.sign(c.grad.numpy()[big]), rtol=1e-3)
