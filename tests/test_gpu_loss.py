"""digs_project_loss: the forward projection with the L2 projection loss of Sec. 4.2 (mean over every
pixel of the call of (I - M)^2) summed inside the raster kernel, against the FP64 oracle; and the
warm start's full-scan loss, which adds the per-chunk losses of that call weighted by their sizes."""
import numpy as np
import pytest
import torch

import synth
from oracle import digs_oracle as O

pytestmark = pytest.mark.gpu


def T(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()


def _case(n_proj):
    wl = synth.tiny(n_proj=n_proj)
    ref = synth.tiny(n_proj=n_proj, motion_seed=9)
    meas = O.render(dict(mu0=ref.mu0 + 0.4, scale=ref.scale, quat=ref.quat, rho=ref.rho * 0.9), ref.lattice, ref.phi,
                    ref.w, ref.views)
    I = O.render(dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho), wl.lattice, wl.phi, wl.w, wl.views)
    return wl, meas, I


@pytest.mark.parametrize("n_proj", [3, 17])
def test_project_loss_matches_oracle(n_proj):
    import paper_2506_22280_gb300 as pkg
    wl, meas, I = _case(n_proj)
    pj = pkg.Projector(wl.lattice, wl.views)
    proj = torch.empty(n_proj, 64, 64, device="cuda")
    ins = [T(wl.mu0), T(wl.scale), T(wl.quat), T(wl.rho), T(wl.phi), T(wl.w)]
    loss = float(pj.loss(*ins, T(meas), proj=proj).item())
    assert pj.status() == 0
    L = O.mse_loss(I, meas)
    assert abs(loss - L) / L < 1e-5, (loss, L)
    assert np.linalg.norm(proj.cpu().numpy() - I) / np.linalg.norm(I) < 1e-5
    # without the projection output
    assert abs(float(pj.loss(*ins, T(meas)).item()) - L) / L < 1e-5


def test_scan_loss_over_uneven_chunks():
    import paper_2506_22280_gb300 as pkg
    from paper_2506_22280_gb300 import digs as D
    from paper_2506_22280_gb300 import warmstart as WS
    wl, meas, I = _case(40)
    rec = pkg.Reconstruction(wl.mu0, wl.scale, wl.quat, wl.rho, wl.phi, wl.w, wl.lattice,
                             D.adam_config([0.0] * 6, [0.0] * 6, 10))
    got = WS.scan_loss(rec, T(meas), wl.views, rec.w, chunk=16)  # chunks of 16, 16 and 8 views
    L = O.mse_loss(I, meas)
    assert abs(got - L) / L < 1e-5, (got, L)
