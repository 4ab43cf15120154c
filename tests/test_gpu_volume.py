"""Evaluation volumes through the C-ABI against the FP64 oracle: the attenuation volume of the deformed
cloud and the displacement field at one time point."""
import numpy as np
import pytest
import torch

import synth
from oracle import digs_oracle as O

pytestmark = pytest.mark.gpu


def relL2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


def T(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()


def test_voxelize_and_dvf_match_oracle():
    from paper_2506_22280_gb300 import digs as D
    wl = synth.tiny(n=300)
    grid = dict(nx=36, ny=30, nz=33, origin=[-34.0, -30.0, -32.0], spacing=[1.9, 2.1, 2.0])   # ragged, anisotropic
    w_row = wl.w[5]
    vol = D.voxelize(T(wl.mu0), T(wl.scale), T(wl.quat), T(wl.rho), T(wl.phi), T(w_row), wl.lattice, grid)
    ref = O.voxelize(dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho), wl.lattice, wl.phi, w_row, grid)
    assert relL2(vol.cpu().numpy(), ref) < 1e-5
    d = D.dvf(T(wl.phi), T(w_row), wl.lattice, grid)
    dref = O.dvf(wl.lattice, wl.phi, w_row, grid)
    assert relL2(d.cpu().numpy(), dref) < 1e-5
