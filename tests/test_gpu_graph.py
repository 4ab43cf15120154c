"""A step captured in a CUDA graph and replayed (device-side step counter) does what the same step does
when called directly: the same parameters, Adam moments and losses after the same sequence of batches."""
import numpy as np
import pytest
import torch

import synth
from oracle import digs_oracle as O

pytestmark = pytest.mark.gpu

LR0 = [0.02, 0.005, 0.002, 0.01, 0.02, 0.01]
LR1 = [x / 10 for x in LR0]


@pytest.fixture(scope="module")
def P():
    assert torch.cuda.is_available()
    import paper_2506_22280_gb300 as pkg
    pkg.lib()
    return pkg


def _rec(P, wl):
    from paper_2506_22280_gb300 import digs as D
    return P.Reconstruction(wl.mu0, wl.scale, wl.quat, wl.rho, wl.phi, wl.w, wl.lattice,
                            D.adam_config(LR0, LR1, 40))


def test_graph_replay_matches_direct_steps(P):
    wl = synth.tiny()
    ref = synth.tiny(motion_seed=77)
    meas = O.render(dict(mu0=ref.mu0 + 0.3, scale=ref.scale, quat=ref.quat, rho=ref.rho * 1.1), ref.lattice,
                    ref.phi, ref.w, ref.views)
    batches = [[0, 5, 9, 13], [2, 6, 10, 14], [1, 7, 11, 15], [3, 4, 8, 12]]
    M = [torch.as_tensor(meas[b], dtype=torch.float32, device="cuda").contiguous() for b in batches]
    V = [[wl.views[i] for i in b] for b in batches]
    a, g = _rec(P, wl), _rec(P, wl)
    # one direct step each (sizes the workspace, initialises the kernels)
    a.step(M[0], batches[0], V[0])
    g.step(M[0], batches[0], V[0])
    graphs = g.capture([(M[k], batches[k], V[k]) for k in range(1, 4)])
    la, lg = [], []
    for rnd in range(2):
        for k in range(1, 4):
            la.append(float(a.step(M[k], batches[k], V[k]).item()))
            graphs[k - 1].replay()
            lg.append(float(g.loss.item()))
    torch.cuda.synchronize()
    assert a.status() == 0 and g.status() == 0
    assert a.iter == g.iter == 7
    assert np.allclose(la, lg, rtol=1e-5), (la, lg)
    # the control-point gradient is summed with float atomics, so the two runs may differ in rounding;
    # Adam can turn a rounding-level difference of a near-zero gradient into a full step, hence the
    # element fraction rather than every element
    for k in ("mu0", "scale", "quat", "rho", "phi", "w", "m", "v"):
        x, y = getattr(a, k).cpu().numpy(), getattr(g, k).cpu().numpy()
        ok = np.isclose(x, y, rtol=1e-4, atol=1e-6 * (np.abs(x).max() + 1e-30))
        assert ok.mean() > 0.999, (k, ok.mean())
