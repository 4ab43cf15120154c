"""Several scans with uneven Gaussian counts in one digs_step (one launch per stage for all of them):
loss, every in-step gradient and the Adam update against the FP64 oracle run scan by scan."""
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


@pytest.fixture(scope="module")
def P():
    assert torch.cuda.is_available()
    import paper_2506_22280_gb300 as pkg
    pkg.lib()
    return pkg


def _scans():
    """Three tiny scans of 2000, 1100 and 600 Gaussians with their own motion, weights and measurements."""
    out = []
    for s, n in enumerate((2000, 1100, 600)):
        wl = synth.tiny(seed=10 + s, n=n)
        ref = synth.tiny(seed=10 + s, n=n, motion_seed=300 + s)
        g_meas = dict(mu0=ref.mu0 + 0.3, scale=ref.scale, quat=ref.quat, rho=ref.rho * 1.1)
        meas = O.render(g_meas, ref.lattice, ref.phi, ref.w, ref.views)
        out.append((wl, meas))
    return out


def _stack(P, scans, total=100):
    from paper_2506_22280_gb300 import digs as D
    cat = lambda k: np.concatenate([getattr(wl, k) for wl, _ in scans], 0)
    phi = np.stack([wl.phi for wl, _ in scans], 0)
    w = np.concatenate([wl.w for wl, _ in scans], 0)  # scan s, projection p -> row 16 s + p
    rec = P.Reconstruction(cat("mu0"), cat("scale"), cat("quat"), cat("rho"), phi, w, scans[0][0].lattice,
                           D.adam_config(LR0, LR1, total), scan_sizes=[wl.n for wl, _ in scans])
    return rec


# (scan, projection) items of one batch: uneven counts per scan, interleaved
BATCH = [(0, 0), (1, 3), (2, 7), (0, 5), (1, 9), (1, 12), (2, 2), (0, 11)]


def test_multiscan_step_matches_oracle_per_scan(P):
    scans = _scans()
    rec = _stack(P, scans)
    n_proj = len(scans[0][0].views)
    views, rows, M = [], [], []
    for s, p in BATCH:
        v = dict(scans[s][0].views[p])
        v["scan"] = s
        views.append(v)
        rows.append(n_proj * s + p)
        M.append(scans[s][1][p])
    Mt = torch.as_tensor(np.stack(M), dtype=torch.float32, device="cuda").contiguous()
    loss = float(rec.step(Mt, rows, views).item())
    assert rec.status() == 0
    grad = rec.grad.cpu().numpy().astype(np.float64)
    N = sum(wl.n for wl, _ in scans)
    nphi = scans[0][0].phi.size
    npix = float(len(BATCH) * M[0].size)
    sq = 0.0
    g_w_ref = np.zeros((len(scans) * n_proj, 2))
    for s, (wl, meas) in enumerate(scans):
        items = [k for k, (ss, _) in enumerate(BATCH) if ss == s]
        ids = [BATCH[k][1] for k in items]
        g = dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)
        I = O.render(g, wl.lattice, wl.phi, wl.w[ids], [wl.views[i] for i in ids])
        sq += float(((I - meas[ids]) ** 2).sum())
        ref = O.project_vjp(g, wl.lattice, wl.phi, wl.w[ids], [wl.views[i] for i in ids],
                            2.0 * (I - meas[ids]) / npix)
        a, b = rec.scan_off[s], rec.scan_off[s + 1]
        got = {"mu0": grad[3 * a:3 * b], "scale": grad[3 * N + 3 * a:3 * N + 3 * b],
               "quat": grad[6 * N + 4 * a:6 * N + 4 * b], "rho": grad[10 * N + a:10 * N + b],
               "phi": grad[11 * N + s * nphi:11 * N + (s + 1) * nphi]}
        for k in got:
            assert relL2(got[k], ref[k].ravel()) < 1e-4, (s, k, relL2(got[k], ref[k].ravel()))
        for j, i in enumerate(ids):
            g_w_ref[n_proj * s + i] += ref["w"][j]
    assert abs(loss - sq / npix) / (sq / npix) < 1e-5, (loss, sq / npix)
    g_w = grad[11 * N + len(scans) * nphi:].reshape(-1, 2)
    assert relL2(g_w, g_w_ref) < 1e-4


def test_multiscan_equals_single_scan_steps_for_one_scan_batches(P):
    """A batch drawn from one scan of a multi-scan state moves that scan's parameters exactly as a
    single-scan state holding only that scan would (same gradients; Adam state starts at zero)."""
    from paper_2506_22280_gb300 import digs as D
    scans = _scans()
    rec = _stack(P, scans)
    s, ids = 1, [2, 6, 10]
    wl = scans[s][0]
    views = [dict(wl.views[i], scan=s) for i in ids]
    M = torch.as_tensor(scans[s][1][ids], dtype=torch.float32, device="cuda").contiguous()
    rec.step(M, [16 * s + i for i in ids], views)
    one = P.Reconstruction(wl.mu0, wl.scale, wl.quat, wl.rho, wl.phi, wl.w, wl.lattice, D.adam_config(LR0, LR1, 100))
    one.step(M, ids, [wl.views[i] for i in ids])
    assert rec.status() == 0 and one.status() == 0
    a, b = rec.scan_off[s], rec.scan_off[s + 1]
    for k in ("mu0", "scale", "quat", "rho"):
        x = getattr(rec, k)[a:b].cpu().numpy()
        y = getattr(one, k).cpu().numpy()
        assert np.allclose(x, y, rtol=1e-5, atol=1e-6), k
    assert np.allclose(rec.phi[s].cpu().numpy().ravel(), one.phi.cpu().numpy().ravel(), rtol=1e-5, atol=1e-6)
    # the other scans' Gaussians and control points received no gradient and did not move
    for t in (0, 2):
        a2, b2 = rec.scan_off[t], rec.scan_off[t + 1]
        assert np.allclose(rec.mu0[a2:b2].cpu().numpy(), scans[t][0].mu0.astype(np.float32))
        assert np.allclose(rec.phi[t].cpu().numpy().ravel(), scans[t][0].phi.astype(np.float32).ravel())
