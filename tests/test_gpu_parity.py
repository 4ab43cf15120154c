"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances (rel-L2 = ||x_gpu - x_ref|| / ||x_ref|| over the whole tensor): projections <= 1e-5,
every gradient tensor <= 1e-4, the same 3.5-sigma cutoff on both sides.  The FP32 kernels evaluate each
pair with ~1e-6 relative error (a handful of roundings of O(1) quantities plus the approximate rsqrt /
exp2), and a cutoff flip changes a pixel by at most exp(-12.25/2) ~ 0.2 % of one Gaussian's peak, so
both bounds leave an order of magnitude of margin at these sizes.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import digs_oracle as O

pytestmark = pytest.mark.gpu


def relL2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def dev():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch.device("cuda:0")


@pytest.fixture(scope="module")
def P():
    import paper_2506_22280_gb300 as pkg
    pkg.lib()
    return pkg


def T(a, dev):
    return torch.as_tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous()


def gpu_inputs(wl, dev):
    return [T(wl.mu0, dev), T(wl.scale, dev), T(wl.quat, dev), T(wl.rho, dev), T(wl.phi, dev), T(wl.w, dev)]


def gauss(wl):
    return dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho)


# ----------------------------------------------------------------------------- FFD
def test_ffd_eval_matches_oracle(dev, P):
    wl = synth.tiny()
    rng = np.random.default_rng(0)
    x = np.concatenate([wl.mu0[:500], rng.uniform(-60, 60, size=(300, 3))])  # incl. points outside the lattice
    U, dU = P.ffd_eval(T(wl.phi, dev), wl.lattice, T(x, dev))
    Uo, dUo = O.ffd_eval(torch.tensor(wl.phi), wl.lattice, torch.tensor(x))
    assert relL2(U.cpu().numpy(), Uo.numpy()) < 1e-6
    assert relL2(dU.cpu().numpy(), dUo.numpy()) < 1e-6


# ----------------------------------------------------------------------------- forward
@pytest.fixture(scope="module")
def tiny_ref():
    wl = synth.tiny()
    proj = O.render(gauss(wl), wl.lattice, wl.phi, wl.w, wl.views)
    return wl, proj


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_project_fwd_tiny(dev, P, tiny_ref, tile):
    wl, ref = tiny_ref
    pj = P.Projector(wl.lattice, wl.views, tile=tile)
    out = pj.forward(*gpu_inputs(wl, dev))
    assert pj.status() == 0
    e = relL2(out.cpu().numpy(), ref)
    assert e < 1e-5, e


def test_project_fwd_ragged_detector_offsets_and_parallel(dev, P):
    wl = synth.tiny(n=600, n_proj=3, nu=61, nv=47)
    views = [dict(v) for v in wl.views]
    views[1]["off_u"], views[1]["off_v"] = 2.5, -1.25
    views[2]["parallel"] = True
    wl.views = views
    ref = O.render(gauss(wl), wl.lattice, wl.phi, wl.w, wl.views)
    for tile in (8, 32):
        out = P.Projector(wl.lattice, wl.views, tile=tile).forward(*gpu_inputs(wl, dev))
        for b in range(3):
            assert relL2(out[b].cpu().numpy(), ref[b]) < 1e-5, (tile, b)


def test_project_fwd_binning_paths(dev, P):
    # 16-pixel tiles on 288 x 256: 288 tiles per projection, the counting-sort binning; 8-pixel tiles:
    # 1152 tiles, beyond its limit, so the emitted pairs go through the radix sort
    wl = synth.tiny(n=300, n_proj=2, nu=288, nv=256)
    ref = O.render(gauss(wl), wl.lattice, wl.phi, wl.w, wl.views)
    for tile in (16, 8):
        out = P.Projector(wl.lattice, wl.views, tile=tile).forward(*gpu_inputs(wl, dev))
        for b in range(2):
            assert relL2(out[b].cpu().numpy(), ref[b]) < 1e-5, (tile, b)


def test_project_fwd_degenerate_cases(dev, P):
    wl = synth.tiny(n=50, n_proj=2)
    # one Gaussian exactly at a tile corner, one far off the detector, one folded by the deformation
    wl.mu0[0] = [0.0, 0.0, 0.0]
    wl.mu0[1] = [0.0, 0.0, 400.0]
    ref = O.render(gauss(wl), wl.lattice, wl.phi, wl.w, wl.views)
    out = P.Projector(wl.lattice, wl.views).forward(*gpu_inputs(wl, dev))
    assert relL2(out.cpu().numpy(), ref) < 1e-5
    # zero weights: the deformation is the identity
    w0 = np.zeros_like(wl.w)
    ref0 = O.render(gauss(wl), wl.lattice, wl.phi, w0, wl.views)
    ins = gpu_inputs(wl, dev)
    ins[5] = T(w0, dev)
    assert relL2(P.Projector(wl.lattice, wl.views).forward(*ins).cpu().numpy(), ref0) < 1e-5
    # folded: a weight so large that det K <= 0 for some Gaussians; both sides drop them
    wbig = wl.w * 40.0
    refb = O.render(gauss(wl), wl.lattice, wl.phi, wbig, wl.views)
    ins[5] = T(wbig, dev)
    outb = P.Projector(wl.lattice, wl.views).forward(*ins).cpu().numpy()
    assert relL2(outb, refb) < 1e-5
    # single Gaussian, single projection
    w1 = wl.subset([2]).select_views([1])
    r1 = O.render(gauss(w1), w1.lattice, w1.phi, w1.w, w1.views)
    o1 = P.Projector(w1.lattice, w1.views).forward(*gpu_inputs(w1, dev))
    assert relL2(o1.cpu().numpy(), r1) < 1e-5


def test_project_fwd_amplitude_range(dev, P):
    # the forward folds |amp| into each entry's quadratic form when 2^-40 <= |amp| <= 2^40 and applies
    # the sign in the accumulation; outside that range (and for amp = 0) it multiplies by amp instead.
    # Densities of mixed sign with zeros, and whole clouds scaled far below and far above that range.
    wl = synth.tiny(n=800, n_proj=4)
    rng = np.random.default_rng(31)
    base = wl.rho.copy()
    cases = {"mixed": base * rng.choice([1.0, -1.0, 0.0], size=base.shape),
             "tiny": base * 1e-30, "huge": base * 1e25}
    for name, rho in cases.items():
        wl.rho = rho.astype(np.float32)
        ref = O.render(gauss(wl), wl.lattice, wl.phi, wl.w, wl.views)
        out = P.Projector(wl.lattice, wl.views).forward(*gpu_inputs(wl, dev))
        assert np.isfinite(out.cpu().numpy()).all(), name
        e = relL2(out.cpu().numpy(), ref)
        assert e < 1e-5, (name, e)


def test_project_fwd_empty_cloud(dev, P):
    wl = synth.tiny(n=5, n_proj=2).subset([])
    pj = P.Projector(wl.lattice, wl.views)
    out = pj.forward(*gpu_inputs(wl, dev))
    assert out.shape == (2, 64, 64) and float(out.abs().max()) == 0.0


# ----------------------------------------------------------------------------- backward
@pytest.fixture(scope="module")
def tiny_grad_ref():
    wl = synth.tiny().select_views([0, 3, 7, 12])
    gp = synth.random_grad_proj(4, 64, 64, seed=11)
    grads = O.project_vjp(gauss(wl), wl.lattice, wl.phi, wl.w, wl.views, gp)
    return wl, gp, grads


@pytest.mark.parametrize("tile,lanes", [(16, 16), (32, 16), (16, 32), (8, 32)])
def test_project_bwd_tiny(dev, P, tiny_grad_ref, tile, lanes):
    wl, gp, ref = tiny_grad_ref
    pj = P.Projector(wl.lattice, wl.views, tile=tile, bwd_lanes=lanes)
    g = pj.backward(*gpu_inputs(wl, dev), T(gp, dev))
    assert pj.status() == 0
    for k in ("mu0", "scale", "quat", "rho", "phi", "w"):
        e = relL2(g[k].cpu().numpy(), ref[k])
        assert e < 1e-4, (k, e)


def test_project_bwd_reuses_forward_binning(dev, P, tiny_grad_ref):
    wl, gp, ref = tiny_grad_ref
    pj = P.Projector(wl.lattice, wl.views)
    ins = gpu_inputs(wl, dev)
    pj.forward(*ins)
    g = pj.backward(*ins, T(gp, dev), reuse=True)
    for k in ("mu0", "scale", "quat", "rho", "phi", "w"):
        assert relL2(g[k].cpu().numpy(), ref[k]) < 1e-4, k


def test_autograd_function(dev, P):
    wl = synth.tiny(n=300).select_views([1, 9])
    pj = P.Projector(wl.lattice, wl.views)
    ins = [t.requires_grad_(True) for t in gpu_inputs(wl, dev)]
    out = P.DigsRender.apply(pj, *ins)
    gp = synth.random_grad_proj(2, 64, 64, seed=5)
    (out * T(gp, dev)).sum().backward()
    ref = O.project_vjp(gauss(wl), wl.lattice, wl.phi, wl.w, wl.views, gp)
    for k, t in zip(("mu0", "scale", "quat", "rho", "phi", "w"), ins):
        assert relL2(t.grad.cpu().numpy(), ref[k]) < 1e-4, k


def test_capacity_overflow_is_reported_not_faulted(dev, P):
    wl = synth.tiny(n=200, n_proj=2)
    pj = P.Projector(wl.lattice, wl.views)
    ins = gpu_inputs(wl, dev)
    pj.cap = 10  # far fewer pairs than needed
    pj.ws.ensure(pj._size(200, 10))
    pj.forward(*ins)
    assert pj.status() == 3  # DIGS_ERR_CAPACITY, reported on the host
    assert pj.status() == 0  # and cleared
    pj.reserve(*ins, force=True)
    wl_ref = O.render(gauss(wl), wl.lattice, wl.phi, wl.w, wl.views)
    assert relL2(pj.forward(*ins).cpu().numpy(), wl_ref) < 1e-5
