"""digs_project_fwd_static: the forward projection for callers that cannot allocate device memory.

Its scratch is a fixed 32 MiB array inside the library, so a caller that has no way to call cudaMalloc
(a plug-in whose host owns the device memory, a fixed memory budget) can still project.  This test calls
it through the C-ABI, twice in a row and on two different problems, and checks each result against the
workspace-based digs_project_fwd and against the FP64 oracle within the projection tolerance used
everywhere else (rel-L2 1e-5); then checks that a problem too large for the array is refused before
anything runs, and that a problem whose pairs overflow the array reports DIGS_ERR_CAPACITY while the next
call starts clean.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from oracle import digs_oracle as O

pytestmark = pytest.mark.gpu


def _relL2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _setup():
    assert torch.cuda.is_available(), "needs a GPU"
    from paper_2506_22280_gb300 import digs as D
    L = D.lib()
    f = L.digs_project_fwd_static
    f.restype = C.c_int
    f.argtypes = [C.c_void_p] * 5 + [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
    return D, f


def _tensors(wl):
    t = lambda a: torch.as_tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()
    return [t(wl.mu0), t(wl.scale), t(wl.quat), t(wl.rho), t(wl.phi), t(wl.w)]


def _call_static(D, f, wl, ins, out):
    g = D.gauss_struct(*ins[:4])
    lat = D.lattice_struct(wl.lattice)
    varr = D.views_array(wl.views)
    opts = D.opts_struct()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return f(C.byref(g), C.byref(lat), C.c_void_p(ins[4].data_ptr()), C.c_void_p(ins[5].data_ptr()), varr,
             len(wl.views), C.byref(opts), C.c_void_p(out.data_ptr()), stream)


def _oracle(wl):
    return O.render(dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho), wl.lattice, wl.phi, wl.w, wl.views)


def test_static_scratch_forward_matches_workspace_forward():
    D, f = _setup()
    first = synth.tiny()                                   # 2,000 Gaussians, 16 views of 64 x 64
    second = synth.tiny(seed=3, n=700, n_proj=3, nu=61, nv=47)
    refs = {id(first): _oracle(first), id(second): _oracle(second)}
    for wl in (first, second, first):                      # consecutive calls reuse the same array
        ins = _tensors(wl)
        ref = D.Projector(wl.lattice, wl.views).forward(*ins)
        out = torch.full_like(ref, float("nan"))
        assert _call_static(D, f, wl, ins, out) == 0
        torch.cuda.synchronize()
        assert torch.isfinite(out).all()
        got = out.cpu().numpy()
        assert _relL2(got, ref.cpu().numpy()) <= 1e-5
        assert _relL2(got, refs[id(wl)]) <= 1e-5


def test_static_scratch_refuses_oversized_problem():
    D, f = _setup()
    # 128 views of 256 x 256 need 64 MiB of per-pixel scratch alone: refused with DIGS_ERR_ARG
    wl = synth.tiny(n=10, n_proj=128, nu=256, nv=256)
    ins = _tensors(wl)
    out = torch.zeros(128, 256, 256, device="cuda")
    assert _call_static(D, f, wl, ins, out) == 1
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0


def test_static_scratch_pair_overflow_then_clean_call():
    D, f = _setup()
    # 1,000 wide Gaussians (scales x 8) seen from 128 views of 64 x 64: every record covers most of the
    # 16 tiles of its view, about 2 M (tile, Gaussian) pairs, more than the array holds after the
    # pair-independent part (about 20 MB of the 32 MiB)
    big = synth.tiny(seed=4, n=1000, n_proj=128)
    big.scale = big.scale * 8.0
    fixed = D.workspace_size(big.n, 128, 64, 64, big.R, 0)
    assert fixed < (32 << 20)
    ins = _tensors(big)
    out = torch.zeros(128, 64, 64, device="cuda")
    assert _call_static(D, f, big, ins, out) == 3           # DIGS_ERR_CAPACITY
    torch.cuda.synchronize()
    assert torch.isfinite(out).all()
    small = synth.tiny(seed=6, n=500, n_proj=4)
    ins = _tensors(small)
    out = torch.full((4, 64, 64), float("nan"), device="cuda")
    assert _call_static(D, f, small, ins, out) == 0
    torch.cuda.synchronize()
    ref = D.Projector(small.lattice, small.views).forward(*ins)
    assert _relL2(out.cpu().numpy(), ref.cpu().numpy()) <= 1e-5
    assert _relL2(out.cpu().numpy(), _oracle(small)) <= 1e-5
