"""Device-detected errors reach the host as status codes, without faulting the GPU and without leaving
non-finite output, and a later call on the same workspace is clean.

* A non-finite reference parameter (a mean, scale, quaternion or density that is NaN or infinite) makes
  the projection set-up drop that Gaussian and record DIGS_ERR_NONFINITE; digs_sync_status reports it
  and clears it.  The projection is then that of the cloud without the Gaussian (checked against the
  oracle with the row removed) and stays finite.
* The tensor-core GEMM's bounded mbarrier waits: with the K-loop wait limit set to zero tests, every
  wait of the loop gives up at once, the kernel drains its own tensor-core operations (with the default
  bound), frees its tensor memory and sets the status word to 1; with the default limit restored, the
  next GEMM is correct and leaves the status at 0.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import digs_oracle as O
from oracle import cnn_oracle as CO

pytestmark = pytest.mark.gpu

DIGS_ERR_NONFINITE = 5


def relL2(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def T(a):
    return torch.as_tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous()


@pytest.fixture(scope="module")
def pkg():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2506_22280_gb300 as P
    P.lib()
    return P


@pytest.mark.parametrize("field,row,col,value", [("mu0", 5, 1, np.nan), ("scale", 11, 2, np.inf),
                                                 ("rho", 17, None, np.nan), ("quat", 23, 0, -np.inf)])
def test_nonfinite_parameter_is_reported_and_dropped(pkg, field, row, col, value):
    wl = synth.tiny(n=300, n_proj=3)
    bad = {k: np.array(getattr(wl, k)) for k in ("mu0", "scale", "quat", "rho")}
    if col is None:
        bad[field][row] = value
    else:
        bad[field][row, col] = value
    pj = pkg.Projector(wl.lattice, wl.views)
    out = pj.forward(T(bad["mu0"]), T(bad["scale"]), T(bad["quat"]), T(bad["rho"]), T(wl.phi), T(wl.w))
    assert pj.status() == DIGS_ERR_NONFINITE
    img = out.cpu().numpy()
    assert np.isfinite(img).all()
    keep = np.arange(wl.n) != row
    ref = O.render(dict(mu0=wl.mu0[keep], scale=wl.scale[keep], quat=wl.quat[keep], rho=wl.rho[keep]), wl.lattice,
                   wl.phi, wl.w, wl.views)
    assert relL2(img, ref) < 1e-5
    # the status was cleared by the read; a clean call on the same workspace reports nothing
    out2 = pj.forward(T(wl.mu0), T(wl.scale), T(wl.quat), T(wl.rho), T(wl.phi), T(wl.w))
    assert pj.status() == 0
    full = O.render(dict(mu0=wl.mu0, scale=wl.scale, quat=wl.quat, rho=wl.rho), wl.lattice, wl.phi, wl.w, wl.views)
    assert relL2(out2.cpu().numpy(), full) < 1e-5


def _gemm_bound_ok(c, a, b):
    """Every element within the FP32 summation bound of the product of the BF16-rounded operands."""
    ref = CO.gemm_bf16(a, b, trans_b=True)
    absref = CO.gemm_bf16(np.abs(a), np.abs(b), trans_b=True)
    K = a.shape[1]
    return bool(np.all(np.abs(c - ref) <= 4 * K * 2.0 ** -24 * absref + 1e-30))


def test_gemm_wait_give_up_sets_status_and_next_gemm_is_correct(pkg):
    from paper_2506_22280_gb300 import digs as D
    rng = np.random.default_rng(5)
    a = rng.normal(size=(300, 1152)).astype(np.float32)   # 18 K slices: the loop waits from slice 2 on
    b = rng.normal(size=(130, 1152)).astype(np.float32)
    try:
        D.set_wait_limit(0)
        _, st = D.gemm_bf16(T(a), T(b), trans_b=True)
        torch.cuda.synchronize()
        assert int(st.item()) == 1
    finally:
        D.set_wait_limit(-1)
    c, st = D.gemm_bf16(T(a), T(b), trans_b=True)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    assert _gemm_bound_ok(c.cpu().numpy().astype(np.float64), a, b)
