"""The weight-predictor CNN's kernels (through the C-ABI) against the FP64 oracle: FP32 forward and
parameter gradient; the tensor-core forward and gradient against the oracle with the same operands
rounded to bfloat16 (batch 6, and batch 64 for multi-tile and split-reduction launches), on parameters
whose ReLU decisions are not at the mercy of rounding; BF16 inference; the input 2x2 average;
initialisation statistics; and training (FP32 and tensor-core) that fits a fixed batch."""
import numpy as np
import pytest
import torch

from oracle import cnn_oracle as C

pytestmark = pytest.mark.gpu

R = 3


def relL2(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def P():
    assert torch.cuda.is_available()
    import paper_2506_22280_gb300 as pkg
    pkg.lib()
    return pkg


def _inputs(B, seed=0):
    rng = np.random.default_rng(seed)
    img = rng.uniform(0.0, 1.0, size=(B, 128, 128)).astype(np.float32)
    th = rng.uniform(0, 2 * np.pi, size=B)
    cs = np.stack([np.cos(th), np.sin(th)], 1).astype(np.float32)
    return img, cs


def _biased(net):
    """Non-zero biases so that the test also covers them."""
    n = net.params.numel()
    off = 0
    p = net.params.cpu().numpy()
    rng = np.random.default_rng(5)
    for name, shape in C.param_shapes(R):
        k = int(np.prod(shape))
        if name.startswith("b"):
            p[off:off + k] = rng.normal(0, 0.05, size=k)
        off += k
    assert off == n
    net.params.copy_(torch.as_tensor(p))


def test_init_statistics(P):
    net = P.WeightPredictor(R, seed=3)
    p = net.params.cpu().numpy().astype(np.float64)
    off = 0
    for name, shape in C.param_shapes(R):
        k = int(np.prod(shape))
        x = p[off:off + k]
        if name.startswith("b"):
            assert np.all(x == 0)
        elif k > 2000:
            std = np.sqrt(2.0 / np.prod(shape[1:]))
            assert abs(x.std() / std - 1) < 0.05 and abs(x.mean()) < 0.05 * std, name
        off += k


def test_forward_and_gradient_match_oracle(P):
    net = P.WeightPredictor(R, seed=1)
    _biased(net)
    img, cs = _inputs(6)
    out = net.forward(torch.as_tensor(img, device="cuda"), torch.as_tensor(cs, device="cuda"))
    flat = net.params.cpu().numpy().astype(np.float64)
    ref = C.forward(flat, R, img, cs)
    assert relL2(out.cpu().numpy(), ref) < 1e-5
    gw = np.random.default_rng(2).normal(size=(6, R)).astype(np.float32)
    g = net.backward(torch.as_tensor(gw, device="cuda")).cpu().numpy()
    gref = C.vjp(flat, R, img, cs, gw)
    off = 0
    for name, shape in C.param_shapes(R):
        k = int(np.prod(shape))
        assert relL2(g[off:off + k], gref[off:off + k]) < 1e-4, name
        off += k


def _stable_masks(net, seed):
    """Parameters whose every ReLU decision is fixed by construction: biases +-4 per unit, weights 0.05 x
    He-normal, so each pre-activation lies about 20 standard deviations from zero on the bias's side.
    A ReLU whose input sits within rounding of zero is decided by rounding (float32 kernels, float64
    oracle), and one such flip moves a gradient by 1e-3 ... 1e-1; here both sides take every decision
    alike, and what remains is FP32 summation and activations on a bfloat16 rounding boundary."""
    rng = np.random.default_rng(seed)
    p = np.zeros(net.params.numel(), dtype=np.float64)
    off = 0
    for name, shape in C.param_shapes(R):
        k = int(np.prod(shape))
        if name.startswith("w"):
            p[off:off + k] = 0.05 * rng.normal(0, np.sqrt(2.0 / np.prod(shape[1:])), size=k)
        elif name != "b_fc2":
            p[off:off + k] = 4.0 * np.where(rng.uniform(size=k) < 0.5, -1.0, 1.0)
        off += k
    net.params.copy_(torch.as_tensor(p, dtype=torch.float32))


@pytest.mark.parametrize("B", [6, 64])
def test_tensor_core_forward_and_gradient(P, B):
    net = P.WeightPredictor(R, seed=6)
    _stable_masks(net, seed=20 + B)
    img, cs = _inputs(B, seed=8)
    out = net.forward(torch.as_tensor(img, device="cuda"), torch.as_tensor(cs, device="cuda"), tensor_cores=True)
    flat = net.params.cpu().numpy().astype(np.float64)
    # same rounding sites as the kernels (the float32 arithmetic of the same rounded network lies <= 6e-4
    # from the float64 one in every parameter group for such inputs)
    assert relL2(out.cpu().numpy(), C.forward(flat, R, img, cs, bf16=True)) < 1e-3
    gw = np.random.default_rng(9).normal(size=(B, R)).astype(np.float32)
    g = net.backward(torch.as_tensor(gw, device="cuda"), tensor_cores=True).cpu().numpy()
    gref = C.vjp(flat, R, img, cs, gw, bf16=True)
    off = 0
    for name, shape in C.param_shapes(R):
        k = int(np.prod(shape))
        assert relL2(g[off:off + k], gref[off:off + k]) < 3e-3, (name, relL2(g[off:off + k], gref[off:off + k]))
        off += k


def test_tensor_core_forward_with_random_biases(P):
    # the forward with ReLU decisions near zero: the output is continuous in them, so a flip moves it little
    net = P.WeightPredictor(R, seed=6)
    _biased(net)
    img, cs = _inputs(6, seed=8)
    out = net.forward(torch.as_tensor(img, device="cuda"), torch.as_tensor(cs, device="cuda"), tensor_cores=True)
    flat = net.params.cpu().numpy().astype(np.float64)
    assert relL2(out.cpu().numpy(), C.forward(flat, R, img, cs, bf16=True)) < 1e-3
    assert relL2(out.cpu().numpy(), C.forward(flat, R, img, cs)) < 3e-2


def test_bf16_inference_matches_oracle(P):
    net = P.WeightPredictor(R, seed=4)
    _biased(net)
    img, cs = _inputs(40, seed=7)
    out = net.predict(torch.as_tensor(img, device="cuda"), torch.as_tensor(cs, device="cuda"), batch=16)
    ref = C.forward(net.params.cpu().numpy().astype(np.float64), R, img, cs)
    assert relL2(out.cpu().numpy(), ref) < 3e-2


def test_prepare_input_is_the_block_mean(P):
    net = P.WeightPredictor(R, input_scale=0.5)
    proj = np.random.default_rng(9).normal(size=(3, 256, 256)).astype(np.float32)
    img = net.prepare(torch.as_tensor(proj, device="cuda")).cpu().numpy()
    assert np.allclose(img, C.downsample(proj, 0.5), rtol=1e-5, atol=1e-6)
    small = np.random.default_rng(10).normal(size=(2, 128, 128)).astype(np.float32)
    img2 = net.prepare(torch.as_tensor(small, device="cuda")).cpu().numpy()
    assert np.allclose(img2, C.downsample(small, 0.5), rtol=1e-6, atol=0)


@pytest.mark.parametrize("tc", [False, True])
def test_training_fits_a_fixed_batch(P, tc):
    net = P.WeightPredictor(R, seed=2, tensor_cores=tc)
    img, cs = _inputs(32, seed=11)
    target = np.random.default_rng(12).normal(size=(32, R)).astype(np.float32)
    I, Cs, Tg = (torch.as_tensor(a, device="cuda") for a in (img, cs, target))
    loss0 = C.mse(net.params.cpu().numpy().astype(np.float64), R, img, cs, target, bf16=tc)
    losses = [float(net.train_step(I, Cs, Tg, 1e-3).item()) for _ in range(100)]
    tol = 2e-3 if tc else 1e-4  # tensor cores: see test_tensor_core_forward_and_gradient
    assert abs(losses[0] - loss0) < tol * loss0, (losses[0], loss0)  # the step reports its starting loss
    final = C.mse(net.params.cpu().numpy().astype(np.float64), R, img, cs, target)
    assert final < 0.1 * loss0, (loss0, final)
