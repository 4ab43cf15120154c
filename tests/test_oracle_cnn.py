"""Pins of the FP64 CNN oracle: the convolution step against an explicit loop (stride, padding and the
[Co][ky][kx][Ci] weight layout), the (y, x, channel) feature order and the angle inputs, central finite
differences of the parameter gradient, and the 2 x 2 average of the input."""
import numpy as np
import pytest
import torch

from oracle import cnn_oracle as C


def test_conv_step_matches_explicit_loop():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 4, 9, 7))            # NCHW, odd sizes exercise the padding
    w = rng.normal(size=(5, 3, 3, 4))            # [Co][ky][kx][Ci]
    b = rng.normal(size=5)
    got = torch.nn.functional.conv2d(torch.tensor(x), torch.tensor(w).permute(0, 3, 1, 2), torch.tensor(b),
                                     stride=2, padding=1).numpy()
    Ho, Wo = (9 + 1) // 2, (7 + 1) // 2
    ref = np.zeros((2, 5, Ho, Wo))
    for n in range(2):
        for co in range(5):
            for y in range(Ho):
                for xx in range(Wo):
                    s = b[co]
                    for ky in range(3):
                        for kx in range(3):
                            iy, ix = 2 * y + ky - 1, 2 * xx + kx - 1
                            if 0 <= iy < 9 and 0 <= ix < 7:
                                s += sum(w[co, ky, kx, ci] * x[n, ci, iy, ix] for ci in range(4))
                    ref[n, co, y, xx] = s
    assert np.allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_feature_order_and_angle_inputs():
    """With identity-like weights the output reads one chosen feature: pins (y, x, c) flattening and the
    position of cos / sin after the image features."""
    R = 3
    flat = np.zeros(C.n_params(R))
    P = C.unpack(torch.tensor(flat), R)
    # a single bright input pixel travels through centre taps only: conv l takes channel 0 -> channel 0
    for l in range(4):
        P[f"w{l}"][0, 1, 1, 0] = 1.0
    y, x = 3, 5
    img = np.zeros((1, 128, 128))
    img[0, 16 * y, 16 * x] = 2.0                 # stride-2 centre taps: output (y, x) reads input (2y, 2x)
    P["w_fc1"][0, (y * 8 + x) * 128 + 0] = 1.0   # feature (y, x, c = 0)
    P["w_fc1"][1, C.FEAT] = 1.0                  # cos
    P["w_fc1"][2, C.FEAT + 1] = 1.0              # sin
    for r in range(3):
        P["w_fc2"][r, r] = 1.0
    cs = np.array([[0.25, 0.75]])
    out = C.forward(torch.cat([v.reshape(-1) for v in P.values()]).numpy(), R, img, cs)
    assert np.allclose(out, [[2.0, 0.25, 0.75]])


def test_gradient_matches_central_differences():
    R = 2
    rng = np.random.default_rng(1)
    flat = np.zeros(C.n_params(R))
    off = 0
    for name, shape in C.param_shapes(R):
        n = int(np.prod(shape))
        fan = int(np.prod(shape[1:])) if len(shape) > 1 else 1
        flat[off:off + n] = rng.normal(size=n) * np.sqrt(2.0 / fan) + (0.05 if name.startswith("b") else 0.0)
        off += n
    img = rng.uniform(0, 1, size=(2, 128, 128))
    cs = rng.normal(size=(2, 2))
    gw = rng.normal(size=(2, R))
    g = C.vjp(flat, R, img, cs, gw)
    f = lambda p: float((C.forward(p, R, img, cs) * gw).sum())
    idx = rng.choice(len(flat), 25, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (f(flat + e) - f(flat - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-7, (i, fd, g[i])


def test_downsample_is_the_block_mean():
    rng = np.random.default_rng(2)
    p = rng.normal(size=(3, 8, 6))
    d = C.downsample(p, 2.0)
    assert d.shape == (3, 4, 3)
    assert np.isclose(d[1, 2, 1], 2.0 * p[1, 4:6, 2:4].mean())


def test_bf16_rounding_ties_to_even_and_matches_torch():
    u = 2.0 ** -8  # half a bfloat16 ulp at 1
    x = np.array([1.0, -2.5, 1 + u, 1 + 3 * u, 1 + u + 2.0 ** -20, 1 - 2.0 ** -9], dtype=np.float32)
    want = np.array([1.0, -2.5, 1.0, 1 + 4 * u, 1 + 2 * u, 1.0])
    assert np.array_equal(C.bf16_round(x), want)
    rng = np.random.default_rng(3)
    y = (rng.normal(size=10000) * 10.0 ** rng.uniform(-30, 30, size=10000)).astype(np.float32)
    ref = torch.tensor(y).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(C.bf16_round(y), ref)


def test_gemm_bf16_definition():
    rng = np.random.default_rng(4)
    A = rng.normal(size=(5, 7)).astype(np.float32)
    B = rng.normal(size=(7, 3)).astype(np.float32)
    bias = rng.normal(size=3)
    ref = C.bf16_round(A) @ C.bf16_round(B) + bias
    assert np.allclose(C.gemm_bf16(A, B, bias=bias), ref, rtol=0, atol=1e-12)
    assert np.allclose(C.gemm_bf16(A.T.copy(), B.T.copy(), True, True, bias, True), np.maximum(ref, 0), atol=1e-12)
    # exact on values that bfloat16 holds: small integers
    Ai = rng.integers(-8, 9, size=(4, 6)).astype(np.float32)
    Bi = rng.integers(-8, 9, size=(6, 2)).astype(np.float32)
    assert np.array_equal(C.gemm_bf16(Ai, Bi), Ai.astype(np.float64) @ Bi.astype(np.float64))


def test_bf16_forward_is_exact_when_every_operand_is_representable_and_close_otherwise():
    R = 2
    shapes = dict(C.param_shapes(R))
    P = {k: np.zeros(v) for k, v in shapes.items()}
    for l, scale in zip(range(4), (1.0, 0.5, 0.5, 0.25)):
        co, _, _, ci = shapes[f"w{l}"]
        for o in range(co):
            P[f"w{l}"][o, 1, 1, o % ci] = scale                       # the centre tap only
    for j in range(C.HID):
        P["w_fc1"][j, j] = 1.0
    P["w_fc2"] = np.random.default_rng(0).normal(size=shapes["w_fc2"])
    flat = np.concatenate([P[k].ravel() for k, _ in C.param_shapes(R)])
    rng = np.random.default_rng(1)
    img = rng.integers(0, 3, size=(2, 128, 128)) * 0.5                 # 0, 0.5, 1
    cs = np.array([[1.0, 0.0], [0.0, 1.0]])
    a, b = C.forward(flat, R, img, cs), C.forward(flat, R, img, cs, bf16=True)
    assert np.array_equal(a, b) and np.abs(a).max() > 0
    # the backward too: output weights and incoming gradients that bfloat16 holds keep every backward
    # operand exact
    P["w_fc2"] = np.random.default_rng(2).choice([-1.0, -0.5, 0.25, 0.5, 1.0], size=shapes["w_fc2"])
    flat = np.concatenate([P[k].ravel() for k, _ in C.param_shapes(R)])
    gw = np.array([[1.0, -2.0], [0.5, 3.0]])
    ga, gb = C.vjp(flat, R, img, cs, gw), C.vjp(flat, R, img, cs, gw, bf16=True)
    assert np.array_equal(ga, gb) and np.abs(ga).max() > 0
    flat2 = rng.normal(size=flat.size) * 0.05
    img2 = rng.uniform(size=(2, 128, 128))
    a, b = C.forward(flat2, R, img2, cs), C.forward(flat2, R, img2, cs, bf16=True)
    rel = np.linalg.norm(a - b) / np.linalg.norm(a)
    assert 1e-5 < rel < 2e-2, rel
    ga, gb = C.vjp(flat2, R, img2, cs, gw), C.vjp(flat2, R, img2, cs, gw, bf16=True)
    rel = np.linalg.norm(ga - gb) / np.linalg.norm(ga)
    assert 1e-5 < rel < 0.3, rel

