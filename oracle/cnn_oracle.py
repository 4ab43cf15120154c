"""FP64 CPU oracle of the weight-predictor CNN.  TEST INFRASTRUCTURE ONLY.

Only ``tests/`` and ``bench.py``'s baseline legs may import or run this module.  It shares no code with
the CUDA path.  The network is the one the warm start of the temporal weights uses (the paper has no
counterpart; it maps one projection to its R low-rank weights):

* input: a [B][256][256] projection stack averaged over 2 x 2 pixel blocks to [B][128][128] and scaled;
* four 3 x 3 convolutions of stride 2 and padding 1 (1 -> 32 -> 64 -> 128 -> 128 channels), each
  followed by ReLU (128^2 -> 64^2 -> 32^2 -> 16^2 -> 8^2);
* the 8 x 8 x 128 features flattened in (y, x, channel) order, then (cos theta, sin theta) of the
  projection's gantry angle: 8194 inputs to a 128-unit ReLU layer, then a linear layer to R outputs;
* training loss: mean over the batch's B x R outputs of (prediction - target)^2.

Parameters are one flat vector, per layer: convolution weights [Co][ky][kx][Ci] and biases [Co] for the
four convolutions, then W1 [128][8194], b1 [128], W2 [R][128], b2 [R].  The steps are library
primitives in float64 (``torch.nn.functional.conv2d`` / ``linear`` / ``relu``), and autograd gives the
gradient of the same definition.  Pins: ``tests/test_oracle_cnn.py`` (convolution against an explicit
loop, the feature order, finite differences of the gradient, the 2 x 2 average, bfloat16 rounding).

``bf16_round`` / ``gemm_bf16``: the tensor-core GEMM's definition -- both operands rounded to bfloat16
(round to nearest, ties to even), then an exact product in float64.
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np
import torch
import torch.nn.functional as F

DT = torch.float64
CH = [1, 32, 64, 128, 128]
HID = 128
FEAT = 8 * 8 * 128
FEAT_IN = FEAT + 2


def param_shapes(R: int) -> List[Tuple[str, Tuple[int, ...]]]:
    out = []
    for l in range(4):
        out.append((f"w{l}", (CH[l + 1], 3, 3, CH[l])))
        out.append((f"b{l}", (CH[l + 1],)))
    out += [("w_fc1", (HID, FEAT_IN)), ("b_fc1", (HID,)), ("w_fc2", (R, HID)), ("b_fc2", (R,))]
    return out


def n_params(R: int) -> int:
    return int(sum(np.prod(s) for _, s in param_shapes(R)))


def unpack(flat: torch.Tensor, R: int) -> Dict[str, torch.Tensor]:
    """Views of the flat parameter vector, in the layouts of the module docstring."""
    out, off = {}, 0
    for name, shape in param_shapes(R):
        n = int(np.prod(shape))
        out[name] = flat[off:off + n].reshape(shape)
        off += n
    return out


def downsample(proj, scale: float) -> np.ndarray:
    """The [B][128][128] network input: scale * the 2 x 2 block means of [B][256][256] projections, or
    scale * [B][128][128] projections as they are."""
    p = np.asarray(proj, dtype=np.float64)
    if p.shape[1] == 128:
        return scale * p
    return scale * 0.25 * (p[:, 0::2, 0::2] + p[:, 0::2, 1::2] + p[:, 1::2, 0::2] + p[:, 1::2, 1::2])


def _bf16_t(t: torch.Tensor) -> torch.Tensor:
    """bf16_round of a tensor's values taken as float32 (no gradient)."""
    return torch.as_tensor(bf16_round(t.detach().numpy().astype(np.float32)), dtype=DT)


class _Bf16Conv(torch.autograd.Function):
    """The stride-2, padding-1 convolution with bfloat16-rounded operands in both directions: forward
    conv(r(x), r(w)) + b; backward dx from r(dy) and r(w), dw from r(x) and r(dy), db = sum dy."""

    @staticmethod
    def forward(ctx, x, w, b):
        ctx.save_for_backward(x, w)
        return F.conv2d(_bf16_t(x), _bf16_t(w), b, stride=2, padding=1)

    @staticmethod
    def backward(ctx, g):
        x, w = ctx.saved_tensors
        gr = _bf16_t(g)
        gx = torch.nn.grad.conv2d_input(x.shape, _bf16_t(w), gr, stride=2, padding=1)
        gw = torch.nn.grad.conv2d_weight(_bf16_t(x), w.shape, gr, stride=2, padding=1)
        return gx, gw, g.sum((0, 2, 3))


class _Bf16Linear(torch.autograd.Function):
    """x W^T + b with bfloat16-rounded operands in both directions (as _Bf16Conv)."""

    @staticmethod
    def forward(ctx, x, w, b):
        ctx.save_for_backward(x, w)
        return _bf16_t(x) @ _bf16_t(w).T + b

    @staticmethod
    def backward(ctx, g):
        x, w = ctx.saved_tensors
        gr = _bf16_t(g)
        return gr @ _bf16_t(w), gr.T @ _bf16_t(x), g.sum(0)


def forward_tensors(flat: torch.Tensor, R: int, img: torch.Tensor, cs: torch.Tensor, bf16: bool = False) -> torch.Tensor:
    """bf16: every operand of the four convolutions and of the 8194-wide layer rounded to bfloat16, in
    the forward (inputs, weights) and in the backward (incoming gradients, inputs, weights) -- the
    tensor-core GEMMs' operands; biases, bias gradients and the output layer unrounded."""
    P = unpack(flat, R)
    x = img.reshape(img.shape[0], 1, 128, 128)                       # NCHW for the library convolution
    for l in range(4):
        w = P[f"w{l}"].permute(0, 3, 1, 2)                           # [Co][Ci][ky][kx]
        x = F.relu(_Bf16Conv.apply(x, w, P[f"b{l}"]) if bf16 else F.conv2d(x, w, P[f"b{l}"], stride=2, padding=1))
    feat = torch.cat([x.permute(0, 2, 3, 1).reshape(x.shape[0], FEAT), cs], 1)   # (y, x, c) order, cos, sin
    h = F.relu(_Bf16Linear.apply(feat, P["w_fc1"], P["b_fc1"]) if bf16 else F.linear(feat, P["w_fc1"], P["b_fc1"]))
    return F.linear(h, P["w_fc2"], P["b_fc2"])


def forward(flat, R: int, img, cs, bf16: bool = False) -> np.ndarray:
    with torch.no_grad():
        t = lambda a: torch.as_tensor(np.asarray(a), dtype=DT)
        return forward_tensors(t(flat), R, t(img), t(cs), bf16).numpy()


def vjp(flat, R: int, img, cs, grad_w, bf16: bool = False) -> np.ndarray:
    """Gradient of sum(grad_w * forward) with respect to the flat parameter vector (bf16: with the
    rounded operands of forward_tensors in both directions)."""
    t = lambda a: torch.as_tensor(np.asarray(a), dtype=DT)
    p = t(flat).clone().requires_grad_(True)
    out = forward_tensors(p, R, t(img), t(cs), bf16)
    (out * t(grad_w)).sum().backward()
    return p.grad.numpy()


def mse(flat, R: int, img, cs, target, bf16: bool = False) -> float:
    out = forward(flat, R, img, cs, bf16)
    return float(((out - np.asarray(target, dtype=np.float64)) ** 2).mean())


def bf16_round(x) -> np.ndarray:
    """Nearest bfloat16 of each float32 value (ties to even), as float64.  A bfloat16 is the upper 16 bits
    of a binary32 pattern: add 0x7FFF plus the lowest kept bit (so that exact halves go to the even
    neighbour) and clear the 16 dropped bits.  Finite inputs only."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float32))
    u = a.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gemm_bf16(A, B, trans_a: bool = False, trans_b: bool = False, bias=None, relu: bool = False) -> np.ndarray:
    """op(A) op(B) (+ bias per column, ReLU) with A and B rounded to bfloat16 and everything after in
    float64; op(X) = X.T when its flag is set."""
    a, b = bf16_round(A), bf16_round(B)
    c = (a.T if trans_a else a) @ (b.T if trans_b else b)
    if bias is not None:
        c = c + np.asarray(bias, dtype=np.float64)[None, :]
    return np.maximum(c, 0.0) if relu else c
