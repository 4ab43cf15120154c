"""The tensor-core GEMM (digs_gemm_bf16, tcgen05 with FP32 accumulation in tensor memory) against its
definition: both operands rounded to bfloat16, exact products, sums in float64 (oracle.cnn_oracle).
Every element must lie within the FP32 summation bound 4 K 2^-24 sum_k |a_k b_k| of the exact value; the
cases cover ragged tile edges, all four operand layouts, a 9-deep K (the first convolution), the bias /
ReLU epilogue, split K with empty splits, a multi-tile product, and bitwise repeatability."""
import numpy as np
import pytest
import torch

from oracle import cnn_oracle as C

pytestmark = pytest.mark.gpu


def _check(M, N, K, ta=False, tb=False, bias=False, relu=False, splits=1, seed=0):
    from paper_2506_22280_gb300 import digs as D
    rng = np.random.default_rng(seed)
    A = rng.normal(size=(K, M) if ta else (M, K)).astype(np.float32)
    B = rng.normal(size=(N, K) if tb else (K, N)).astype(np.float32)
    b = rng.normal(size=N).astype(np.float32) if bias else None
    dev = "cuda"
    out, status = D.gemm_bf16(torch.tensor(A, device=dev), torch.tensor(B, device=dev), ta, tb,
                              torch.tensor(b, device=dev) if bias else None, relu, splits)
    got = out.cpu().numpy().astype(np.float64)
    assert int(status.item()) == 0
    ref = C.gemm_bf16(A, B, ta, tb, b, relu)
    a_, b_ = np.abs(C.bf16_round(A)), np.abs(C.bf16_round(B))
    mag = (a_.T if ta else a_) @ (b_.T if tb else b_) + (np.abs(b)[None, :] if bias else 0.0)
    err = np.abs(got - ref)
    bound = 4.0 * max(K, 1) * 2.0 ** -24 * mag + 1e-30
    assert np.all(err <= bound), (M, N, K, ta, tb, float((err / bound).max()))
    return out


def test_single_tile():
    _check(128, 64, 64)


@pytest.mark.parametrize("ta,tb", [(False, False), (False, True), (True, False), (True, True)])
def test_ragged_all_layouts(ta, tb):
    _check(200, 70, 75, ta, tb, seed=1)


def test_shallow_k_bias_relu():
    _check(1000, 32, 9, False, True, bias=True, relu=True, seed=2)


def test_split_k_with_empty_splits():
    _check(96, 40, 1000, True, False, bias=True, splits=5, seed=3)


def test_multi_tile_and_repeatable():
    a = _check(4096, 128, 1152, False, True, seed=4)
    b = _check(4096, 128, 1152, False, True, seed=4)
    assert torch.equal(a, b)
