"""Pins of the oracle's B-spline basis and FFD evaluation (Sec. 3.3, Eq. 10-11) to closed forms.

None of these restates the oracle's formulas: they check identities the uniform cubic B-spline and the
tensor-product FFD must satisfy (partition of unity, linear precision, C2 continuity, affine
reproduction, derivative = finite difference, separability), and the textbook knot values stored in
``tests/golden/bspline_knots.txt``.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import digs_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
DT = torch.float64


def _u(n=101):
    return torch.linspace(0.0, 1.0 - 1e-9, n, dtype=DT)


def test_partition_of_unity_and_derivative_sums():
    u = _u()
    assert torch.allclose(O.bspline(u).sum(-1), torch.ones_like(u), atol=1e-15)
    assert torch.allclose(O.bspline(u, 1).sum(-1), torch.zeros_like(u), atol=1e-14)
    assert torch.allclose(O.bspline(u, 2).sum(-1), torch.zeros_like(u), atol=1e-14)


def test_linear_precision():
    # sum_l (l - 1) B_l(u) = u: the spline of linear control values is the line itself
    u = _u()
    l = torch.arange(4, dtype=DT) - 1
    assert torch.allclose((O.bspline(u) * l).sum(-1), u, atol=1e-15)
    assert torch.allclose((O.bspline(u, 1) * l).sum(-1), torch.ones_like(u), atol=1e-14)
    # quadratic precision of the cubic B-spline: sum_l (l-1)^2 B_l(u) = u^2 + 1/3
    assert torch.allclose((O.bspline(u) * l * l).sum(-1), u * u + 1.0 / 3.0, atol=1e-14)


def test_textbook_knot_values():
    """Uniform cubic B-spline values at u = 0 and u = 1/2 (golden fixture with its citation)."""
    rows = [l for l in open(os.path.join(GOLDEN, "bspline_knots.txt")) if l.strip() and not l.startswith("#")]
    for row in rows:
        vals = [float(Fraction(t)) for t in row.split()]  # fractions written as a/b
        u, expect = vals[0], vals[1:]
        got = O.bspline(torch.tensor([u], dtype=DT))[0].numpy()
        assert np.allclose(got, expect, atol=1e-15), (u, got, expect)


def test_derivatives_match_finite_differences():
    u = torch.linspace(0.05, 0.95, 19, dtype=DT)
    h = 1e-6
    fd1 = (O.bspline(u + h) - O.bspline(u - h)) / (2 * h)
    fd2 = (O.bspline(u + h, 1) - O.bspline(u - h, 1)) / (2 * h)
    assert torch.allclose(O.bspline(u, 1), fd1, atol=1e-8)
    assert torch.allclose(O.bspline(u, 2), fd2, atol=1e-8)


def _spline1d(c, p, deriv=0):
    """1-D uniform cubic spline sum_l B_l(p - floor p) c[floor p - 1 + l] (zero outside c)."""
    p = torch.as_tensor(p, dtype=DT)
    f = torch.floor(p)
    u = p - f
    B = O.bspline(u, deriv)
    out = torch.zeros_like(p)
    for l in range(4):
        idx = (f - 1 + l).long()
        ok = (idx >= 0) & (idx < len(c))
        out = out + B[..., l] * torch.where(ok, torch.as_tensor(c, dtype=DT)[idx.clamp(0, len(c) - 1)], torch.zeros_like(p))
    return out


def test_c2_continuity_across_knots():
    rng = np.random.default_rng(0)
    c = rng.normal(size=12)
    eps = 1e-7
    for k in range(3, 9):
        for deriv, tol in ((0, 1e-6), (1, 1e-6), (2, 1e-5)):
            lo = _spline1d(c, k - eps, deriv)
            hi = _spline1d(c, k + eps, deriv)
            assert abs(float(lo - hi)) < tol, (k, deriv)


def _lattice(n=(7, 6, 8), spacing=(10.0, 12.0, 9.0), origin=(-30.0, -31.0, -27.0), R=2):
    return dict(nx=n[0], ny=n[1], nz=n[2], R=R, origin=np.array(origin), spacing=np.array(spacing))


def _nodes(lat):
    xs = lat["origin"][0] + lat["spacing"][0] * np.arange(lat["nx"])
    ys = lat["origin"][1] + lat["spacing"][1] * np.arange(lat["ny"])
    zs = lat["origin"][2] + lat["spacing"][2] * np.arange(lat["nz"])
    Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
    return np.stack([X, Y, Z], -1)  # [nz][ny][nx][3]


def _interior_points(lat, n, rng):
    lo = lat["origin"] + lat["spacing"] * 1.0
    hi = lat["origin"] + lat["spacing"] * (np.array([lat["nx"], lat["ny"], lat["nz"]]) - 3.0)
    return rng.uniform(lo, hi, size=(n, 3))


def test_affine_control_points_reproduce_affine_field():
    """d = A x + t on every node => u(x) = A x + t and grad u = A wherever all 64 nodes are inside."""
    rng = np.random.default_rng(1)
    lat = _lattice()
    nodes = _nodes(lat)
    A = rng.normal(size=(2, 3, 3)) * 0.1
    t = rng.normal(size=(2, 3))
    phi = np.stack([nodes @ A[r].T + t[r] for r in range(2)])
    x = _interior_points(lat, 200, rng)
    U, dU = O.ffd_eval(torch.tensor(phi), lat, torch.tensor(x))
    for r in range(2):
        assert np.allclose(U[:, r].numpy(), x @ A[r].T + t[r], atol=1e-12)
        assert np.allclose(dU[:, r].numpy(), np.broadcast_to(A[r], (200, 3, 3)), atol=1e-12)


def test_gradient_matches_finite_difference_including_padded_border():
    rng = np.random.default_rng(2)
    lat = _lattice()
    phi = rng.normal(size=(2, lat["nz"], lat["ny"], lat["nx"], 3))
    lo = lat["origin"] - 0.5 * lat["spacing"]
    hi = lat["origin"] + lat["spacing"] * (np.array([lat["nx"], lat["ny"], lat["nz"]]) - 0.5)
    x = rng.uniform(lo, hi, size=(100, 3))
    # keep away from knot planes so the central difference stays inside one cell
    p = (x - lat["origin"]) / lat["spacing"]
    x = lat["origin"] + lat["spacing"] * (np.floor(p) + np.clip(p - np.floor(p), 0.01, 0.99))
    X = torch.tensor(x)
    _, dU = O.ffd_eval(torch.tensor(phi), lat, X)
    h = 1e-5
    for j in range(3):
        e = torch.zeros(3, dtype=DT)
        e[j] = h
        Up, _ = O.ffd_eval(torch.tensor(phi), lat, X + e)
        Um, _ = O.ffd_eval(torch.tensor(phi), lat, X - e)
        assert torch.allclose(dU[..., j], (Up - Um) / (2 * h), atol=1e-7)


def test_single_node_bump_and_zero_padding():
    """One non-zero node: u at the node equals (2/3)^3 d; a point whose neighbourhood includes
    out-of-lattice nodes only sees the in-lattice ones (zero padding)."""
    lat = _lattice(n=(4, 4, 4), spacing=(10.0, 10.0, 10.0), origin=(0.0, 0.0, 0.0), R=1)
    phi = np.zeros((1, 4, 4, 4, 3))
    phi[0, 0, 0, 0] = [1.0, -2.0, 3.0]          # corner node at the origin
    U, _ = O.ffd_eval(torch.tensor(phi), lat, torch.tensor([[0.0, 0.0, 0.0], [5.0, 5.0, 5.0]]))
    assert np.allclose(U[0, 0].numpy(), (2.0 / 3.0) ** 3 * np.array([1.0, -2.0, 3.0]), atol=1e-15)
    # at the cell centre u = 1/2 the corner node is l = 1 on each axis: B_1(1/2) = 23/48
    assert np.allclose(U[1, 0].numpy(), (23.0 / 48.0) ** 3 * np.array([1.0, -2.0, 3.0]), atol=1e-15)


def test_separable_field_axis_order():
    """phi = f(i) g(j) h(k) e_c gives u = F(x) G(y) H(z) e_c with F, G, H 1-D splines: pins that the
    x index runs fastest in phi[r][k][j][i] and that lattice coordinates use the right axis."""
    rng = np.random.default_rng(3)
    lat = _lattice(R=1)
    f, g, h = rng.normal(size=lat["nx"]), rng.normal(size=lat["ny"]), rng.normal(size=lat["nz"])
    phi = np.zeros((1, lat["nz"], lat["ny"], lat["nx"], 3))
    phi[0, ..., 1] = h[:, None, None] * g[None, :, None] * f[None, None, :]
    x = rng.uniform(lat["origin"], lat["origin"] + lat["spacing"] * 5, size=(50, 3))
    U, dU = O.ffd_eval(torch.tensor(phi), lat, torch.tensor(x))
    p = (x - lat["origin"]) / lat["spacing"]
    F, G, H = _spline1d(f, p[:, 0]), _spline1d(g, p[:, 1]), _spline1d(h, p[:, 2])
    assert torch.allclose(U[:, 0, 1], F * G * H, atol=1e-13)
    assert torch.allclose(U[:, 0, 0], torch.zeros(50, dtype=DT)) and torch.allclose(U[:, 0, 2], torch.zeros(50, dtype=DT))
    dF = _spline1d(f, p[:, 0], 1) / lat["spacing"][0]
    assert torch.allclose(dU[:, 0, 1, 0], dF * G * H, atol=1e-13)


# ---- temporal B-spline of the weights (Sec. 4.2) ------------------------------------------------
def test_temporal_weights_reproduce_constants_lines_and_knot_values():
    from oracle import digs_oracle as O
    t_step = 4.0
    n_ctrl = 12
    rows = list(range(0, 30))
    const = np.full((n_ctrl, 2), 1.7)
    w = O.temporal_weights(const, t_step, rows).numpy()
    assert np.allclose(w, 1.7, atol=1e-12)                     # partition of unity (all nodes inside)
    j = np.arange(n_ctrl, dtype=float)
    lin = np.stack([0.5 * j - 2.0, -1.5 * j + 0.25], 1)
    w = O.temporal_weights(lin, t_step, rows).numpy()
    tau = np.asarray(rows) / t_step + 1.0
    assert np.allclose(w[:, 0], 0.5 * tau - 2.0, atol=1e-12)  # linear precision: w = line(tau)
    assert np.allclose(w[:, 1], -1.5 * tau + 0.25, atol=1e-12)
    spike = np.zeros((n_ctrl, 1))
    spike[5, 0] = 6.0
    # at a knot (u = 0) the basis is (1/6, 4/6, 1/6, 0): p = 16 -> tau = 5, f = 4, nodes 4..7
    assert np.allclose(O.temporal_weights(spike, t_step, [16]).numpy(), [[4.0]])
    assert np.allclose(O.temporal_weights(spike, t_step, [12]).numpy(), [[1.0]])   # tau = 4: node 5 is f + 2
    # nodes past the end read as zero
    # p = 40: tau = 11, nodes 10..13 of which 10, 11 exist (1/6 + 4/6); p = 44: only node 11 (1/6)
    assert np.allclose(O.temporal_weights(const, t_step, [40, 44]).numpy(), [[1.7 * 5 / 6] * 2, [1.7 / 6] * 2])
