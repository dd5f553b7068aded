"""Pins of the prefilter network's FP64 oracle (oracle/mlp.py).

GELU against its closed form, unit-norm outputs, the loss at its zero, and
the finite-difference gradient against torch autograd in FP64 (an independent
library computation of the same derivative).
"""
import math

import numpy as np
import pytest

from oracle import mlp


def test_gelu_closed_forms():
    assert mlp.gelu(0.0) == 0.0
    # gelu(v) = v Phi(v): Phi(1) = 0.841344746068543, Phi(-1) = 0.158655253931457
    assert float(mlp.gelu(1.0)) == pytest.approx(0.8413447460685429, abs=1e-15)
    assert float(mlp.gelu(-1.0)) == pytest.approx(-0.15865525393145707, abs=1e-15)
    assert float(mlp.gelu(30.0)) == 30.0


def _params(rng, D=12, H=8, P=4):
    return [rng.standard_normal((H, D)) / math.sqrt(D), 0.1 * rng.standard_normal(H),
            rng.standard_normal((P, H)) / math.sqrt(H), 0.1 * rng.standard_normal(P)]


def test_outputs_are_unit_vectors():
    rng = np.random.default_rng(0)
    p = _params(rng)
    e = mlp.forward(p, rng.standard_normal((5, 12)))
    np.testing.assert_allclose(np.linalg.norm(e, axis=1), 1.0, atol=1e-14)


def test_loss_is_zero_at_its_targets():
    rng = np.random.default_rng(1)
    p = _params(rng)
    xq, xd = rng.standard_normal((6, 12)), rng.standard_normal((6, 12))
    y = np.sum(mlp.forward(p, xq) * mlp.forward(p, xd), axis=1)
    assert mlp.loss(p, xq, xd, y) < 1e-28
    assert mlp.loss(p, xq, xd, y + 0.1) == pytest.approx(0.01, rel=1e-12)


def test_finite_differences_match_autograd():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    p = _params(rng)
    xq, xd = rng.standard_normal((7, 12)), rng.standard_normal((7, 12))
    y = rng.uniform(-1, 1, 7)
    w = rng.uniform(0.5, 2.0, 7)
    fd = mlp.fd_grad(p, xq, xd, y, w)
    tp = [torch.tensor(a, dtype=torch.float64, requires_grad=True) for a in p]

    def f(x):
        h = torch.tensor(x) @ tp[0].T + tp[1]
        g = h * 0.5 * (1 + torch.erf(h / math.sqrt(2.0)))
        z = g @ tp[2].T + tp[3]
        return z / z.norm(dim=1, keepdim=True)

    s = (f(xq) * f(xd)).sum(dim=1)
    wt = torch.tensor(w)
    L = (wt * (s - torch.tensor(y)) ** 2).sum() / wt.sum()
    L.backward()
    ad = np.concatenate([t.grad.numpy().ravel() for t in tp])
    np.testing.assert_allclose(fd, ad, rtol=1e-6, atol=1e-9)
