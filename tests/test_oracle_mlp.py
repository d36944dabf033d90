"""Pins of the FP64 proposal-network oracle (closed forms, finite differences,
a single-layer case that reduces to a library matmul)."""
import math

import pytest
import torch

from oracle import mlp

DT = torch.float64


def test_gelu_hand_values():
    x = torch.tensor([0.0, 1.0, -1.0, 3.0], dtype=DT)
    # Phi(1) = 0.841344746..., Phi(3) = 0.998650101...
    expect = torch.tensor([0.0, 0.8413447460685429, -0.15865525393145707, 2.9959502965], dtype=DT)
    assert torch.allclose(mlp.gelu(x), expect, atol=1e-9)


def test_nll_closed_form():
    out = torch.tensor([[1.0, 0.0, math.log(2.0), 0.0]], dtype=DT)   # mu = (1, 0), log sigma = (ln 2, 0)
    y = torch.tensor([[3.0, 5.0]], dtype=DT)
    mask = torch.tensor([[1.0, 0.0]], dtype=DT)
    # (3 - 1)^2 / (2 * 4) + ln 2, second target masked out
    assert float(mlp.nll(out, y, mask)) == pytest.approx(0.5 + math.log(2.0), abs=1e-15)


def test_forward_matches_layerwise_library_matmuls_without_rounding():
    theta = mlp.init_params(3)
    x = torch.randn(5, mlp.IN, dtype=DT, generator=torch.Generator().manual_seed(4))
    a = x
    for i, (W, b) in enumerate(mlp.unpack(theta)):
        z = torch.nn.functional.linear(a, W, b)
        a = torch.nn.functional.gelu(z) if i < 3 else z
    assert torch.allclose(mlp.forward(theta, x, rounding=False), a, atol=1e-12)


def test_gradient_matches_central_differences_without_rounding():
    n_in, hid, n_out = 6, 8, 4
    theta = mlp.init_params(5, n_in, hid, n_out)
    g0 = torch.Generator().manual_seed(6)
    x = torch.randn(7, n_in, dtype=DT, generator=g0)
    y = torch.randn(7, n_out // 2, dtype=DT, generator=g0)
    mask = (torch.rand(7, n_out // 2, generator=g0) > 0.3).to(DT)
    _, g = mlp.loss_and_grad(theta, x, y, mask, False, n_in, hid, n_out)
    h = 1e-6
    fd = torch.zeros_like(theta)
    for i in range(theta.numel()):
        tp, tm = theta.clone(), theta.clone()
        tp[i] += h
        tm[i] -= h
        fd[i] = (mlp.nll(mlp.forward(tp, x, False, n_in, hid, n_out), y, mask)
                 - mlp.nll(mlp.forward(tm, x, False, n_in, hid, n_out), y, mask)) / (2 * h)
    assert torch.allclose(g, fd, atol=1e-7, rtol=1e-6)


def test_bf16_rounding_is_round_to_nearest_even():
    t = torch.tensor([1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9], dtype=DT)
    # bf16 has 8 significand bits: 1 + 2^-8 ties to even (1.0), 1 + 3*2^-8 ties to 1 + 2^-6... to even 1 + 2^-6
    assert mlp.bf16(t).tolist() == [1.0, 1.0 + 2 ** -6, 1.0]


def test_param_count():
    assert mlp.n_params() == 256 * 48 + 256 + 2 * (256 * 256 + 256) + 32 * 256 + 32
