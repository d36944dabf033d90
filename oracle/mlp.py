"""Proposal network in FP64 (oracle; test infrastructure only).

Four dense layers in -> 256 -> 256 -> 256 -> out with exact GELU between them
(x * Phi(x), Phi the standard normal CDF via erf), trained with the Gaussian
negative log-likelihood of targets under the predicted means and log standard
deviations.  The network does not come from the paper (it only cites learned
samplers as particle seeds); its precision mirrors the GPU kernels: weights,
inputs and every inter-layer activation rounded to bfloat16, all arithmetic in
FP64 (the kernels accumulate in FP32).

Parameter layout (flat float vector, shared with the C ABI tamp_mlp_*):
W1 [H][IN], b1 [H], W2 [H][H], b2 [H], W3 [H][H], b3 [H], W4 [OUT][H], b4 [OUT].
Output k < OUT/2 is the mean of target k, output OUT/2 + k its log sigma.
"""
from __future__ import annotations

import math

import torch

DT = torch.float64
IN, H, OUT = 48, 256, 32


def shapes(n_in: int = IN, hidden: int = H, n_out: int = OUT):
    return [((hidden, n_in), (hidden,)), ((hidden, hidden), (hidden,)), ((hidden, hidden), (hidden,)),
            ((n_out, hidden), (n_out,))]


def n_params(n_in: int = IN, hidden: int = H, n_out: int = OUT) -> int:
    return sum(w[0] * w[1] + b[0] for w, b in shapes(n_in, hidden, n_out))


def unpack(theta: torch.Tensor, n_in: int = IN, hidden: int = H, n_out: int = OUT):
    out, o = [], 0
    for (wr, wc), (bn,) in shapes(n_in, hidden, n_out):
        W = theta[o:o + wr * wc].view(wr, wc)
        o += wr * wc
        b = theta[o:o + bn]
        o += bn
        out.append((W, b))
    return out


def bf16(t: torch.Tensor, on: bool = True) -> torch.Tensor:
    """Round to bfloat16 (round to nearest even) and back; identity in the
    backward pass (the kernels differentiate the rounded values as they are)."""
    if not on:
        return t
    r = t.detach().to(torch.bfloat16).to(t.dtype)
    return t + (r - t).detach()


def gelu(x: torch.Tensor) -> torch.Tensor:
    """Exact GELU: x * Phi(x) = x * (1 + erf(x / sqrt 2)) / 2."""
    return 0.5 * x * (1.0 + torch.erf(x / math.sqrt(2.0)))


def forward(theta: torch.Tensor, x: torch.Tensor, rounding: bool = True, n_in: int = IN, hidden: int = H,
            n_out: int = OUT):
    """Outputs [B, n_out] for inputs x [B, n_in] (FP64 arithmetic)."""
    a = bf16(x.to(DT), rounding)
    layers = unpack(theta, n_in, hidden, n_out)
    for i, (W, b) in enumerate(layers):
        z = a @ bf16(W, rounding).t() + b
        if i < len(layers) - 1:
            a = bf16(gelu(z), rounding)
        else:
            return z


def nll(out: torch.Tensor, y: torch.Tensor, mask: torch.Tensor) -> torch.Tensor:
    """Mean over rows of sum over masked targets of (y - mu)^2 / (2 sigma^2) + log sigma."""
    k = y.shape[1]
    mu, ls = out[:, :k], out[:, k:2 * k]
    per = 0.5 * (y - mu) ** 2 * torch.exp(-2.0 * ls) + ls
    return (per * mask).sum(dim=1).mean()


def loss_and_grad(theta, x, y, mask, rounding: bool = True, n_in: int = IN, hidden: int = H, n_out: int = OUT):
    th = theta.detach().clone().to(DT).requires_grad_(True)
    L = nll(forward(th, x, rounding, n_in, hidden, n_out), y.to(DT), mask.to(DT))
    (g,) = torch.autograd.grad(L, th)
    return L.detach(), g


def init_params(seed: int, n_in: int = IN, hidden: int = H, n_out: int = OUT) -> torch.Tensor:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for (wr, wc), (bn,) in shapes(n_in, hidden, n_out):
        lim = 1.0 / math.sqrt(wc)
        parts.append((torch.rand(wr * wc, generator=g, dtype=DT) * 2 - 1) * lim)
        parts.append(torch.zeros(bn, dtype=DT))
    return torch.cat(parts)
