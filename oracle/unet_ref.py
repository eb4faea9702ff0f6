"""CPU oracle of the warm-start U-Net (plain PyTorch CPU ops, FP32 or FP64).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg).  It builds
the network described in include/tvcut.h from the same flat parameter vector:
for each of the 18 convolutions in forward order, weights [9][Cout][Cin]
(tap 3*ky + kx reads pixel (y + ky - 1, x + kx - 1), zero padding) then bias
[Cout]; 2x2 average pooling, nearest 2x upsampling, concatenation
[upsampled, skip]; ReLU after every convolution but the last; input padded
from 3 to 16 channels with zeros; output channels 0 and 1; loss = mean
squared error over those two channels.  Gradients come from autograd; the
pins in tests/test_oracle_unet.py check them against finite differences, the
convolution against a direct loop, and the wiring (pooling, upsampling, the
skip connections and the concatenation order, the ReLU placement) against a
hand-derived closed form (tests/golden/unet_wiring.json).

``bf16_storage=True`` rounds every stored tensor to BF16 where the library
stores one (the packed input, each convolution's output but the last, each
pooled tensor; in the backward pass the gradient of each of those tensors
and of the output), with the arithmetic between stores in the oracle's own
precision.  Element-wise comparisons of the library's BF16 network are made
against this; it is the definition above with the storage precision made
explicit, not a model of any kernel's summation order.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F


def layer_shapes(base: int):
    C = base
    return [(16, C), (C, C), (C, 2 * C), (2 * C, 2 * C), (2 * C, 4 * C), (4 * C, 4 * C),
            (4 * C, 8 * C), (8 * C, 8 * C), (8 * C, 4 * C), (8 * C, 4 * C), (4 * C, 4 * C),
            (4 * C, 2 * C), (4 * C, 2 * C), (2 * C, 2 * C), (2 * C, C), (2 * C, C), (C, C), (C, 16)]


def num_params(base: int) -> int:
    return sum(9 * ci * co + co for ci, co in layer_shapes(base))


def unpack(theta: torch.Tensor, base: int):
    """Flat vector -> list of (weight [Cout, Cin, 3, 3], bias [Cout])."""
    out, off = [], 0
    for ci, co in layer_shapes(base):
        w = theta[off:off + 9 * co * ci].reshape(3, 3, co, ci).permute(2, 3, 0, 1)
        off += 9 * co * ci
        b = theta[off:off + co]
        off += co
        out.append((w, b))
    return out


def conv(x, wb, relu=True):
    y = F.conv2d(x, wb[0], wb[1], padding=1)
    return F.relu(y) if relu else y


class _StoreBF16(torch.autograd.Function):
    """Identity up to BF16 rounding (round to nearest even) of the value in
    the forward pass and of the incoming gradient in the backward pass."""

    @staticmethod
    def forward(ctx, t):
        return t.to(torch.bfloat16).to(t.dtype)

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.bfloat16).to(g.dtype)


class _GradBF16(torch.autograd.Function):
    """Identity in the forward pass; BF16 rounding of the gradient."""

    @staticmethod
    def forward(ctx, t):
        return t.view_as(t)

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.bfloat16).to(g.dtype)


def forward(theta: torch.Tensor, x: torch.Tensor, base: int, bf16_storage: bool = False) -> torch.Tensor:
    """x: (N, H, W, 3) -> (N, H, W, 2)."""
    L = unpack(theta, base)
    n, h, w, _ = x.shape
    st = _StoreBF16.apply if bf16_storage else (lambda t: t)
    xin = torch.zeros(n, 16, h, w, dtype=theta.dtype)
    xin[:, :3] = x.permute(0, 3, 1, 2)
    xin = st(xin)
    c = lambda t, i: st(conv(t, L[i]))
    pool = lambda t: st(F.avg_pool2d(t, 2))
    e1 = c(c(xin, 0), 1)
    e2 = c(c(pool(e1), 2), 3)
    e3 = c(c(pool(e2), 4), 5)
    e4 = c(c(pool(e3), 6), 7)
    up = lambda t: F.interpolate(t, scale_factor=2, mode="nearest")
    d3 = c(c(torch.cat([c(up(e4), 8), e3], 1), 9), 10)
    d2 = c(c(torch.cat([c(up(d3), 11), e2], 1), 12), 13)
    d1 = c(c(torch.cat([c(up(d2), 14), e1], 1), 15), 16)
    out = conv(d1, L[17], relu=False)
    if bf16_storage:
        out = _GradBF16.apply(out)
    return out[:, :2].permute(0, 2, 3, 1)


def loss_and_grad(theta: np.ndarray, x: np.ndarray, target: np.ndarray, base: int, dtype=torch.float32,
                  bf16_storage: bool = False):
    th = torch.tensor(theta, dtype=dtype, requires_grad=True)
    out = forward(th, torch.tensor(x, dtype=dtype), base, bf16_storage)
    loss = ((out - torch.tensor(target, dtype=dtype)) ** 2).mean()
    loss.backward()
    return float(loss.detach()), th.grad.numpy(), out.detach().numpy()
