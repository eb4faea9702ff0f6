"""CPU oracle of the warm-start U-Net (plain PyTorch CPU ops, FP32 or FP64).

TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg).  It builds
the network described in include/tvcut.h from the same flat parameter vector:
for each of the 18 convolutions in forward order, weights [9][Cout][Cin]
(tap 3*ky + kx reads pixel (y + ky - 1, x + kx - 1), zero padding) then bias
[Cout]; 2x2 average pooling, nearest 2x upsampling, concatenation
[upsampled, skip]; ReLU after every convolution but the last; input padded
from 3 to 16 channels with zeros; output channels 0 and 1; loss = mean
squared error over those two channels.  Gradients come from autograd; the
pins in tests/test_oracle_unet.py check them against finite differences and
the convolution against a direct loop.
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


def forward(theta: torch.Tensor, x: torch.Tensor, base: int) -> torch.Tensor:
    """x: (N, H, W, 3) -> (N, H, W, 2)."""
    L = unpack(theta, base)
    n, h, w, _ = x.shape
    xin = torch.zeros(n, 16, h, w, dtype=theta.dtype)
    xin[:, :3] = x.permute(0, 3, 1, 2)
    e1 = conv(conv(xin, L[0]), L[1])
    e2 = conv(conv(F.avg_pool2d(e1, 2), L[2]), L[3])
    e3 = conv(conv(F.avg_pool2d(e2, 2), L[4]), L[5])
    e4 = conv(conv(F.avg_pool2d(e3, 2), L[6]), L[7])
    up = lambda t: F.interpolate(t, scale_factor=2, mode="nearest")
    d3 = conv(conv(torch.cat([conv(up(e4), L[8]), e3], 1), L[9]), L[10])
    d2 = conv(conv(torch.cat([conv(up(d3), L[11]), e2], 1), L[12]), L[13])
    d1 = conv(conv(torch.cat([conv(up(d2), L[14]), e1], 1), L[15]), L[16])
    out = conv(d1, L[17], relu=False)
    return out[:, :2].permute(0, 2, 3, 1)


def loss_and_grad(theta: np.ndarray, x: np.ndarray, target: np.ndarray, base: int, dtype=torch.float32):
    th = torch.tensor(theta, dtype=dtype, requires_grad=True)
    out = forward(th, torch.tensor(x, dtype=dtype), base)
    loss = ((out - torch.tensor(target, dtype=dtype)) ** 2).mean()
    loss.backward()
    return float(loss.detach()), th.grad.numpy(), out.detach().numpy()
