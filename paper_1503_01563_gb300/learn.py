"""Learned warm start: data generation, training and use of the U-Net.

The product-space iteration (Sec. 4) starts from z = 0.  Sec. 4.4 warm-starts
it from the dual variables y_k of a similar, earlier problem.  Here a U-Net
predicts those per-block duals directly from the problem (unary and edge
weights) and the solver starts from z = y_hat.  Training pairs come from the
method itself: a batched solve of many generated problems, whose final shadow
y_k = Pi_{K_k}(z_k) (the chain projection of the converged state) is the
target.  Everything numerical runs in libtvcut's kernels; this module only
arranges calls and tensors.

Scale: the TV solution is jointly homogeneous in (w, a), so inputs and targets
are divided by s = max(max|w|, max a) of each problem.
"""
from __future__ import annotations

import numpy as np

from . import inputs, tvcut


def features(w, a):
    """(H, W, 3) float32 features [w, a_down, a_right] / s and the scale s, on
    the host (training data; tvcut_unet_predict_state builds the same
    features on the device for a solver's problem).  a[0]: (H-1, W) vertical
    weights, a[1]: (H, W-1) horizontal weights."""
    H, W = w.shape
    f = np.zeros((H, W, 3), dtype=np.float32)
    s = float(max(np.abs(w).max(), max(x.max() for x in a), 1e-12))
    f[:, :, 0] = w / s
    f[:-1, :, 1] = a[0] / s
    f[:, :-1, 2] = a[1] / s
    return f, s


def solve_targets(problems, iters: int, stream=None, dtype=tvcut.F32):
    """Batched solve of `problems` [(w, a)] for `iters` AAR iterations; returns
    per problem the two block duals y_k (2, H, W) of the final state."""
    import torch
    dims = [p[0].shape for p in problems]
    b = tvcut.Batch(dims, dtype=dtype, stream=stream)
    for g, (w, a) in enumerate(problems):
        b.set_problem(g, torch.from_numpy(np.ascontiguousarray(w)).cuda(),
                      [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in a])
    b.reset()
    b.iterate(iters)
    tdt = torch.float64 if dtype == tvcut.F64 else torch.float32
    out = []
    for g, (w, a) in enumerate(problems):
        z = torch.from_numpy(b.state(g)).cuda()
        y = torch.empty_like(z)
        for k in range(2):
            ak = torch.from_numpy(a[k].astype(np.float64 if dtype == tvcut.F64 else np.float32)).cuda()
            tvcut.tvcut_project_chains(w.shape, k, z[k].contiguous(), ak, y[k], what=0)
        out.append(y.to(tdt))
    torch.cuda.synchronize()
    b.close()
    return out


def make_training_set(n: int, H: int, W: int, seed: int, iters: int = 800, chunk: int = 1024):
    """n generated problems (w ~ U{-50..50}, a ~ U{1..20}) with their solver
    targets, as CUDA tensors X (n, H, W, 3) and Y (n, H, W, 2)."""
    import torch
    X = torch.empty((n, H, W, 3), dtype=torch.float32, device="cuda")
    Y = torch.empty((n, H, W, 2), dtype=torch.float32, device="cuda")
    for c0 in range(0, n, chunk):
        probs = [inputs.uniform_grid((H, W), seed * 1_000_003 + i) for i in range(c0, min(n, c0 + chunk))]
        ys = solve_targets(probs, iters)
        for j, ((w, a), y) in enumerate(zip(probs, ys)):
            f, s = features(w, a)
            X[c0 + j] = torch.from_numpy(f).cuda()
            Y[c0 + j] = (y / s).permute(1, 2, 0)
    return X, Y


def train(net, X, Y, steps: int, batch: int, lr: float = 1e-3, seed: int = 0, lr_final: float = 1e-4):
    """Adam on random minibatches (cosine learning-rate decay); returns the
    loss history."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    n = X.shape[0]
    H, W = X.shape[1], X.shape[2]
    net.resize(batch, H, W)
    hist = []
    for t in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g).cuda()
        xb = X.index_select(0, idx).contiguous()
        yb = Y.index_select(0, idx).contiguous()
        net.forward(xb)
        hist.append(net.backward(yb))
        cur = lr_final + 0.5 * (lr - lr_final) * (1 + np.cos(np.pi * t / max(1, steps - 1)))
        net.adam(lr=float(cur))
    return hist


def predict_state(net, solver):
    """Warm-start `solver` (a 2D 4-connected tvcut.Solver whose problem is
    set) from the network's predicted block duals: features, inference and
    the rescaling to the problem all run on the device
    (tvcut_unet_predict_state).  H and W must be multiples of 8."""
    net.predict_state(solver)
