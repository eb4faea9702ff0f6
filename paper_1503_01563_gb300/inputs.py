"""Seeded synthetic problem generators.

This module is the only code shared between the CUDA path's tests/benchmarks
and the CPU oracle.  It draws problem data (unary terms w and edge weights a)
and holds none of the solver's arithmetic.  Every generator takes an explicit
seed and uses numpy's PCG64, so the integer problems are identical on every
platform.

Workloads (stand-ins for the vision grids of the paper's experiments, whose
max-flow benchmark datasets are not available here):

- ``uniform_grid``: w ~ U{-50..50}, a ~ U{1..20} per edge, int32 (the small
  exact-check grid and each grid of the batched workload); ``uniform_grid8``
  the same on a 2D 8-connected grid (four weight arrays).
- ``segmentation_problem``: a blob image (sum of Gaussian blobs plus N(0, 0.1^2)
  noise, clipped to [0, 1]) turned into a two-class segmentation energy:
  unary = log-likelihood ratio of N(0.8, 0.15^2) vs N(0.2, 0.15^2), edge weight
  10 * exp(-(I_i - I_j)^2 / (2 * 0.05^2)); ``to_integer`` scales both by 100
  and rounds (weights at least 1) for exact min-cut checks.
- ``volume_problem``: the same unary on a 3D blob volume with integer edge
  weights ~ U{1..30}.
- ``batch_dims``: grid sizes H ~ U{64..1024}, W ~ U{64..768}.

Weights are returned per axis in compact layout: axis k's array has the grid
shape with dims[k] - 1 along axis k.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def compact_shape(dims, axis: int):
    return tuple(d - 1 if k == axis else d for k, d in enumerate(dims))


def uniform_grid(dims, seed: int, w_range=(-50, 50), a_range=(1, 20)):
    """w int32 uniform in w_range (inclusive), one int32 weight array per axis
    uniform in a_range (inclusive)."""
    g = _rng(seed)
    dims = tuple(int(d) for d in dims)
    w = g.integers(w_range[0], w_range[1], size=dims, endpoint=True, dtype=np.int64).astype(np.int32)
    a = [g.integers(a_range[0], a_range[1], size=compact_shape(dims, k), endpoint=True,
                    dtype=np.int64).astype(np.int32) for k in range(len(dims))]
    return w, a


def uniform_grid8(dims, seed: int, w_range=(-50, 50), a_range=(1, 20)):
    """A 2D 8-connected grid: w int32 uniform in w_range and four int32 weight
    arrays uniform in a_range: vertical (H-1, W), horizontal (H, W-1),
    diagonal (r, c)-(r+1, c+1) and anti-diagonal (r, c+1)-(r+1, c), both
    (H-1, W-1)."""
    g = _rng(seed)
    H, W = (int(d) for d in dims)
    w = g.integers(w_range[0], w_range[1], size=(H, W), endpoint=True, dtype=np.int64).astype(np.int32)
    shapes = [(H - 1, W), (H, W - 1), (max(H - 1, 0), max(W - 1, 0)), (max(H - 1, 0), max(W - 1, 0))]
    a = [g.integers(a_range[0], a_range[1], size=sh, endpoint=True, dtype=np.int64).astype(np.int32)
         for sh in shapes]
    return w, a


def blob_image(dims, seed: int, nblobs: int = 20, noise: float = 0.1,
               sigma_px=(20.0, 120.0), amp=(0.3, 1.0)) -> np.ndarray:
    """Sum of `nblobs` isotropic Gaussian blobs with uniform centres, widths
    uniform in sigma_px scaled by min(dims)/1024, amplitudes uniform in amp,
    plus N(0, noise^2) noise, clipped to [0, 1].  FP64, shape dims."""
    g = _rng(seed)
    dims = tuple(int(d) for d in dims)
    scale = min(dims) / 1024.0
    img = np.zeros(dims, dtype=np.float64)
    coords = [np.arange(d, dtype=np.float64) for d in dims]
    for _ in range(nblobs):
        c = [g.uniform(0, d) for d in dims]
        s = g.uniform(sigma_px[0], sigma_px[1]) * scale
        h = g.uniform(amp[0], amp[1])
        prof = [np.exp(-((coords[k] - c[k]) ** 2) / (2.0 * s * s)) for k in range(len(dims))]
        blob = prof[0]
        for p in prof[1:]:
            blob = np.multiply.outer(blob, p)
        img += h * blob
    img += g.normal(0.0, noise, size=dims)
    np.clip(img, 0.0, 1.0, out=img)
    return img


def segmentation_terms(img: np.ndarray, mu=(0.2, 0.8), sigma: float = 0.15,
                       contrast: float = 10.0, beta: float = 0.05):
    """Two-class Gaussian log-likelihood-ratio unary and contrast-sensitive
    edge weights of an image (FP64)."""
    w = ((img - mu[0]) ** 2 - (img - mu[1]) ** 2) / (2.0 * sigma * sigma)
    a = []
    for k in range(img.ndim):
        d = np.diff(img, axis=k)
        a.append(contrast * np.exp(-(d * d) / (2.0 * beta * beta)))
    return w, a


def to_integer(w, a, scale: float = 100.0):
    """Scale by `scale` and round to int32; weights are at least 1."""
    wi = np.rint(np.asarray(w, dtype=np.float64) * scale).astype(np.int32)
    ai = [np.maximum(1, np.rint(np.asarray(x, dtype=np.float64) * scale)).astype(np.int32) for x in a]
    return wi, ai


def segmentation_problem(dims, seed: int, integer: bool = True, scale: float = 100.0):
    """Blob-image segmentation energy on a 2D (or 3D) grid."""
    img = blob_image(dims, seed)
    w, a = segmentation_terms(img)
    if integer:
        return to_integer(w, a, scale)
    return w.astype(np.float32), [x.astype(np.float32) for x in a]


def segmentation_problem8(dims, seed: int, scale: float = 100.0, contrast: float = 10.0, beta: float = 0.05):
    """The blob-image segmentation energy on a 2D 8-connected grid: weights
    [vertical, horizontal, diagonal (r, c)-(r+1, c+1), anti-diagonal
    (r, c+1)-(r+1, c)], the contrast formula on each neighbour pair, the two
    diagonal directions scaled by 1/sqrt(2); integer-scaled like to_integer."""
    img = blob_image(dims, seed)
    w, a = segmentation_terms(img, contrast=contrast, beta=beta)
    cw = lambda d: contrast * np.exp(-(d * d) / (2.0 * beta * beta))
    ad = cw(img[1:, 1:] - img[:-1, :-1]) / np.sqrt(2.0)
    aa = cw(img[1:, :-1] - img[:-1, 1:]) / np.sqrt(2.0)
    return to_integer(w, a + [ad, aa], scale)


def volume_problem(dims, seed: int, a_range=(1, 30), scale: float = 100.0):
    """3D blob-volume unary (integer-scaled LLR) with int32 edge weights
    uniform in a_range."""
    img = blob_image(dims, seed)
    w, _ = segmentation_terms(img)
    w = np.rint(w * scale).astype(np.int32)
    g = _rng(seed + 7919)
    a = [g.integers(a_range[0], a_range[1], size=compact_shape(dims, k), endpoint=True,
                    dtype=np.int64).astype(np.int32) for k in range(len(dims))]
    return w, a


def batch_dims(count: int, seed: int, h_range=(64, 1024), w_range=(64, 768)):
    g = _rng(seed)
    hs = g.integers(h_range[0], h_range[1], size=count, endpoint=True)
    ws = g.integers(w_range[0], w_range[1], size=count, endpoint=True)
    return [(int(h), int(w)) for h, w in zip(hs, ws)]


def random_chain(m: int, seed: int, scale: float = 10.0, a_scale: float = 3.0):
    """A random chain (v, a) for prox tests: v ~ N(0, scale^2) with a few
    steps, a ~ U[0, a_scale]."""
    g = _rng(seed)
    v = g.normal(0.0, scale, size=m)
    if m > 4:
        steps = g.integers(0, m, size=3)
        for s in steps:
            v[s:] += g.normal(0.0, 3 * scale)
    a = g.uniform(0.0, a_scale, size=max(m - 1, 0))
    return v, a
