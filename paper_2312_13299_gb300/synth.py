"""Seeded synthetic workloads shaped like the paper's (numpy only).

This module holds no arithmetic of the sort or of the loss: it only draws the
inputs that both the CUDA path and the CPU oracle consume.  The paper's scenes
(Mip-NeRF360, Tanks&Temples, Deep Blending, Synthetic-NeRF) are not available,
so these distributions stand in for them:

* ``rgb_uniform``: the supplementary's random 512x512x3 colour grid, U[0,1).
* ``gaussians_3dgs``: 3DGS-shaped attributes.  14 sort channels = xyz from a
  mixture of 64 anisotropic 3-D Gaussians in [-10,10]^3, scale = exp(N(-4,1))
  x3 (activated, Sec. 3.1 sorts activated values), unit quaternion x4, opacity
  = sigmoid(N(0,2)), DC colour N(0,0.5) x3; 45 carried SH-rest channels
  N(0,0.1).
* ``request_stream``: Poisson arrivals of sort requests with grid sides drawn
  uniformly from an integer range.
"""
from __future__ import annotations

import numpy as np

SORT_CHANNELS = 14
CARRIED_CHANNELS = 45


def rgb_uniform(side_h: int, side_w: int | None = None, seed: int = 0) -> np.ndarray:
    side_w = side_h if side_w is None else side_w
    rng = np.random.default_rng(seed)
    return rng.random((side_h * side_w, 3), dtype=np.float32)


def _random_rotations(rng: np.random.Generator, k: int) -> np.ndarray:
    q = rng.standard_normal((k, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    w, x, y, z = q.T
    return np.stack([
        np.stack([1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)], -1),
        np.stack([2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)], -1),
        np.stack([2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)], -1),
    ], 1)


def gaussians_3dgs(n: int, seed: int = 0, with_carried: bool = True):
    """Returns (x [n, 14] float32, carried [n, 45] float32 or None)."""
    rng = np.random.default_rng(seed)
    k = 64
    means = rng.uniform(-10.0, 10.0, (k, 3))
    stds = rng.uniform(0.2, 2.0, (k, 3))
    rots = _random_rotations(rng, k)
    comp = rng.integers(0, k, n)
    local = rng.standard_normal((n, 3)) * stds[comp]
    xyz = np.einsum("nij,nj->ni", rots[comp], local) + means[comp]
    xyz = np.clip(xyz, -10.0, 10.0)
    scale = np.exp(rng.normal(-4.0, 1.0, (n, 3)))
    quat = rng.standard_normal((n, 4))
    quat /= np.linalg.norm(quat, axis=1, keepdims=True)
    opacity = 1.0 / (1.0 + np.exp(-rng.normal(0.0, 2.0, (n, 1))))
    dc = rng.normal(0.0, 0.5, (n, 3))
    x = np.concatenate([xyz, scale, quat, opacity, dc], axis=1).astype(np.float32)
    carried = None
    if with_carried:
        carried = rng.normal(0.0, 0.1, (n, CARRIED_CHANNELS)).astype(np.float32)
    return x, carried


def loss_grid(H: int, W: int, seed: int = 0) -> np.ndarray:
    """H x W x 59 channel-last grid built from the 3DGS-shaped generator."""
    x, c = gaussians_3dgs(H * W, seed)
    return np.concatenate([x, c], axis=1).reshape(H, W, SORT_CHANNELS + CARRIED_CHANNELS)


def paper_smoothness_weights() -> np.ndarray:
    """Per-channel smoothness-loss weights of the paper's configuration
    (supplementary, Tab. "params": opacity 0.09, rotation 0.91, the other
    attributes 0) for the 59-channel layout of loss_grid: xyz 0-2, scale
    3-5, rotation 6-9, opacity 10, DC colour 11-13, SH rest 14-58."""
    lam = np.zeros(SORT_CHANNELS + CARRIED_CHANNELS, np.float32)
    lam[6:10] = 0.91
    lam[10] = 0.09
    return lam


def request_stream(n: int = 64, seed: int = 0, side_lo: int = 128, side_hi: int = 1024,
                   rate_per_s: float = 10.0):
    """n requests: (arrival time in s, grid side); exponential inter-arrivals."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_per_s, n)
    t = np.cumsum(gaps) - gaps[0]
    sides = rng.integers(side_lo, side_hi + 1, n)
    return [(float(a), int(s)) for a, s in zip(t, sides)]
