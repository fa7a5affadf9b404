"""Seeded synthetic image-factorisation problems.

This module is the one piece shared by the CUDA path's callers (tests, bench) and
by the FP64 oracle's callers: it draws inputs and holds none of the
factorisation's arithmetic (no restriction, prolongation, sweep or objective).

Workload shape (stand-in for the image datasets of Section 5, Table 2, which are
not available): each column of M is an image on an H x W pixel grid, vectorised
row-major (pixel (y, x) -> row y*W + x).  M = max(0, V0 W0 + N) where

* V0 (m x r): column k is a sum of three isotropic Gaussian bumps with amplitude
  U[0.5, 1], continuous centre U[0, H-1] x U[0, W-1] and width ``sigma``;
* W0 (r x n): Exp(1) entries, each zeroed with probability 1/2;
* N: Gaussian noise with standard deviation 1 % of mean(V0 W0).

The initial iterate (V, W) is U[0, 1] drawn from ``init_seed`` (0 by default).
Every array is produced in float64 and rounded once to float32; callers that
need float64 (the oracle) widen the float32 values, so both sides see the same
numbers exactly.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), evaluated counter-style: the
i-th draw of a stream is mix64(key + (i + 1) * 0x9E3779B97F4A7C15).  Uniforms use
the top 53 bits, Gaussians Box-Muller, exponentials -log(1 - U).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)

# stream identifiers: one independent SplitMix64 stream per drawn quantity
STREAM_V0, STREAM_W0, STREAM_NOISE, STREAM_V_INIT, STREAM_W_INIT = 1, 2, 3, 4, 5


def _mix64(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    z = (z ^ (z >> np.uint64(30))) * _MIX1
    z = (z ^ (z >> np.uint64(27))) * _MIX2
    return z ^ (z >> np.uint64(31))


def _stream_key(seed: int, stream: int) -> np.uint64:
    base = np.array([(seed & 0xFFFFFFFFFFFFFFFF)], dtype=np.uint64)
    k = _mix64(base ^ _mix64(np.array([stream], dtype=np.uint64)))
    return k[0]


def splitmix64(seed: int, stream: int, count: int) -> np.ndarray:
    """``count`` raw 64-bit draws of stream ``stream`` under ``seed``."""
    key = _stream_key(seed, stream)
    ctr = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix64(key + ctr * _GOLDEN)


def uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """U[0, 1) doubles with 53 random bits."""
    return (splitmix64(seed, stream, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian(seed: int, stream: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs."""
    half = (count + 1) // 2
    u = uniform(seed, stream, 2 * half)
    u1 = 1.0 - u[0::2]  # in (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * half)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count]


def exponential(seed: int, stream: int, count: int) -> np.ndarray:
    """Exp(1) draws."""
    return -np.log1p(-uniform(seed, stream, count))


@dataclass
class Problem:
    """One synthetic instance; all arrays float32, row-major."""

    M: np.ndarray  # m x n, >= 0
    V: np.ndarray  # m x r initial iterate
    W: np.ndarray  # r x n initial iterate
    grid_h: int
    grid_w: int
    r: int
    V0: np.ndarray  # m x r planted basis
    W0: np.ndarray  # r x n planted weights

    @property
    def m(self) -> int:
        return self.M.shape[0]

    @property
    def n(self) -> int:
        return self.M.shape[1]


def planted_basis(grid_h: int, grid_w: int, r: int, sigma: float, seed: int) -> np.ndarray:
    """V0: each column the sum of three Gaussian bumps on the pixel grid (float64)."""
    u = uniform(seed, STREAM_V0, r * 3 * 3).reshape(r, 3, 3)
    yy, xx = np.meshgrid(np.arange(grid_h, dtype=np.float64), np.arange(grid_w, dtype=np.float64), indexing="ij")
    V0 = np.zeros((grid_h * grid_w, r))
    for k in range(r):
        col = np.zeros((grid_h, grid_w))
        for b in range(3):
            amp = 0.5 + 0.5 * u[k, b, 0]
            cy = u[k, b, 1] * (grid_h - 1)
            cx = u[k, b, 2] * (grid_w - 1)
            col += amp * np.exp(-((yy - cy) ** 2 + (xx - cx) ** 2) / (2.0 * sigma * sigma))
        V0[:, k] = col.reshape(-1)
    return V0


def planted_weights(r: int, n: int, seed: int) -> np.ndarray:
    """W0: Exp(1) entries, each kept with probability 1/2 (float64)."""
    e = exponential(seed, STREAM_W0, r * n).reshape(r, n)
    keep = uniform(seed, STREAM_W0 + 100, r * n).reshape(r, n) >= 0.5
    return np.where(keep, e, 0.0)


def planted_weights_sequence(r: int, n: int, seed: int) -> np.ndarray:
    """W0 for image sequences (video frames, spectral bands): row k is smooth along the
    sequence, a_k exp(-(j - c_k)^2 / (2 s^2)) (1 + cos(2 pi f_k j / n + phi_k)) / 2 with
    a_k ~ Exp(1), c_k ~ U[0, n), s = n / 6, f_k ~ U[0.5, 3], phi_k ~ U[0, 2 pi) (float64)."""
    a = exponential(seed, STREAM_W0 + 200, r)
    u = uniform(seed, STREAM_W0 + 300, r * 3).reshape(r, 3)
    j = np.arange(n, dtype=np.float64)
    s = n / 6.0
    W0 = np.zeros((r, n))
    for k in range(r):
        c, f, phi = u[k, 0] * n, 0.5 + 2.5 * u[k, 1], 2.0 * np.pi * u[k, 2]
        W0[k] = a[k] * np.exp(-((j - c) ** 2) / (2.0 * s * s)) * 0.5 * (1.0 + np.cos(2.0 * np.pi * f * j / n + phi))
    return W0


def initial_iterate(m: int, n: int, r: int, init_seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """(V, W) ~ U[0, 1], float32."""
    V = uniform(init_seed, STREAM_V_INIT, m * r).reshape(m, r).astype(np.float32)
    W = uniform(init_seed, STREAM_W_INIT, r * n).reshape(r, n).astype(np.float32)
    return V, W


def make_problem(grid_h: int, grid_w: int, n: int, r: int, sigma: float | None = None,
                 data_seed: int = 1, init_seed: int = 0, noise: float = 0.01, sequence: bool = False) -> Problem:
    """Draw M = max(0, V0 W0 + N) and the U[0,1] initial iterate.

    ``sigma`` defaults to 2 px.  ``noise`` is the noise level relative to
    mean(V0 W0); 0 gives the exact planted factorisation M = V0 W0.  ``sequence``:
    the columns form a smooth sequence (planted_weights_sequence) instead of
    independent images.
    """
    if sigma is None:
        sigma = 2.0
    m = grid_h * grid_w
    V0 = planted_basis(grid_h, grid_w, r, sigma, data_seed)
    W0 = planted_weights_sequence(r, n, data_seed) if sequence else planted_weights(r, n, data_seed)
    X = V0 @ W0
    if noise > 0:
        X = X + noise * X.mean() * gaussian(data_seed, STREAM_NOISE, m * n).reshape(m, n)
    M = np.maximum(X, 0.0).astype(np.float32)
    V, W = initial_iterate(m, n, r, init_seed)
    return Problem(M=M, V=V, W=W, grid_h=grid_h, grid_w=grid_w, r=r,
                   V0=V0.astype(np.float32), W0=W0.astype(np.float32))


# Workload shapes: (grid_h, grid_w, n, r, sigma)
WORKLOADS = {
    # 16x16 grid, 1000 images, r = 10
    "grid16_n1000_r10": (16, 16, 1000, 10, 2.0),
    # 19x19 grid (CBCL face shape), 2429 images, r = 49
    "grid19_n2429_r49": (19, 19, 2429, 49, 2.0),
    # 112x92 grid (ORL face shape), 400 images, r = 40, sigma = 4 % of grid width
    "grid112x92_n400_r40": (112, 92, 400, 40, 0.04 * 92),
    # 256x256 grid, 2000 images, r = 64, sigma = 4 % of grid width
    "grid256_n2000_r64": (256, 256, 2000, 64, 0.04 * 256),
}

# Image sequences (make_problem(..., sequence=True)): (grid_h, grid_w, n, r, sigma)
SEQUENCE_WORKLOADS = {
    # 16x16 frames, 1024 of them, r = 10
    "seq16_n1024_r10": (16, 16, 1024, 10, 2.0),
    # 32x32 frames, 4096 of them, r = 16, sigma = 3 px
    "seq32_n4096_r16": (32, 32, 4096, 16, 3.0),
}


def batched_sizes(count: int = 64, seed0: int = 0) -> list[tuple[int, int, int]]:
    """Uneven problem sizes (side, n, r): side from {16,19,32,64,92,128}, n ~ U[200,4000], r ~ U[5,64]."""
    sides = (16, 19, 32, 64, 92, 128)
    out = []
    for i in range(count):
        u = uniform(seed0 + i, 77, 3)
        side = sides[min(int(u[0] * len(sides)), len(sides) - 1)]
        n = 200 + min(int(u[1] * 3801), 3800)
        r = 5 + min(int(u[2] * 60), 59)
        out.append((side, n, r))
    return out
