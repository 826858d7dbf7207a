"""Seeded synthetic inputs for the circular-geometry PAT/TAT operators.

This module is shared by the FP64 oracle, the tests and the benchmark.  It
holds no arithmetic of the operators themselves: only a counter-based random
stream, the random-ellipse phantoms, white Gaussian noise and region-of-
interest masks.

Workloads follow the paper's description of its test objects: "smoothed
characteristic functions" (Section 4.1) and training sets of randomly
generated ellipses (Section 4.2.1).  The paper's own phantom and training set
are not published, so the recipe below is a stand-in:

* E ~ U{5..20} ellipses per image;
* centre at radius sqrt(U)*0.6 with a uniform angle;
* semi-axes a, b ~ U(0.05, 0.3); rotation ~ U(0, pi); intensity ~ U(0, 1);
* overlapping ellipses add; every ellipse lies inside radius 0.9;
* values are sampled at the nodes x_i = -1 + 2 i/(n-1) of the node-centred
  n x n grid on [-1, 1]^2 (unit radius detector circle);
* ``smooth`` > 0 replaces the sharp edge by a C^1 ramp of that width.

Noise (Section 4.3): delta = eps * ||A f||_2 * xi / ||xi||_2 with xi iid N(0,1).
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Counter-based SplitMix64: element i is mix(seed + (offset+i+1)*golden)."""
    with np.errstate(over="ignore"):
        ctr = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + ctr * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of the SplitMix64 stream."""
    z = splitmix64(seed, count, offset)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def gaussian(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """iid N(0,1) by the Box-Muller transform of pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m, 2 * offset)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])
    out = np.empty(2 * m)
    out[0::2] = z[:m]
    out[1::2] = z[m:]
    return out[:count]


def ellipse_params(seed: int) -> np.ndarray:
    """Rows (cx, cy, a, b, rot, intensity) of one random-ellipse phantom."""
    e = 5 + int(uniform(seed, 1)[0] * 16)
    u = uniform(seed, 6 * e, offset=1).reshape(e, 6)
    r = np.sqrt(u[:, 0]) * 0.6
    ang = 2 * np.pi * u[:, 1]
    a = 0.05 + 0.25 * u[:, 2]
    b = 0.05 + 0.25 * u[:, 3]
    rot = np.pi * u[:, 4]
    inten = u[:, 5]
    return np.stack([r * np.cos(ang), r * np.sin(ang), a, b, rot, inten], axis=1)


def ellipse_phantom(n: int, seed: int, smooth: float = 0.0) -> np.ndarray:
    """One n x n phantom (float64, row iy = y index, column ix = x index)."""
    x = -1.0 + 2.0 * np.arange(n) / (n - 1)
    X, Y = np.meshgrid(x, x, indexing="xy")
    f = np.zeros((n, n))
    for cx, cy, a, b, rot, inten in ellipse_params(seed):
        c, s = np.cos(rot), np.sin(rot)
        xr = (X - cx) * c + (Y - cy) * s
        yr = -(X - cx) * s + (Y - cy) * c
        rho = np.sqrt((xr / a) ** 2 + (yr / b) ** 2)
        if smooth > 0:
            d = (1.0 - rho) * min(a, b) / smooth + 0.5
            d = np.clip(d, 0.0, 1.0)
            f += inten * d * d * (3.0 - 2.0 * d)
        else:
            f += inten * (rho <= 1.0)
    return f


def phantom_batch(n: int, batch: int, seed0: int = 0, smooth: float = 0.0) -> np.ndarray:
    """Images seed0 .. seed0+batch-1 stacked as (batch, n, n) float64."""
    return np.stack([ellipse_phantom(n, seed0 + s, smooth) for s in range(batch)])


def random_sinogram(n_det: int, n_t: int, seed: int) -> np.ndarray:
    """A dense N(0,1) field on the detector/time grid, used to probe A*."""
    return gaussian(seed, n_det * n_t).reshape(n_det, n_t)


def add_noise(g: np.ndarray, eps: float, seed: int) -> np.ndarray:
    """g + eps*||g||*xi/||xi|| (relative white Gaussian noise)."""
    xi = gaussian(seed, g.size).reshape(g.shape)
    return g + eps * np.linalg.norm(g) * xi / np.linalg.norm(xi)


def roi_mask(n: int, radius: float = 0.98, upper_half: bool = False) -> np.ndarray:
    """Region of interest Omega_0 as an n x n 0/1 array (f[iy, ix]).

    The disk |x| <= radius of the node-centred grid, optionally cut to its
    upper half y >= 0 (the visible half for detectors on theta in [0, pi),
    Section 4.4).  An input choice of the caller, not part of A.
    """
    s = (2 * np.arange(n) - (n - 1)).astype(np.float64)   # (n-1) * x_i
    rr = (radius * (n - 1)) ** 2
    m = (s[None, :] ** 2 + s[:, None] ** 2) <= rr
    if upper_half:
        m &= (s[:, None] >= 0)
    return m.astype(np.float64)
