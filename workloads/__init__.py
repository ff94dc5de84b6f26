"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the method: it only draws point clouds and
white noise from numpy's PCG64 generator (FP64 draws rounded to FP32), with
the shapes and distributions of the paper's workloads:

* ``unit_gaussian``  -- 3-D standard normal (the benchmark cloud of Fig. 1 and
  Fig. 2);
* ``uniform_cube``   -- i.i.d. uniform in [0, 1]^3;
* ``ldr_cloud``      -- large dynamic range: 90 % radii log-uniform in
  [1e-3, 1] with isotropic directions, 10 % uniform in [-1, 1]^3;
* ``blobs``          -- mixture of Gaussian blobs with log-uniform widths plus a
  uniform background in [0, 1]^3;
* ``white_noise``    -- xi ~ N(0, 1) in FP32.
"""
from __future__ import annotations

import numpy as np

MATERN12, MATERN32, MATERN52, SQEXP = 0, 1, 2, 3


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_cube(N: int, seed: int) -> np.ndarray:
    return _rng(seed).random((N, 3)).astype(np.float32)


def unit_gaussian(N: int, seed: int) -> np.ndarray:
    return _rng(seed).standard_normal((N, 3)).astype(np.float32)


def ldr_cloud(N: int, seed: int, background: float = 0.1) -> np.ndarray:
    rng = _rng(seed)
    nb = int(round(background * N))
    nc = N - nb
    d = rng.standard_normal((nc, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = 10.0 ** rng.uniform(-3.0, 0.0, size=(nc, 1))
    core = d * r
    bg = rng.uniform(-1.0, 1.0, size=(nb, 3))
    pts = np.concatenate([core, bg], axis=0)
    return pts[rng.permutation(N)].astype(np.float32)


def blobs(N: int, seed: int, n_blobs: int = 10_000, background: float = 0.1,
          log10_width=(-4.0, -1.0), chunk: int = 1 << 24) -> np.ndarray:
    rng = _rng(seed)
    centres = rng.random((n_blobs, 3))
    widths = 10.0 ** rng.uniform(log10_width[0], log10_width[1], size=n_blobs)
    out = np.empty((N, 3), np.float32)
    nb = int(round(background * N))
    for s in range(0, N, chunk):
        e = min(N, s + chunk)
        n = e - s
        which = rng.integers(0, n_blobs, size=n)
        pts = centres[which] + widths[which, None] * rng.standard_normal((n, 3))
        is_bg = np.arange(s, e) < nb
        if is_bg.any():
            pts[is_bg] = rng.random((int(is_bg.sum()), 3))
        out[s:e] = pts
    return out


def white_noise(N: int, seed: int) -> np.ndarray:
    return _rng(seed).standard_normal(N).astype(np.float32)


def cloud(kind: str, N: int, seed: int) -> np.ndarray:
    return {"uniform": uniform_cube, "gaussian": unit_gaussian, "ldr": ldr_cloud,
            "blobs": blobs}[kind](N, seed)


# Workloads with the shapes of the configurations the method is measured on.
WORKLOADS = {
    # tiny: uniform cube, Matern-3/2 (s2=1, l=0.1, nugget 1e-6), k=8
    "tiny": dict(cloud="uniform", N=4096, k=8, kernel=(MATERN32, 1.0, 0.1, 1e-6), seed=0, xi_seed=1),
    # large dynamic range, Matern-3/2 l=0.05, no nugget, k=16
    "ldr": dict(cloud="ldr", N=1 << 20, k=16, kernel=(MATERN32, 1.0, 0.05, 0.0), seed=2, xi_seed=3),
    # differentiation: uniform cube, squared exponential l=0.03, nugget 1e-4, k=32
    "diff": dict(cloud="uniform", N=1 << 22, k=32, kernel=(SQEXP, 1.0, 0.03, 1e-4), seed=4, xi_seed=5),
    # headline: unit Gaussian cloud, N=2^26, k=16, Matern-3/2 l=0.1, nugget 1e-6
    "metric": dict(cloud="gaussian", N=1 << 26, k=16, kernel=(MATERN32, 1.0, 0.1, 1e-6), seed=6, xi_seed=7),
    # scale: 1e4 blobs + 10 % background, N=2^29, k=16, Matern-3/2 l=0.02, nugget 1e-6
    "scale": dict(cloud="blobs", N=1 << 29, k=16, kernel=(MATERN32, 1.0, 0.02, 1e-6), seed=9, xi_seed=10),
}
