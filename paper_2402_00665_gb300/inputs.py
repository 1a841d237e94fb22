"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module only draws random numbers; it holds none of the method's
arithmetic, and both the CUDA path and the CPU oracle take their inputs from
it. Every generator is deterministic in its seed and uses numpy's PCG64
(``numpy.random.default_rng``), so the same arrays come out on x86 and Arm.

Workloads (the paper's own experiments use synthetic clouds as well, Sec. 5):

* ``uniform_points`` - FP32 xyz uniform in [0, 1]^3.
* ``gaussian_mixture_boxes`` - centres from a mixture of isotropic Gaussians
  (component centres uniform in [0, 1]^3, equal weights), half-extents
  lognormal per axis. At 30-bit codes most centres of a component share a
  Morton code, which stresses the index tie-break.
* ``gaussian_mixture_points`` - points from the same kind of mixture.
* ``batched_clouds`` - many independent uniform clouds with log-uniform sizes.
* ``random_rays`` - ray segments with uniform origins and directions.
* ``poisson_requests`` - arrival times and sizes of a served request stream.
* ``filled_cube`` / ``hollow_cube`` - the two point clouds of the paper's
  construction-rate experiment: uniform inside [-a, a]^3, and uniform on the
  six faces taken in turn, with a = n^(1/3).
* ``radius_for_neighbours`` - the ball radius that holds ``k`` expected points
  of a unit-density-``n`` uniform cloud: (3 k / (4 pi n))^(1/3).
"""
from __future__ import annotations

import math

import numpy as np


def radius_for_neighbours(n: int, k: float = 16.0) -> np.float32:
    """Radius r with (4/3) pi r^3 n = k, rounded to float32."""
    return np.float32((3.0 * k / (4.0 * math.pi * max(n, 1))) ** (1.0 / 3.0))


def uniform_points(n: int, seed: int = 0) -> np.ndarray:
    """float32[n, 3] uniform in [0, 1)^3."""
    return np.random.default_rng(seed).random((n, 3), dtype=np.float32)


def gaussian_mixture_boxes(n: int, seed: int = 0, components: int = 64, sigma: float = 0.005,
                           log_half_mu: float = math.log(1e-4), log_half_sigma: float = 0.5,
                           component_seed: int | None = None) -> np.ndarray:
    """float32[n, 6] boxes (lo.xyz, hi.xyz).

    Component centres come from ``component_seed`` (default: ``seed``) so a
    query set can be drawn from the same mixture with a different ``seed``.
    """
    crng = np.random.default_rng(seed if component_seed is None else component_seed)
    centres = crng.random((components, 3))
    rng = np.random.default_rng([seed, 1])
    which = rng.integers(0, components, size=n)
    c = centres[which] + rng.normal(0.0, sigma, size=(n, 3))
    h = rng.lognormal(log_half_mu, log_half_sigma, size=(n, 3))
    out = np.empty((n, 6), np.float32)
    out[:, :3] = (c - h).astype(np.float32)
    out[:, 3:] = (c + h).astype(np.float32)
    return out


def gaussian_mixture_points(n: int, seed: int = 0, components: int = 64, sigma: float = 0.005) -> np.ndarray:
    """float32[n, 3] points from a mixture of isotropic Gaussians (component
    centres uniform in [0, 1]^3, equal weights)."""
    crng = np.random.default_rng(seed)
    centres = crng.random((components, 3))
    rng = np.random.default_rng([seed, 3])
    which = rng.integers(0, components, size=n)
    return (centres[which] + rng.normal(0.0, sigma, size=(n, 3))).astype(np.float32)


def random_rays(count: int, seed: int = 0, tmax: float = np.inf) -> np.ndarray:
    """float32[count, 8] ray segments {origin.xyz, tmin = 0, direction.xyz,
    tmax}: origins uniform in [0, 1)^3, directions uniform on the unit sphere
    (normalised Gaussian triples)."""
    rng = np.random.default_rng(seed)
    out = np.zeros((count, 8), np.float32)
    out[:, :3] = rng.random((count, 3))
    d = rng.normal(size=(count, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    out[:, 4:7] = d
    out[:, 7] = tmax
    return out


def cloud_sizes(count: int, lo: int, hi: int, seed: int = 1) -> np.ndarray:
    """int64[count] sizes floor(exp(U(ln lo, ln hi)))."""
    rng = np.random.default_rng(seed)
    return np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def batched_clouds(count: int = 4096, lo: int = 256, hi: int = 262144, seed: int = 1):
    """Sizes and one concatenated float32[sum, 3] array of uniform clouds."""
    sizes = cloud_sizes(count, lo, hi, seed)
    pts = np.random.default_rng([seed, 2]).random((int(sizes.sum()), 3), dtype=np.float32)
    return sizes, pts


def poisson_requests(count: int, rate_per_s: float = 2000.0, lo: int = 1024, hi: int = 4194304,
                     seed: int = 2):
    """Arrival times (s), sizes and a mixture flag (0 uniform, 1 Gaussian mixture)."""
    rng = np.random.default_rng(seed)
    arrivals = np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
    sizes = np.floor(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)
    kinds = rng.integers(0, 2, size=count)
    return arrivals, sizes, kinds


def filled_cube(n: int, seed: int = 0) -> np.ndarray:
    a = float(n) ** (1.0 / 3.0)
    return np.random.default_rng(seed).uniform(-a, a, size=(n, 3)).astype(np.float32)


def hollow_cube(n: int, seed: int = 0) -> np.ndarray:
    """Points on the faces of [-a, a]^3, face i % 6 for point i."""
    a = float(n) ** (1.0 / 3.0)
    rng = np.random.default_rng(seed)
    uv = rng.uniform(-a, a, size=(n, 2))
    out = np.empty((n, 3), np.float64)
    face = np.arange(n) % 6
    axis = face // 2
    side = np.where(face % 2 == 0, -a, a)
    for ax in range(3):
        m = axis == ax
        others = [k for k in range(3) if k != ax]
        out[m, ax] = side[m]
        out[m, others[0]] = uv[m, 0]
        out[m, others[1]] = uv[m, 1]
    return out.astype(np.float32)


def duplicated_points(n: int, distinct: int, seed: int = 0) -> np.ndarray:
    """n points drawn (with repetition) from ``distinct`` uniform points."""
    rng = np.random.default_rng(seed)
    base = rng.random((max(distinct, 1), 3), dtype=np.float32)
    return base[rng.integers(0, max(distinct, 1), size=n)]


def collinear_points(n: int, seed: int = 0) -> np.ndarray:
    """Points on the x axis (zero extent in y and z)."""
    rng = np.random.default_rng(seed)
    p = np.zeros((n, 3), np.float32)
    p[:, 0] = rng.random(n, dtype=np.float32)
    return p
