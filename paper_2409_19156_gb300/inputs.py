"""Seeded synthetic inputs: mode lists, points, coefficient sets and the batched mix.

This module holds no Zernike arithmetic. It only draws or lays out inputs, so both the
CUDA path (tests, benchmark) and the CPU oracle's tests can use it.

Mode-number rule (paper Sec. 2, the sentence after the binomial radial sum): n >= 0,
|m| <= n and n - |m| even.  The paper prints no output-column order; full sets here use
n ascending, then m ascending (m from -n to n in steps of 2 for Z, 0..n for R).

Workload recipes (sizes, distributions) follow the five named workloads:
  * basis_n20:     full Z set n <= 20 (231 modes), 1000 points, r ~ U[0,1], theta ~ U[0,2pi)
  * radial_n100:   0 <= m <= n <= 100 (2601 modes), 100000 Chebyshev-Gauss points in [0,1]
  * series_n24:    full Z set n <= 24 (325 modes), 250x200 polar grid (Gauss-Legendre in r^2),
                   256 coefficient sets, c_nm ~ N(0, 1/(n+1)^2)
  * mixed_n32:     full Z set n <= 32 (561 modes), 1e6 points r = sqrt(U), theta ~ U,
                   4096 coefficient sets, c_nm ~ N(0, 1/(n+1)^2)
  * batched_512:   512 instances, n_max ~ U{8..64}, points log-uniform in [1e3, 2e5],
                   16 coefficient sets, c ~ N(0,1)
The seed of each workload is its index 0..4 in that list.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

TWO_PI = 2.0 * math.pi


def full_zernike_modes(n_max: int) -> tuple[np.ndarray, np.ndarray]:
    """All (n, m) with 0 <= n <= n_max, m = -n, -n+2, ..., n.  Count (n_max+1)(n_max+2)/2."""
    ns, ms = [], []
    for n in range(n_max + 1):
        for m in range(-n, n + 1, 2):
            ns.append(n)
            ms.append(m)
    return np.asarray(ns, dtype=np.int32), np.asarray(ms, dtype=np.int32)


def radial_modes(n_max: int) -> tuple[np.ndarray, np.ndarray]:
    """All (n, m) with 0 <= m <= n <= n_max and n - m even (radial-only set)."""
    ns, ms = [], []
    for n in range(n_max + 1):
        for m in range(n % 2, n + 1, 2):
            ns.append(n)
            ms.append(m)
    return np.asarray(ns, dtype=np.int32), np.asarray(ms, dtype=np.int32)


def uniform_points(n_points: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """r ~ U[0,1), theta ~ U[0, 2pi), float64, from numpy's PCG64 stream `seed`."""
    rng = np.random.default_rng(seed)
    r = rng.random(n_points)
    theta = rng.random(n_points) * TWO_PI
    return r, theta


def sqrt_uniform_points(n_points: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """r = sqrt(U[0,1)) (uniform over the disc area), theta ~ U[0, 2pi)."""
    rng = np.random.default_rng(seed)
    r = np.sqrt(rng.random(n_points))
    theta = rng.random(n_points) * TWO_PI
    return r, theta


def chebyshev_gauss_points(n_points: int) -> np.ndarray:
    """Chebyshev-Gauss nodes mapped to [0,1]: r_i = (1 + cos((2i-1) pi / (2P))) / 2, i = 1..P."""
    i = np.arange(1, n_points + 1, dtype=np.float64)
    return 0.5 * (1.0 + np.cos((2.0 * i - 1.0) * math.pi / (2.0 * n_points)))


def linspace_points(n_points: int) -> np.ndarray:
    """Linearly spaced rho on [0,1] (the accuracy/timing grid of the paper's Figs. 1 and 3)."""
    return np.linspace(0.0, 1.0, n_points)


def polar_grid(n_r: int = 250, n_theta: int = 200) -> tuple[np.ndarray, np.ndarray]:
    """Polar grid, r-major: r_i = sqrt((1 + t_i)/2) with t_i Gauss-Legendre on [-1,1],
    theta_j = 2 pi j / n_theta.  Returns flattened (r, theta) of length n_r * n_theta."""
    t, _ = np.polynomial.legendre.leggauss(n_r)
    r_nodes = np.sqrt(0.5 * (1.0 + t))
    th_nodes = TWO_PI * np.arange(n_theta, dtype=np.float64) / n_theta
    r = np.repeat(r_nodes, n_theta)
    theta = np.tile(th_nodes, n_r)
    return r, theta


def scaled_normal_coeffs(n: np.ndarray, n_sets: int, seed: int, scaled: bool = True) -> np.ndarray:
    """Coefficient sets C[j, s] ~ N(0, 1/(n_j+1)^2) (or N(0,1) if not scaled), row-major [J][S]."""
    rng = np.random.default_rng(seed + 1000)
    c = rng.standard_normal((len(n), n_sets))
    if scaled:
        c = c / (np.asarray(n, dtype=np.float64)[:, None] + 1.0)
    return np.ascontiguousarray(c)


@dataclass
class Instance:
    n_max: int
    n: np.ndarray
    m: np.ndarray
    r: np.ndarray
    theta: np.ndarray
    coeffs: np.ndarray  # [J][S]


def batched_instances(n_instances: int = 512, n_sets: int = 16, seed: int = 4,
                      n_max_range: tuple[int, int] = (8, 64),
                      points_range: tuple[float, float] = (1e3, 2e5),
                      point_scale: float = 1.0) -> list[Instance]:
    """Uneven batch: n_max ~ U{lo..hi} (full Z set), P_i log-uniform in points_range
    (times point_scale, at least 1), r ~ U[0,1), theta ~ U[0,2pi), c ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    lo, hi = n_max_range
    out = []
    lp0, lp1 = math.log(points_range[0]), math.log(points_range[1])
    for _ in range(n_instances):
        n_max = int(rng.integers(lo, hi + 1))
        p = max(1, int(round(math.exp(rng.uniform(lp0, lp1)) * point_scale)))
        n, m = full_zernike_modes(n_max)
        r = rng.random(p)
        theta = rng.random(p) * TWO_PI
        c = rng.standard_normal((len(n), n_sets))
        out.append(Instance(n_max, n, m, r, theta, np.ascontiguousarray(c)))
    return out


# Named workloads: (description, sizes).  Kept as data so the benchmark and tests agree.
WORKLOADS = {
    "basis_n20": dict(seed=0, n_max=20, n_points=1000, max_deriv=2),
    "radial_n100": dict(seed=1, n_max=100, n_points=100_000, max_deriv=3),
    "series_n24": dict(seed=2, n_max=24, n_r=250, n_theta=200, n_sets=256),
    "mixed_n32": dict(seed=3, n_max=32, n_points=1_000_000, n_sets=4096),
    "batched_512": dict(seed=4, n_instances=512, n_sets=16),
}
