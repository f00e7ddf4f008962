"""Seeded synthetic point clouds shared by the oracle, the tests and the benchmark.

This module holds only input generation: point sets and the names of the kernel
functions.  It contains none of the compression method's arithmetic, so both the
CUDA path and the CPU oracle can take their inputs from it without sharing code.

The shapes follow the paper's test geometries (Section 5): points in the unit
hypercube, a uniform grid, closed surfaces in 3D and the noisy line of Section 5.1.
The paper's own problems need solvers that are not part of this project (recursive
skeletonization, FMM3D, UMFPACK), so these clouds stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 220503406

# Kernel functions K(x, y) of the built-in black-box operator.  The ids match
# the HM_K_* constants of include/hm.h.
K_LOG = 1          # log|x - y|, zero where x == y
K_LAPLACE3D = 2    # 1 / (4 pi |x - y|), zero where x == y
K_INVR = 3         # 1 / |x - y|, zero where x == y
K_EXP = 4          # exp(-|x - y|)
K_NAMES = {K_LOG: "log", K_LAPLACE3D: "laplace3d", K_INVR: "invr", K_EXP: "exp"}


def line1d(n: int, seed: int) -> np.ndarray:
    """n points uniform on [0, 1), shape (n, 1)."""
    rng = np.random.default_rng(seed)
    return rng.random((n, 1))


def grid2d(n_side: int) -> np.ndarray:
    """Cell centres of an n_side x n_side grid in the unit square.

    Point i*n_side + j sits at ((i + 1/2)/n_side, (j + 1/2)/n_side).
    """
    i, j = np.meshgrid(np.arange(n_side), np.arange(n_side), indexing="ij")
    pts = np.stack([(i.ravel() + 0.5) / n_side, (j.ravel() + 0.5) / n_side], axis=1)
    return np.ascontiguousarray(pts, dtype=np.float64)


def torus(n: int, seed: int, R: float = 1.0, rho: float = 0.3) -> np.ndarray:
    """n points on a torus, uniform in the (u, v) parameter square [0, 2pi)^2.

    The density per unit area is proportional to 1 / (1 + rho cos v), so the
    cloud is non-uniform on the surface.
    """
    rng = np.random.default_rng(seed)
    uv = rng.random((n, 2)) * (2.0 * math.pi)
    u, v = uv[:, 0], uv[:, 1]
    ring = R + rho * np.cos(v)
    pts = np.stack([ring * np.cos(u), ring * np.sin(u), rho * np.sin(v)], axis=1)
    return np.ascontiguousarray(pts)


def curve2d(n: int, lobes: int = 5, amp: float = 0.3) -> np.ndarray:
    """n points equispaced in angle on the closed curve r(t) = 1 + amp cos(lobes t)
    (a smooth star-shaped contour standing in for the paper's 2D boundary)."""
    t = 2.0 * math.pi * np.arange(n) / n
    rad = 1.0 + amp * np.cos(lobes * t)
    return np.ascontiguousarray(np.stack([rad * np.cos(t), rad * np.sin(t)], axis=1))


def sphere(n: int, seed: int, jitter: float = 0.1) -> np.ndarray:
    """Fibonacci points on the unit sphere with seeded Gaussian jitter.

    z_i = 1 - (2i+1)/n, phi_i = i * pi (3 - sqrt 5); jitter of standard deviation
    jitter * sqrt(4 pi / n) is added and the points are projected back onto |x| = 1.
    """
    rng = np.random.default_rng(seed)
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    pts = np.stack([s * np.cos(phi), s * np.sin(phi), z], axis=1)
    pts = pts + rng.standard_normal(pts.shape) * (jitter * math.sqrt(4.0 * math.pi / n))
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    return np.ascontiguousarray(pts)


def noisy_line(n: int, d: int, noise: float, seed: int) -> np.ndarray:
    """Section 5.1: a uniform grid on a randomly oriented line through the
    centre of [0,1]^d, perturbed by Gaussian noise, clipped to the cube."""
    rng = np.random.default_rng(seed)
    direction = rng.standard_normal(d)
    direction /= np.linalg.norm(direction)
    t = (np.arange(n) + 0.5) / n - 0.5
    half = 0.5 / np.max(np.abs(direction))
    pts = 0.5 + np.outer(t * 2.0 * half, direction)
    pts += noise * rng.standard_normal(pts.shape)
    return np.ascontiguousarray(np.clip(pts, 0.0, 1.0))


def log_kernel_dense(x: np.ndarray) -> np.ndarray:
    """The stored dense matrix A_ij = log|x_i - x_j|, A_ii = 0 (1D workload).

    This builds the *input* matrix of the dense black-box operator; it is data,
    not a step of the compression method.
    """
    diff = x[:, None, :] - x[None, :, :]
    r = np.sqrt(np.sum(diff * diff, axis=2))
    with np.errstate(divide="ignore"):
        a = np.where(r > 0.0, np.log(np.where(r > 0.0, r, 1.0)), 0.0)
    return a


@dataclass
class Workload:
    """One compression problem: points, kernel, tree and truncation settings."""
    name: str
    points: np.ndarray
    kernel: int
    leaf_size: int
    r: int                 # columns per colour (k + oversampling)
    rank: int = 0          # > 0: fixed rank
    tol: float = 0.0       # > 0: relative truncation tolerance
    uniform_depth: int = 0 # > 0: force a uniform tree of this depth
    dense: np.ndarray | None = field(default=None, repr=False)  # stored matrix op
    seed: int = SEED_BASE
    oversample: int = 10   # p: tolerance mode keeps k <= r - p

    @property
    def n(self) -> int:
        return self.points.shape[0]

    @property
    def d(self) -> int:
        return self.points.shape[1]


def line1d_dense(n: int = 2048) -> Workload:
    """1D, N=2048 uniform on [0,1], A_ij = log|x_i-x_j| stored dense, depth-5
    binary tree, fixed rank 20 (r = 30)."""
    seed = SEED_BASE + 1
    x = line1d(n, seed)
    return Workload("line1d_dense", x, K_LOG, leaf_size=64, r=30, rank=20,
                    uniform_depth=5, dense=log_kernel_dense(x), seed=seed)


def grid2d_log(n_side: int = 256, rank: int = 40, tol: float = 0.0) -> Workload:
    """2D grid, log kernel on the fly, quadtree leaf 64, rank 40 (r = 50)."""
    seed = SEED_BASE + 2
    return Workload(f"grid2d_log_{n_side}", grid2d(n_side), K_LOG, leaf_size=64,
                    r=50, rank=rank, tol=tol, seed=seed)


def torus_laplace(n: int = 200_000, tol: float = 1e-6, r: int = 32) -> Workload:
    """3D torus surface (R=1, rho=0.3), K = 1/(4 pi |x-y|), adaptive octree
    leaf <= 64, relative tolerance 1e-6 with r = 32 columns per colour."""
    seed = SEED_BASE + 3
    return Workload(f"torus_laplace_{n}", torus(n, seed), K_LAPLACE3D, leaf_size=64,
                    r=r, tol=tol, seed=seed)


def sphere_invr(n: int = 1 << 20, tol: float = 1e-8, r: int = 40) -> Workload:
    """Jittered Fibonacci sphere, K = 1/|x-y|, octree leaf 64."""
    seed = SEED_BASE + 5
    return Workload(f"sphere_invr_{n}", sphere(n, seed), K_INVR, leaf_size=64,
                    r=r, tol=tol, seed=seed)


def serving_jobs(count: int, n_min: int = 4096, n_max: int = 65536, tol: float = 1e-6, seed: int = SEED_BASE + 4):
    """A stream of compression jobs: N log-uniform in [n_min, n_max], geometry and
    kernel alternating between a 2D closed curve with log|x - y|, and the torus
    with 1/|x - y| or exp(-|x - y|); tolerance tol, r = 32 (leaf 64 in 3D, 32 in 2D)."""
    rng = np.random.default_rng(seed)
    jobs = []
    for k in range(count):
        n = int(math.exp(rng.uniform(math.log(n_min), math.log(n_max))))
        kind = k % 3
        if kind == 0:
            jobs.append(Workload(f"curve_log_{n}", curve2d(n), K_LOG, leaf_size=32, r=32, tol=tol, seed=seed + k))
        elif kind == 1:
            jobs.append(Workload(f"torus_invr_{n}", torus(n, seed + k), K_INVR, leaf_size=64, r=32, tol=tol,
                                 seed=seed + k))
        else:
            jobs.append(Workload(f"torus_exp_{n}", torus(n, seed + k), K_EXP, leaf_size=64, r=32, tol=tol,
                                 seed=seed + k))
    return jobs
