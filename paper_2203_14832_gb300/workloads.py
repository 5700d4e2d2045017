"""Seeded synthetic inputs shaped like the paper's workloads.

This module only draws point clouds and vectors and names the benchmark
workloads; it holds none of the method's arithmetic, so both the CUDA path and
the CPU oracle can take their inputs from it.

Workload recipes (all seeded with numpy's default_rng):

* ``log2d_4096``   : N = 4096 points i.i.d. uniform in [-1, 1]^2, K = log r,
                     K(x, x) = 0, leaf size 64, ACA tolerance 1e-8,
                     x ~ U[-1, 1]. Shape of the 2D uniform experiment (Sec. 5.1).
* ``invr3d_1m``    : N = 1,048,576 points i.i.d. uniform in [0, 1]^3, K = 1/r,
                     K(x, x) = 0, leaf size 64, ACA tolerance 1e-6, x ~ N(0, 1).
                     Shape of the 3D uniform experiment (Sec. 5.3).
* ``sphere_512k``  : N = 524,288 points uniform by area on the unit sphere
                     (normalised Gaussian triples), K = 1/(4 pi r) * (4 pi / N),
                     diagonal 1.0, ACA tolerance 1e-7: a boundary-integral
                     analogue of the integral-equation experiment (Sec. 5.5).
* ``gauss_mix_256k``: N = 262,144 points from 8 equal Gaussians (sigma 0.1,
                     centres uniform in [0, 1]^3), K = exp(-r^2 / (2 h^2)),
                     h = 0.2, ACA tolerance 1e-6, 64 right-hand sides: the
                     Gaussian kernel of the SVM experiment (Sec. 5.6).

* ``cheb2d_102k``  : the 320 x 320 tensor-product Chebyshev grid on [-1, 1]^2,
                     kernel (i) of the experiments with a = 1e-4, leaf size 64,
                     ACA tolerance 1e-9, x ~ N(0, 1) (Sec. 5, Experiment 2).
* ``cheb3d_262k``  : the 64^3 tensor-product Chebyshev grid on [-1, 1]^3,
                     kernel (ii) with a = 1e-4, ACA tolerance 1e-7 (Experiment 4).
* ``fredholm3d_262k``: the 64^3 cell-centred uniform grid on [-1, 1]^3 and the
                     Nystrom matrix of the second-kind equation of Experiment 5:
                     A = I + h^3 K with K = 1/r off the diagonal (h = 2/64),
                     ACA tolerance 1e-7; sigma ~ N(0, 1), f = A sigma.
* ``batch32``      : 32 independent problems, N_k log-uniform in
                     [16,384; 524,288], points uniform in [0, 1]^3, 16 with
                     K = 1/r and 16 with K = exp(-r^2 / (2 h^2)), h = 0.2,
                     ACA tolerance 1e-6, 8 right-hand sides x ~ N(0, 1)
                     (batched uneven problems; ``batch_workloads``).

The paper's experiments are all synthetic; no dataset stands behind them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

K_LOG, K_INV_R, K_GAUSS, K_MATERN, K_PAPER_I, K_PAPER_II, K_SEPARABLE, K_POLY2 = range(8)


def uniform_cube(n: int, d: int, seed: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=(n, d))


def sphere_surface(n: int, seed: int) -> np.ndarray:
    g = np.random.default_rng(seed).standard_normal((n, 3))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def gaussian_mixture(n: int, d: int, seed: int, k: int = 8, sigma: float = 0.1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(k, d))
    lab = np.repeat(np.arange(k), (n + k - 1) // k)[:n]
    return centres[lab] + sigma * rng.standard_normal((n, d))


def chebyshev_grid(m: int, d: int) -> np.ndarray:
    """Tensor-product Chebyshev points on [-1, 1]^d, m per dimension."""
    t = np.cos(np.pi * (np.arange(m) + 0.5) / m)
    grids = np.meshgrid(*([t] * d), indexing="ij")
    return np.stack([g.ravel() for g in grids], axis=1)


def uniform_grid(m: int, d: int) -> np.ndarray:
    """Cell-centred uniform grid on [-1, 1]^d, m points per dimension."""
    t = -1.0 + (np.arange(m) + 0.5) * (2.0 / m)
    grids = np.meshgrid(*([t] * d), indexing="ij")
    return np.stack([g.ravel() for g in grids], axis=1)


def grid_side(n: int, d: int) -> int:
    """m with m^d = n (grids are given by their point count)."""
    m = int(round(n ** (1.0 / d)))
    if m ** d != n:
        raise ValueError(f"{n} points is not a {d}-dimensional grid")
    return m


def vector_uniform(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    v = np.random.default_rng(seed).uniform(-1.0, 1.0, size=(nrhs, n))
    return v[0] if nrhs == 1 else v


def vector_normal(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    v = np.random.default_rng(seed).standard_normal((nrhs, n))
    return v[0] if nrhs == 1 else v


@dataclass
class Workload:
    name: str
    n: int
    d: int
    kernel: int
    kparam: tuple
    leaf_size: int
    aca_tol: float
    nrhs: int
    seed: int
    points: str            # generator name
    vector: str            # generator name
    note: str = ""

    def make_points(self, n: int | None = None) -> np.ndarray:
        n = self.n if n is None else n
        if self.points == "uniform_pm1":
            return uniform_cube(n, self.d, self.seed, -1.0, 1.0)
        if self.points == "uniform_01":
            return uniform_cube(n, self.d, self.seed, 0.0, 1.0)
        if self.points == "sphere":
            return sphere_surface(n, self.seed)
        if self.points == "gauss_mix":
            return gaussian_mixture(n, self.d, self.seed)
        if self.points == "chebyshev":
            return chebyshev_grid(grid_side(n, self.d), self.d)
        if self.points == "grid":
            return uniform_grid(grid_side(n, self.d), self.d)
        raise ValueError(self.points)

    def make_vector(self, n: int | None = None) -> np.ndarray:
        n = self.n if n is None else n
        if self.vector == "uniform":
            return vector_uniform(n, self.seed + 1, self.nrhs)
        return vector_normal(n, self.seed + 1, self.nrhs)

    def scaled(self, n: int) -> "Workload":
        """The same recipe at another size (the sphere weight follows N)."""
        kp = self.kparam
        if self.name.startswith("sphere"):
            kp = (sphere_weight(n),) + tuple(kp[1:])
        if self.name.startswith("fredholm"):
            kp = (nystrom_weight(n, self.d),) + tuple(kp[1:])
        return Workload(self.name + f"@{n}", n, self.d, self.kernel, kp, self.leaf_size, self.aca_tol,
                        self.nrhs, self.seed, self.points, self.vector, self.note)


def sphere_weight(n: int) -> float:
    """K = 1/(4 pi r) times the equal quadrature weight 4 pi / N, as one scale factor."""
    return (1.0 / (4.0 * math.pi)) * (4.0 * math.pi / n)


def nystrom_weight(n: int, d: int) -> float:
    """Quadrature weight h^d of the cell-centred grid on [-1, 1]^d with n points."""
    return (2.0 / grid_side(n, d)) ** d


WORKLOADS = {
    "log2d_4096": Workload("log2d_4096", 4096, 2, K_LOG, (1.0, 0.0, 0.0, 0.0), 64, 1e-8, 1, 1000,
                           "uniform_pm1", "uniform", "2D uniform, log r, dense-checked"),
    "invr3d_1m": Workload("invr3d_1m", 1 << 20, 3, K_INV_R, (1.0, 0.0, 0.0, 0.0), 64, 1e-6, 1, 2000,
                          "uniform_01", "normal", "3D uniform, 1/r"),
    "sphere_512k": Workload("sphere_512k", 1 << 19, 3, K_INV_R, (sphere_weight(1 << 19), 0.0, 1.0, 0.0), 64,
                            1e-7, 1, 3000, "sphere", "normal", "unit sphere, 1/(4 pi r) * 4 pi / N"),
    "cheb2d_102k": Workload("cheb2d_102k", 320 * 320, 2, K_PAPER_I, (1.0, 1e-4, 0.0, 0.0), 64, 1e-9, 1, 6000,
                            "chebyshev", "normal", "2D Chebyshev grid, kernel (i), a = 1e-4"),
    "cheb3d_262k": Workload("cheb3d_262k", 64 ** 3, 3, K_PAPER_II, (1.0, 1e-4, 0.0, 0.0), 64, 1e-7, 1, 7000,
                            "chebyshev", "normal", "3D Chebyshev grid, kernel (ii), a = 1e-4"),
    "fredholm3d_262k": Workload("fredholm3d_262k", 64 ** 3, 3, K_INV_R, ((2.0 / 64) ** 3, 0.0, 1.0, 0.0), 64, 1e-7, 1,
                                8000, "grid", "normal", "Nystrom matrix I + h^3/r on the uniform grid"),
    "gauss_mix_256k": Workload("gauss_mix_256k", 1 << 18, 3, K_GAUSS, (1.0, 0.2, 1.0, 0.0), 64, 1e-6, 64,
                               4000, "gauss_mix", "normal", "8-Gaussian mixture, Gaussian kernel h = 0.2"),
}


def batch_workloads(count: int = 32, seed: int = 5000, n_lo: int = 1 << 14, n_hi: int = 1 << 19,
                    nrhs: int = 8) -> list:
    """The ``batch32`` recipe: ``count`` problems with sizes log-uniform in [n_lo, n_hi],
    the first half with K = 1/r, the second half with the Gaussian kernel (h = 0.2)."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=count)).astype(np.int64)
    out = []
    for k, n in enumerate(sizes):
        gauss = k >= count // 2
        out.append(Workload(f"batch32[{k}]", int(n), 3, K_GAUSS if gauss else K_INV_R,
                            (1.0, 0.2, 1.0, 0.0) if gauss else (1.0, 0.0, 0.0, 0.0), 64, 1e-6, nrhs, seed + 10 * (k + 1),
                            "uniform_01", "normal", "batched uneven problems"))
    return out
