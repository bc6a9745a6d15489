"""Seeded synthetic inputs shared by the CUDA path, its tests and the benchmark.

This module holds no arithmetic of the solver itself: it only builds the
frozen density fields, the Dirichlet masks, the tip-edge loads and random test
vectors that both the CPU oracle and the CUDA library consume.  It imports
nothing from the rest of the package.

Layout conventions (shared by every consumer):

* element field ``rho[ez, ey, ex]`` (x fastest), float32;
* node ``n = i + (nx+1) * (j + (ny+1) * k)``; DOF ``3*n + c`` (c = x, y, z);
* per-DOF fixed flags ``uint8[3*n_nodes]`` (1 = fixed, 0 = free).

The cantilever set-up follows the paper's frozen-coefficient state equation
(Sec. "Problem Setup", Eq. state_eq): the whole x = 0 face is clamped, which
reproduces the free-DOF counts of Table e7 (e.g. 100x50x25 -> 397,800).  The
paper does not state the load; the reading used here puts a unit total load in
-z on the nodes of the edge x = nx, z = 0, split equally over its ny+1 nodes.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Config",
    "CONFIGS",
    "n_nodes",
    "clamp_xmin_mask",
    "tip_edge_load",
    "rotated_tip_edge_load",
    "uniform_density",
    "filtered_random_density",
    "random_free_vector",
    "he_normal_params",
]


@dataclasses.dataclass(frozen=True)
class Config:
    """One synthetic cantilever workload (grid, density recipe, solver knobs)."""

    name: str
    nx: int
    ny: int
    nz: int
    density: str  # "uniform" | "filtered"
    rho0: float = 0.5
    seed: int = 0
    p: float = 3.0
    levels: int = 0  # 0 = automatic depth
    smoother: str = "jacobi"  # "jacobi" | "chebyshev"
    degree: int = 2
    omega: float = 0.6
    tol: float = 1e-6
    maxit: int = 200

    @property
    def n_elem(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def n_nodes(self) -> int:
        return n_nodes(self.nx, self.ny, self.nz)

    def rho(self) -> np.ndarray:
        if self.density == "uniform":
            return uniform_density(self.nx, self.ny, self.nz, self.rho0)
        return filtered_random_density(self.nx, self.ny, self.nz, self.seed)

    def fixed(self) -> np.ndarray:
        return clamp_xmin_mask(self.nx, self.ny, self.nz)

    def load(self) -> np.ndarray:
        return tip_edge_load(self.nx, self.ny, self.nz)


# The three single-GPU configurations.  C0: small 3-level Jacobi case; C1: the
# 40^3 heterogeneous field (p = 3 by default, p in {1, 2, 3} in the tests; two
# Jacobi sweeps with the paper's damping cap 0.5, since 0.6 times the fine-level
# lambda_max exceeds 2 at p = 3); C2: the 100^3 uniform-modulus 5-level
# degree-3 Chebyshev solve (the throughput case).
CONFIGS = {
    "c0": Config("c0", 16, 8, 8, "uniform", rho0=0.5, p=3.0, levels=3,
                 smoother="jacobi", degree=2, omega=0.6),
    "c1": Config("c1", 40, 40, 40, "filtered", seed=1, p=3.0, levels=4,
                 smoother="jacobi", degree=2, omega=0.5),
    "c2": Config("c2", 100, 100, 100, "uniform", rho0=0.5, p=3.0, levels=5,
                 smoother="chebyshev", degree=3),
}


def n_nodes(nx: int, ny: int, nz: int) -> int:
    return (nx + 1) * (ny + 1) * (nz + 1)


def clamp_xmin_mask(nx: int, ny: int, nz: int) -> np.ndarray:
    """uint8[3*n_nodes]: every DOF of every node on the face i = 0 is fixed."""
    fixed = np.zeros((nz + 1, ny + 1, nx + 1, 3), dtype=np.uint8)
    fixed[:, :, 0, :] = 1
    return fixed.reshape(-1)


def tip_edge_load(nx: int, ny: int, nz: int, total: float = 1.0) -> np.ndarray:
    """float64[3*n_nodes]: -z load spread equally over the nodes (nx, j, 0)."""
    f = np.zeros((nz + 1, ny + 1, nx + 1, 3), dtype=np.float64)
    f[0, :, nx, 2] = -total / (ny + 1)
    return f.reshape(-1)


def rotated_tip_edge_load(nx: int, ny: int, nz: int, k: int, nrhs: int = 16) -> np.ndarray:
    """Tip-edge load rotated in the y-z plane by theta_k = 2*pi*k/nrhs."""
    th = 2.0 * math.pi * k / nrhs
    f = np.zeros((nz + 1, ny + 1, nx + 1, 3), dtype=np.float64)
    f[0, :, nx, 1] = math.sin(th) / (ny + 1)
    f[0, :, nx, 2] = -math.cos(th) / (ny + 1)
    return f.reshape(-1)


def uniform_density(nx: int, ny: int, nz: int, value: float = 0.5) -> np.ndarray:
    return np.full((nz, ny, nx), value, dtype=np.float32)


def filtered_random_density(nx: int, ny: int, nz: int, seed: int,
                            sigma: float = 1.5, lo: float = 1e-3) -> np.ndarray:
    """Seeded i.i.d. U[0,1] per element, Gaussian-filtered (sigma in elements,
    radius ceil(4 sigma), mirror boundary), min-max rescaled to [0,1], clipped
    to [lo, 1], stored as float32."""
    from scipy.ndimage import gaussian_filter

    rng = np.random.default_rng(seed)
    raw = rng.uniform(0.0, 1.0, size=(nz, ny, nx))
    sm = gaussian_filter(raw, sigma=sigma, mode="reflect", truncate=4.0)
    span = sm.max() - sm.min()
    sm = (sm - sm.min()) / (span if span > 0 else 1.0)
    return np.clip(sm, lo, 1.0).astype(np.float32)


def checkerboard_density(nx: int, ny: int, nz: int, solid: float = 1.0, void: float = 1e-3) -> np.ndarray:
    """Deterministic stress state: elements alternate between solid and void in
    all three directions ((i + j + k) even -> solid), FP32 [nz][ny][nx]."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.where((i + j + k) % 2 == 0, solid, void).astype(np.float32)


def layered_band_density(nx: int, ny: int, nz: int, solid: float = 1.0, void: float = 1e-3) -> np.ndarray:
    """Deterministic stress state: the lower half of the beam in z is solid and
    the upper half void (a half-solid / half-void band), FP32 [nz][ny][nx]."""
    rho = np.full((nz, ny, nx), void, dtype=np.float32)
    rho[: nz // 2] = solid
    return rho


def random_free_vector(fixed: np.ndarray, seed: int, dtype=np.float32) -> np.ndarray:
    """Seeded U[-1,1] on free DOFs, exactly 0 on fixed DOFs."""
    rng = np.random.default_rng(seed)
    v = rng.uniform(-1.0, 1.0, size=fixed.shape[0]).astype(dtype)
    v[fixed.astype(bool)] = 0
    return v


def he_normal_params(shapes, seed: int) -> np.ndarray:
    """Seeded initial parameters of a stack of 3-D convolution layers, flat
    float32: for each (cout, taps, cin) in ``shapes`` the weights
    [cout][taps][cin] drawn N(0, 2 / (taps * cin)), followed by cout zero
    biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for cout, taps, cin in shapes:
        std = math.sqrt(2.0 / (taps * cin))
        parts.append(rng.normal(0.0, std, size=cout * taps * cin))
        parts.append(np.zeros(cout))
    return np.concatenate(parts).astype(np.float32)
