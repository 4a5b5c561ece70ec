"""Seeded synthetic inputs for the discrete-velocity collision operator.

This module is shared by the CPU oracle tests, the GPU parity tests and the
benchmark.  It only builds distribution functions ``f`` on the velocity grid
(and random cotangents); it contains none of the collision operator's
arithmetic.

Grid convention (used everywhere in this repository): ``N`` points per axis on
the periodic box ``[-L, L)^d``, step ``h = 2L/N``, node ``j`` at
``v_j = -L + j*h``; arrays are row-major with the last axis fastest.

Workloads (all synthetic, from the configurations the method is measured on):

* ``two_maxwellians_2d``  -- 2D, two isotropic Maxwellians at +-(2,0) with
  temperatures 1 and 1.5, unit discrete mass.
* ``bkw_2d``              -- the BKW profile of Section 4 with S = 0.6 (unit
  mass), and ``bkw_literal_2d`` the variant with the factor (1-K)|v|^2/K.
* ``trimaxwellian_3d``    -- 3D Gaussian with temperatures (0.5, 1, 2) per axis
  and drift (0.5, 0, 0).
* ``batch_2d``            -- many cells with mixed N, each a mixture of two
  Maxwellians with random drifts in [-1,1]^2 and temperatures in [0.5,2].
* ``batch_3d``            -- the same recipe in 3D for a fixed N.
* ``integer_field``       -- small non-negative integers (exact-arithmetic
  tests), ``gaussian``    -- N(0,1) cotangents / tangents.
"""
from __future__ import annotations

import math

import numpy as np


def grid_axis(N: int, L: float) -> np.ndarray:
    """Nodes v_j = -L + j h, h = 2L/N, j = 0..N-1 (float64)."""
    h = 2.0 * L / N
    return -L + h * np.arange(N, dtype=np.float64)


def grid(d: int, N: int, L: float) -> list[np.ndarray]:
    """Broadcastable coordinate arrays (v_0, ..., v_{d-1}) of shape N^d."""
    ax = grid_axis(N, L)
    return list(np.meshgrid(*([ax] * d), indexing="ij"))


def maxwellian(d: int, N: int, L: float, rho: float, u, T) -> np.ndarray:
    """rho * prod_a (2 pi T_a)^(-1/2) exp(-(v_a - u_a)^2 / (2 T_a)) on the grid.

    ``T`` may be a scalar (isotropic) or a length-d sequence (one temperature
    per axis).
    """
    u = np.broadcast_to(np.asarray(u, dtype=np.float64), (d,))
    T = np.broadcast_to(np.asarray(T, dtype=np.float64), (d,))
    vs = grid(d, N, L)
    out = np.full(vs[0].shape, float(rho))
    for a in range(d):
        out = out * np.exp(-((vs[a] - u[a]) ** 2) / (2.0 * T[a])) / math.sqrt(2.0 * math.pi * T[a])
    return out


def normalize_mass(f: np.ndarray, d: int, N: int, L: float, mass: float = 1.0) -> np.ndarray:
    h = 2.0 * L / N
    return f * (mass / (h ** d * f.sum()))


def two_maxwellians_2d(N: int = 16, L: float = 8.0) -> np.ndarray:
    """Two isotropic Maxwellians: mass 0.5 at +(2,0) with T=1, mass 0.5 at
    -(2,0) with T=1.5, renormalised to unit discrete mass."""
    f = maxwellian(2, N, L, 0.5, (2.0, 0.0), 1.0) + maxwellian(2, N, L, 0.5, (-2.0, 0.0), 1.5)
    return normalize_mass(f, 2, N, L)


def bkw_2d(N: int = 64, L: float = 8.0, S: float = 0.6) -> np.ndarray:
    """BKW profile exp(-|v|^2/2S) / (2 pi S^2) * (2S - 1 + (1-S)|v|^2/(2S))
    (Section 4), sampled on the grid; unit mass in the continuum."""
    v0, v1 = grid(2, N, L)
    r2 = v0 ** 2 + v1 ** 2
    return np.exp(-r2 / (2.0 * S)) / (2.0 * math.pi * S ** 2) * (2.0 * S - 1.0 + (1.0 - S) * r2 / (2.0 * S))


def bkw_literal_2d(N: int = 64, L: float = 8.0, K: float = 0.6) -> np.ndarray:
    """exp(-|v|^2/2K)(2K - 1 + (1-K)|v|^2/K)/(2 pi K^2), the variant with the
    factor (1-K)|v|^2/K (mass 1/K in the continuum)."""
    v0, v1 = grid(2, N, L)
    r2 = v0 ** 2 + v1 ** 2
    return np.exp(-r2 / (2.0 * K)) * (2.0 * K - 1.0 + (1.0 - K) * r2 / K) / (2.0 * math.pi * K ** 2)


def trimaxwellian_3d(N: int = 32, L: float = 6.0) -> np.ndarray:
    """Gaussian with temperatures (0.5, 1, 2) per axis and drift (0.5, 0, 0),
    unit discrete mass."""
    f = maxwellian(3, N, L, 1.0, (0.5, 0.0, 0.0), (0.5, 1.0, 2.0))
    return normalize_mass(f, 3, N, L)


def mixture(d: int, N: int, L: float, rng: np.random.Generator) -> np.ndarray:
    """Two isotropic Maxwellians of mass 0.5 each, drifts U[-1,1]^d,
    temperatures U[0.5,2], renormalised to unit discrete mass."""
    f = np.zeros((N,) * d)
    for _ in range(2):
        u = rng.uniform(-1.0, 1.0, size=d)
        T = rng.uniform(0.5, 2.0)
        f = f + maxwellian(d, N, L, 0.5, u, T)
    return normalize_mass(f, d, N, L)


class Batch:
    """A ragged batch of cells stored back to back.

    ``Ns[c]`` is the grid size of cell ``c``; cell ``c`` occupies
    ``f[offsets[c] : offsets[c] + Ns[c]**d]`` (row-major, last axis fastest).
    """

    def __init__(self, d: int, L: float, Ns: np.ndarray, f: np.ndarray):
        self.d = d
        self.L = L
        self.Ns = np.asarray(Ns, dtype=np.int64)
        sizes = self.Ns ** d
        self.offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        self.f = f
        self.total = int(sizes.sum())

    @property
    def n_cells(self) -> int:
        return int(self.Ns.shape[0])

    def cell(self, c: int, arr: np.ndarray | None = None) -> np.ndarray:
        a = self.f if arr is None else arr
        n = int(self.Ns[c])
        o = int(self.offsets[c])
        return a[o:o + n ** self.d].reshape((n,) * self.d)


def batch_2d(n_cells: int = 4096, Ns=(16, 32, 48, 64), L: float = 8.0, seed: int = 0) -> Batch:
    """Cells with N drawn uniformly from ``Ns`` (seeded), each a two-Maxwellian
    mixture with random drifts in [-1,1]^2 and temperatures in [0.5,2]."""
    rng = np.random.default_rng(seed)
    Nc = rng.choice(np.asarray(Ns, dtype=np.int64), size=n_cells)
    parts = [mixture(2, int(n), L, rng).ravel() for n in Nc]
    return Batch(2, L, Nc, np.concatenate(parts))


def batch_2d_relaxing(n_cells: int = 4096, Ns=(16, 32, 48, 64), L: float = 8.0, seed: int = 3) -> Batch:
    """Cells at different distances from equilibrium, as in a space-
    inhomogeneous solve where most of the domain has relaxed: each cell is
    (1 - w) M(u1, T1) + w M(u2, T2) with drifts U[-1,1]^2, temperatures
    U[0.5,2] and a second-component weight w = 0.5 U^3 (U uniform on
    [0, 1]: half the cells have w < 0.0625), unit discrete mass."""
    rng = np.random.default_rng(seed)
    Nc = rng.choice(np.asarray(Ns, dtype=np.int64), size=n_cells)
    parts = []
    for n in Nc:
        n = int(n)
        w = 0.5 * rng.uniform() ** 3
        f = np.zeros((n, n))
        for wt in (1.0 - w, w):
            u = rng.uniform(-1.0, 1.0, size=2)
            T = rng.uniform(0.5, 2.0)
            f = f + maxwellian(2, n, L, wt, u, T)
        parts.append(normalize_mass(f, 2, n, L).ravel())
    return Batch(2, L, Nc, np.concatenate(parts))


def batch_3d(n_cells: int = 256, N: int = 32, L: float = 6.0, seed: int = 1) -> Batch:
    """Cells of a fixed N, each a two-Maxwellian mixture in 3D (drifts
    U[-1,1]^3, temperatures U[0.5,2])."""
    rng = np.random.default_rng(seed)
    parts = [mixture(3, N, L, rng).ravel() for _ in range(n_cells)]
    return Batch(3, L, np.full(n_cells, N, dtype=np.int64), np.concatenate(parts))


def integer_field(d: int, N: int, maxval: int = 3, seed: int = 0) -> np.ndarray:
    """Uniform random integers in [0, maxval] as float64 (exact-arithmetic
    tests)."""
    rng = np.random.default_rng(seed)
    return rng.integers(0, maxval + 1, size=(N,) * d).astype(np.float64)


def compact_support(d: int, N: int, S: int, seed: int = 0) -> np.ndarray:
    """Random positive values on lattice offsets |i|_inf <= S around the box
    centre (i = j - N//2), zero elsewhere."""
    rng = np.random.default_rng(seed)
    f = np.zeros((N,) * d)
    sl = tuple(slice(N // 2 - S, N // 2 + S + 1) for _ in range(d))
    f[sl] = rng.uniform(0.1, 1.0, size=f[sl].shape)
    return f


def gaussian(shape, seed: int = 2) -> np.ndarray:
    """N(0,1) samples (cotangents or tangents)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=shape)
