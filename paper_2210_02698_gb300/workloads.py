"""Seeded synthetic inputs shared by the CUDA path, the tests and the oracle.

This module holds no arithmetic of the Hadamard-Babich method.  It only
describes the inputs of the volume integrator U = K I of Sec. 3.1 (Eq. m_v2v):

* the cell grid (cell-centred, unit square, N x N cells, natural order
  index = b*N + a with a the x index, x fastest);
* the media n(r) the paper's 2D experiments are shaped on (Sec. 5.1.1):
  homogeneous, constant velocity gradient c(z) = c0 + g z with n = 1/c, and a
  smooth Gaussian lens;
* the Chebyshev node order n_I of each workload;
* seeded right-hand sides (complex Gaussian cell sources, the paper's point
  source, Gaussian source, line segments and wavepackets, Sec. 5.1.1 and
  Eq. taper).

Random numbers come from numpy's PCG64 ``default_rng(seed)`` only.
Nothing here imports the CUDA binding or the oracle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


# ---------------------------------------------------------------- media ----
@dataclass(frozen=True)
class Medium:
    """Refractive index n(r) on the unit square.

    kind = "homogeneous": n = n0.
    kind = "gradient":    velocity c(z) = c0 + g*z, n = 1/c (z = 2nd coord).
    kind = "lens":        n = 1 + amp*exp(-|r - r_c|^2 / w^2).
    """

    kind: str
    n0: float = 1.0
    c0: float = 1.0
    g: float = 0.5
    amp: float = 0.1
    w: float = 0.3
    center: tuple = (0.5, 0.5)

    def n(self, x, z):
        x = np.asarray(x, dtype=np.float64)
        z = np.asarray(z, dtype=np.float64)
        if self.kind == "homogeneous":
            return np.full(np.broadcast(x, z).shape, self.n0)
        if self.kind == "gradient":
            return 1.0 / (self.c0 + self.g * z + 0.0 * x)
        if self.kind == "lens":
            r2 = (x - self.center[0]) ** 2 + (z - self.center[1]) ** 2
            return 1.0 + self.amp * np.exp(-r2 / self.w**2)
        raise ValueError(self.kind)

    @property
    def key(self) -> str:
        if self.kind == "homogeneous":
            return f"homog_n{self.n0:g}"
        if self.kind == "gradient":
            return f"grad_c{self.c0:g}_g{self.g:g}"
        return f"lens_a{self.amp:g}_w{self.w:g}"


HOMOGENEOUS = Medium("homogeneous", n0=1.0)
GRADIENT = Medium("gradient", c0=1.0, g=0.5)
LENS = Medium("lens", amp=0.1, w=0.3)


# ----------------------------------------------------------------- grid ----
@dataclass(frozen=True)
class Grid:
    """N x N cells of size h = 1/N on [0,1]^2, centroids ((a+1/2)h, (b+1/2)h)."""

    N: int

    @property
    def h(self) -> float:
        return 1.0 / self.N

    @property
    def Nv(self) -> int:
        return self.N * self.N

    def centroids(self):
        a = np.arange(self.N, dtype=np.float64)
        c = (a + 0.5) * self.h
        x = np.tile(c, self.N)          # natural order: index = b*N + a
        z = np.repeat(c, self.N)
        return x, z


# ------------------------------------------------------------ workloads ----
@dataclass(frozen=True)
class Workload:
    name: str
    N: int
    medium: Medium
    omega: float
    n_I: int
    nrhs: int
    eps: float = 1e-6
    chi: float = 20.0
    leaf: int = 64
    rhs_kind: str = "complex_normal"
    seed0: int = 2000
    note: str = ""

    @property
    def grid(self) -> Grid:
        return Grid(self.N)

    def n_cells(self):
        x, z = self.grid.centroids()
        return self.medium.n(x, z)


WORKLOADS = {
    # 8 wavelengths across, 8 cells per wavelength, homogeneous n = 1.
    "homog64": Workload("homog64", 64, HOMOGENEOUS, 2 * math.pi * 8, 16, 1,
                        rhs_kind="gaussian_center"),
    # Constant-gradient velocity c = 1 + 0.5 z, 32 wavelengths across at n = 1.
    "grad256": Workload("grad256", 256, GRADIENT, 2 * math.pi * 32, 16, 16),
    # Gaussian lens, 128 wavelengths across, 64 mixed sources.
    "lens1024": Workload("lens1024", 1024, LENS, 2 * math.pi * 128, 16, 64,
                         rhs_kind="mixed64"),
    # Source inversion workload of the gradient medium at 512^2.
    "grad512": Workload("grad512", 512, GRADIENT, 2 * math.pi * 64, 16, 1),
    # Large constant-gradient workload, 256 wavelengths across, 128 sources.
    # Intermediate constant-gradient size (scaling between 512^2 and 2048^2).
    "grad1024": Workload("grad1024", 1024, GRADIENT, 2 * math.pi * 128, 16, 32),
    "grad2048": Workload("grad2048", 2048, GRADIENT, 2 * math.pi * 256, 16, 128),
}


def small_workload(medium: Medium, N: int, wavelengths: float, nrhs: int,
                   n_I: int = 16, eps: float = 1e-6, leaf: int = 64,
                   chi: float = 20.0, seed0: int = 7000) -> Workload:
    """A reduced workload of the same shape: N cells per side, 8 cells per
    wavelength at the largest n when wavelengths = N/8."""
    return Workload(f"{medium.key}_N{N}", N, medium, 2 * math.pi * wavelengths,
                    n_I, nrhs, eps=eps, chi=chi, leaf=leaf, seed0=seed0)


# ---------------------------------------------------------------- sources ----
def complex_normal_sources(Nv: int, nrhs: int, seed0: int) -> np.ndarray:
    """Column k: i.i.d. per cell, Re and Im ~ N(0,1), from default_rng(seed0+k).
    Returned column-major as an (Nv, nrhs) complex128 array (Fortran order)."""
    s = np.empty((Nv, nrhs), dtype=np.complex128, order="F")
    for k in range(nrhs):
        rng = np.random.default_rng(seed0 + k)
        re = rng.standard_normal(Nv)
        im = rng.standard_normal(Nv)
        s[:, k] = re + 1j * im
    return s


def gaussian_center_source(grid: Grid, sigma: float = 0.05) -> np.ndarray:
    """s = exp(-|r - (0.5,0.5)|^2 / (2 sigma^2)), real, one column."""
    x, z = grid.centroids()
    r2 = (x - 0.5) ** 2 + (z - 0.5) ** 2
    return np.exp(-r2 / (2 * sigma**2)).astype(np.complex128).reshape(-1, 1)


def point_source(grid: Grid, a: int, b: int) -> np.ndarray:
    """Point source in cell (a, b): s = 1/h^2 there (Sec. 3.1)."""
    s = np.zeros((grid.Nv, 1), dtype=np.complex128)
    s[b * grid.N + a, 0] = 1.0 / grid.h**2
    return s


def taper(x, w1, w2):
    """Cosine taper of Eq. taper (input shaping only).  As printed, the
    middle branch w1 < x < w2 is empty for the paper's w1 = 0.3, w2 = 0.1;
    it is read as a ramp of width w2: 1 for x <= w1, 0.5(1+cos((x-w1)pi/w2))
    on (w1, w1+w2), 0 beyond (continuous at both ends)."""
    x = np.asarray(x, dtype=np.float64)
    t = np.where(x <= w1, 1.0, 0.0)
    mid = (x > w1) & (x < w1 + w2)
    t = np.where(mid, 0.5 * (1 + np.cos((x - w1) * np.pi / w2)), t)
    return t


def mixed_sources(grid: Grid, omega: float, nrhs: int, seed: int) -> np.ndarray:
    """Uneven batch: quarters of point sources, line segments, complex
    Gaussian bumps and Gaussian wavepackets (sigma 0.15, w1 0.3, w2 0.1,
    omega0 = 0.9 omega, random direction)."""
    rng = np.random.default_rng(seed)
    x, z = grid.centroids()
    N, h = grid.N, grid.h
    out = np.zeros((grid.Nv, nrhs), dtype=np.complex128, order="F")
    q = max(1, nrhs // 4)
    for k in range(nrhs):
        kind = min(3, k // q)
        if kind == 0:
            a, b = rng.integers(0, N, size=2)
            out[b * N + a, k] = 1.0 / h**2
        elif kind == 1:
            p0 = rng.uniform(0.1, 0.9, size=2)
            p1 = rng.uniform(0.1, 0.9, size=2)
            d = p1 - p0
            L2 = float(d @ d)
            t = np.clip(((x - p0[0]) * d[0] + (z - p0[1]) * d[1]) / L2, 0, 1)
            dist = np.hypot(x - (p0[0] + t * d[0]), z - (p0[1] + t * d[1]))
            out[:, k] = np.where(dist <= h / 2, 1.0 / h, 0.0)
        elif kind == 2:
            c = rng.uniform(0.2, 0.8, size=2)
            sig = rng.uniform(0.02, 0.1)
            amp = rng.standard_normal() + 1j * rng.standard_normal()
            out[:, k] = amp * np.exp(-((x - c[0]) ** 2 + (z - c[1]) ** 2) / (2 * sig**2))
        else:
            th = rng.uniform(0, 2 * np.pi)
            dvec = np.array([np.cos(th), np.sin(th)])
            r = np.hypot(x - 0.5, z - 0.5)
            out[:, k] = (np.exp(-r**2 / (2 * 0.15**2))
                         * np.exp(1j * 0.9 * omega * (x * dvec[0] + z * dvec[1]))
                         * taper(r, 0.3, 0.1))
    return out


def workload_sources(w: Workload) -> np.ndarray:
    g = w.grid
    if w.rhs_kind == "complex_normal":
        return complex_normal_sources(g.Nv, w.nrhs, w.seed0)
    if w.rhs_kind == "gaussian_center":
        return gaussian_center_source(g)
    if w.rhs_kind == "mixed64":
        return mixed_sources(g, w.omega, w.nrhs, w.seed0)
    raise ValueError(w.rhs_kind)


# ------------------------------------------------------------------ 3D ----
@dataclass(frozen=True)
class Medium3D:
    """Refractive index n(r) of the paper's 3D examples (Sec. 5.1.2).

    kind = "homogeneous": n = n0.
    kind = "gradient":    n = a / (c - y), i.e. velocity 1/n linear in y with
                          gradient -1/a (a = 1.25, c = 0.885 on [0, 0.52]^3).
    """

    kind: str
    n0: float = 1.0
    a: float = 1.25
    c: float = 0.885

    def n(self, x, y, z):
        x, y, z = (np.asarray(v, dtype=np.float64) for v in (x, y, z))
        shape = np.broadcast(x, y, z).shape
        if self.kind == "homogeneous":
            return np.full(shape, self.n0)
        if self.kind == "gradient":
            return np.broadcast_to(self.a / (self.c - y), shape).copy()
        raise ValueError(self.kind)


HOMOGENEOUS_3D = Medium3D("homogeneous")
GRADIENT_3D = Medium3D("gradient")


@dataclass(frozen=True)
class Grid3D:
    """N^3 cells of side h = L/N on [0, L]^3; natural index (c N + b) N + a
    with a the x index (fastest), b the y index, c the z index."""

    N: int
    L: float = 1.0

    @property
    def h(self) -> float:
        return self.L / self.N

    @property
    def Nv(self) -> int:
        return self.N ** 3

    def centroids(self):
        t = (np.arange(self.N) + 0.5) * self.h
        z, y, x = np.meshgrid(t, t, t, indexing="ij")
        return x.reshape(-1), y.reshape(-1), z.reshape(-1)


# ----------------------------------------------------------- inclusions ----
def circle_segments(center, radius: float, ns: int):
    """An inclusion's boundary for Sec. 3.2: the circle cut into ns equal
    chords, returned as (centres (ns, 2) at the chord midpoints, chord
    lengths (ns,))."""
    t = np.linspace(0.0, 2.0 * math.pi, ns + 1)
    p = np.stack([center[0] + radius * np.cos(t), center[1] + radius * np.sin(t)], axis=1)
    return 0.5 * (p[1:] + p[:-1]), np.hypot(p[1:, 0] - p[:-1, 0], p[1:, 1] - p[:-1, 1])


def sample_rows(Nv: int, m: int, seed: int) -> np.ndarray:
    """m distinct seeded row indices (natural order), sorted."""
    rng = np.random.default_rng(seed)
    m = min(m, Nv)
    return np.sort(rng.choice(Nv, size=m, replace=False)).astype(np.int64)


def random_id_matrices(count: int, m: int, n: int, rank: int, decay: float,
                       seed: int) -> np.ndarray:
    """Seeded complex test matrices for the interpolative decomposition:
    A = U diag(decay^k) W with Gaussian U (m x rank), W (rank x n), so the
    column geometry has a geometric singular-value profile.  Returns a
    (count, n, m) array: each matrix stored column-major (column j is
    A[b, j, :])."""
    rng = np.random.default_rng(seed)
    out = np.empty((count, n, m), dtype=np.complex128)
    for b in range(count):
        U = rng.standard_normal((m, rank)) + 1j * rng.standard_normal((m, rank))
        W = rng.standard_normal((rank, n)) + 1j * rng.standard_normal((rank, n))
        s = decay ** np.arange(rank)
        A = (U * s) @ W
        out[b] = A.T
    return out
