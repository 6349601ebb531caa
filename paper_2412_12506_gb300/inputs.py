"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module only draws random numbers and describes workload shapes.  It holds
none of the method's arithmetic (no basis, no operator, no smoother), so both
sides can take their inputs from it without sharing any numerical code.

Workloads (shapes of the paper's experiments, Sec. 2.4.1, 2.4.3 and 3.4):
  * periodic Poisson on the unit square / cube, mu == 1 (Sec. 2.4.1);
  * two-phase elliptic interface problem: mu = mu_in inside the paper's
    inclusion (1/4, 3/4)^d (Sec. 2.4.3) or inside a seeded circle, mu_out
    outside, decided per element at the element centroid;
  * steady two-phase Stokes (Sec. 3.4.3): viscosity contrast on the same
    inclusion, body force a seeded smooth field of a few Fourier modes.

Right-hand sides: the paper draws the coefficients of b independently at
random (Sec. 2.4, footnote to Eq. (eta)); here they are N(0,1) per coefficient,
laid out [element][mode][rhs] with elements lexicographic (x fastest).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass(frozen=True)
class Workload:
    name: str
    dim: int
    n: int              # elements per axis (uniform periodic Cartesian mesh)
    p: int              # 1D polynomial degree
    smoother: str       # "jacobi" | "sai"
    nu1: int
    nu2: int
    mu: str = "one"     # "one" | "circle"
    mu_in: float = 1e4
    mu_seed: int = 0
    nrhs: int = 1
    tol: float = 1e-10
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.n ** self.dim

    @property
    def b(self) -> int:
        return (self.p + 1) ** self.dim


# 2D periodic Poisson, 16x16, p=2, damped block Jacobi 2/2, CG to 1e-10.
POISSON2D_16_P2 = Workload("poisson2d_n16_p2_jacobi", 2, 16, 2, "jacobi", 2, 2)
# 3D periodic Poisson, 48^3, p=3 (7.08M dofs), SAI1 3/3, CG to 1e-10.
POISSON3D_48_P3 = Workload("poisson3d_n48_p3_sai1", 3, 48, 3, "sai", 3, 3)
# 2D interface problem, 256^2, p=3, balanced SAI1 3/3, mu 1 / 1e4 circle, 64 RHS.
INTERFACE2D_256_P3 = Workload("interface2d_n256_p3_sai1_circle1e4", 2, 256, 3, "sai", 3, 3,
                              mu="circle", mu_in=1e4, mu_seed=0, nrhs=64)

# 2D steady two-phase Stokes, 128^2, p=2 (27 dofs/element: u, v, p), viscosity 1 / 1e3
# on the square inclusion, 8-mode Fourier body force, Stokes-balanced SAI1, GMRES.
STOKES2D_128_P2 = Workload("stokes2d_n128_p2_sai1_square1e3", 2, 128, 2, "sai", 3, 3, mu="square", mu_in=1e3,
                           tol=1e-10, extra={"gamma": 1, "force_modes": 8, "force_seed": 0})

WORKLOADS = {w.name: w for w in (POISSON2D_16_P2, POISSON3D_48_P3, INTERFACE2D_256_P3, STOKES2D_128_P2)}


def circle_mu(dim: int, n: int, seed: int, mu_in: float = 1e4, mu_out: float = 1.0) -> np.ndarray:
    """Per-element coefficient: mu_in inside a seeded circle/sphere, mu_out outside.

    Centre ~ U[0.3, 0.7]^dim, radius ~ U[0.15, 0.3], both from default_rng(seed).
    An element is inside when its centroid lies strictly inside the circle.
    Returns float64 array of length n**dim, element index ix + n*iy (+ n*n*iz).
    """
    rng = np.random.default_rng(seed)
    centre = rng.uniform(0.3, 0.7, size=dim)
    radius = rng.uniform(0.15, 0.3)
    c1 = (np.arange(n) + 0.5) / n
    grids = np.meshgrid(*([c1] * dim), indexing="ij")  # grids[a][i_0, ..., i_{d-1}]
    dist2 = sum((grids[a] - centre[a]) ** 2 for a in range(dim))
    inside = dist2 < radius ** 2
    # element index with x fastest: transpose the (ix, iy, iz) grid to (iz, iy, ix)
    inside = np.transpose(inside, tuple(range(dim - 1, -1, -1))).reshape(-1)
    return np.where(inside, mu_in, mu_out).astype(np.float64)


def square_mu(dim: int, n: int, mu_in: float = 1e4, mu_out: float = 1.0) -> np.ndarray:
    """Per-element coefficient for the paper's inclusion Omega_0 = (1/4, 3/4)^d
    (Sec. 2.4.3): mu_in for elements whose centroid lies in Omega_0, else mu_out."""
    c1 = (np.arange(n) + 0.5) / n
    grids = np.meshgrid(*([c1] * dim), indexing="ij")
    inside = np.ones(grids[0].shape, dtype=bool)
    for a in range(dim):
        inside &= (grids[a] > 0.25) & (grids[a] < 0.75)
    inside = np.transpose(inside, tuple(range(dim - 1, -1, -1))).reshape(-1)
    return np.where(inside, mu_in, mu_out).astype(np.float64)


def element_mu(w: Workload) -> np.ndarray:
    if w.mu == "one":
        return np.ones(w.N, dtype=np.float64)
    if w.mu == "circle":
        return circle_mu(w.dim, w.n, w.mu_seed, w.mu_in)
    if w.mu == "square":
        return square_mu(w.dim, w.n, w.mu_in)
    raise ValueError(w.mu)


def random_rhs(N: int, b: int, nrhs: int = 1, seed: int = 0) -> np.ndarray:
    """N(0,1) coefficients, shape (N*b,) for nrhs == 1 else (N*b, nrhs)."""
    rng = np.random.default_rng(seed)
    if nrhs == 1:
        return rng.standard_normal(N * b)
    return rng.standard_normal((N * b, nrhs))


def random_vector(size: int, seed: int) -> np.ndarray:
    """Generic N(0,1) test vector (operator-apply parity inputs)."""
    return np.random.default_rng(seed).standard_normal(size)


def fourier_force_rhs(dim: int, n: int, p: int, seed: int, nmodes: int = 8) -> np.ndarray:
    """Stokes right-hand side with a smooth seeded body force.

    Each velocity component f_a(x) = sum_{m < nmodes} c_m sin(2 pi k_m . x + phi_m)
    with integer wave vectors k_m, |k_m|_inf in 1..3 (so f_a has zero mean on
    the periodic cell), c_m ~ N(0, 1), phi_m ~ U[0, 2 pi).  The value at each
    element centroid is written into the element's constant mode (mode 0) of
    that velocity field; all other modes and the pressure field are zero.
    Layout: N blocks of (dim + 1) * (p + 1)^dim values, fields u_1..u_dim, p.
    """
    rng = np.random.default_rng(seed)
    bs = (p + 1) ** dim
    nf = dim + 1
    N = n ** dim
    c1 = (np.arange(n) + 0.5) / n
    grids = np.meshgrid(*([c1] * dim), indexing="ij")
    grids = [np.transpose(g, tuple(range(dim - 1, -1, -1))).reshape(-1) for g in grids]
    out = np.zeros((N, nf, bs))
    for a in range(dim):
        field_a = np.zeros(N)
        for _ in range(nmodes):
            k = rng.integers(-3, 4, size=dim)
            while not np.any(k):
                k = rng.integers(-3, 4, size=dim)
            amp = rng.standard_normal()
            ph = rng.uniform(0.0, 2.0 * np.pi)
            field_a += amp * np.sin(2.0 * np.pi * sum(k[t] * grids[t] for t in range(dim)) + ph)
        out[:, a, 0] = field_a
    return out.reshape(-1)


def zero_mean_rhs(N: int, b: int, seed: int, nfields: int = 1) -> np.ndarray:
    """N(0,1) coefficients (N blocks of nfields * b values) with the constant
    mode of each field shifted to zero mean over the elements: the "N(0,1)
    values projected to zero mean" of the workloads, consistent with the
    periodic operators' constant kernel."""
    v = np.random.default_rng(seed).standard_normal((N, nfields, b))
    v[:, :, 0] -= v[:, :, 0].mean(axis=0)
    return v.reshape(-1)


def serving_requests(count: int, seed: int):
    """Request mix of the serving workload: 2D problems (meshes 16^2..256^2,
    p = 1..4) and 3D problems (8^3..32^3, p = 1..3), each Poisson (contrast 1)
    or an interface problem with contrast 1e2 or 1e4 on the inclusion
    (1/4, 3/4)^d, drawn uniformly per field (3 in 4 requests are 2D).
    Returns a list of dicts with dim, n, p, contrast and a right-hand-side
    seed."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        if rng.random() < 0.75:
            dim, n, p = 2, int(rng.choice([16, 32, 64, 128, 256])), int(rng.integers(1, 5))
        else:
            dim, n, p = 3, int(rng.choice([8, 16, 32])), int(rng.integers(1, 4))
        contrast = float(rng.choice([1.0, 1e2, 1e4]))
        out.append({"dim": dim, "n": n, "p": p, "contrast": contrast, "rhs_seed": int(rng.integers(1 << 31))})
    return out
