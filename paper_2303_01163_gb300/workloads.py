"""Seeded synthetic inputs for the advection-diffusion problems ASDSM solves.

This module only draws problem data (coefficients, source term s, boundary
data g) on the uniform grid; it holds none of the method's arithmetic.  Both
the CPU oracle and the CUDA path consume what it returns, so it imports
neither of them.

Grid convention (shared by every caller): a d-dimensional array with ``N``
points per axis including the boundary, point ``x_i = i / (N - 1)``, axis
order (z, y, x) so that x is the fastest-varying index (the vector ordering
of Section 2.2 of the paper).

Workload families (the paper's experiments use manufactured solutions only,
Section 4; there is no dataset):

* ``manufactured_sine_2d`` - u = sin(pi x) sin(pi y) with s derived from
  eq. (1.1) and g = u on the boundary (the smooth setting of Example 1, with
  the sine product instead of sin(pi x + pi y)).
* ``random_fourier_2d`` - alpha_i log-uniform in [1e-2, 1], beta_i uniform
  in [-10, 10], s a sum of 16 random sine modes, zero Dirichlet data.
* ``manufactured_sine_3d`` / ``random_fourier_3d`` - the 3D analogues.
* ``polynomial_2d`` - u = p(x) q(y) with quadratic p, q: central differences
  are exact for it on every uniform mesh, which pins the whole initial guess.
* ``manufactured_variable_2d`` - the second setting of Example 1: coefficients
  that vary in space (alpha_1 = 1 + x^2, alpha_2 = 2 + x y, beta_1 = 2 - x,
  beta_2 = 1 + y, given as functions of (x, y)) and u = sin(4 pi x + 4 pi y);
  ``manufactured_variable_3d`` - the same for the second setting of Example 4.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    """One Dirichlet problem for eq. (1.1) sampled on a uniform grid."""

    d: int
    N: int
    alpha: tuple
    beta: tuple
    s: np.ndarray          # source term on the full grid (boundary entries unused)
    g: np.ndarray          # full grid: boundary entries carry the Dirichlet data, interior 0
    u_exact: np.ndarray | None = None   # continuous solution sampled on the grid, if known
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def unknowns(self) -> int:
        return (self.N - 2) ** self.d


def _axes(N: int, d: int):
    x = np.linspace(0.0, 1.0, N)
    return np.meshgrid(*([x] * d), indexing="ij")  # returns (z, y, x) order for d=3 when reversed


def _grid2(N):
    x = np.linspace(0.0, 1.0, N)
    Y, X = np.meshgrid(x, x, indexing="ij")   # [y, x]
    return X, Y


def _grid3(N):
    x = np.linspace(0.0, 1.0, N)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")   # [z, y, x]
    return X, Y, Z


def _boundary_only(u: np.ndarray) -> np.ndarray:
    g = np.zeros_like(u)
    sl = [slice(1, -1)] * u.ndim
    g[...] = u
    g[tuple(sl)] = 0.0
    return g


def manufactured_sine_2d(N: int, alpha=(1.0, 1.0), beta=(1.0, 1.0)) -> Problem:
    X, Y = _grid2(N)
    ax, ay = alpha
    bx, by = beta
    pi = np.pi
    u = np.sin(pi * X) * np.sin(pi * Y)
    s = ((ax + ay) * pi**2 * np.sin(pi * X) * np.sin(pi * Y)
         + bx * pi * np.cos(pi * X) * np.sin(pi * Y)
         + by * pi * np.sin(pi * X) * np.cos(pi * Y))
    return Problem(2, N, tuple(alpha), tuple(beta), s, _boundary_only(u), u,
                   name=f"sine2d_N{N}")


def manufactured_shifted_sine_2d(N: int, alpha=(1.0, 1.0), beta=(1.0, 1.0), k: float = 1.0) -> Problem:
    """u = sin(k pi x + k pi y): Example 1 of Section 4 (k=1 smooth, k=4 oscillatory)."""
    X, Y = _grid2(N)
    ax, ay = alpha
    bx, by = beta
    w = k * np.pi
    u = np.sin(w * X + w * Y)
    s = (ax + ay) * w**2 * u + (bx + by) * w * np.cos(w * X + w * Y)
    return Problem(2, N, tuple(alpha), tuple(beta), s, _boundary_only(u), u,
                   name=f"shiftsine2d_k{k}_N{N}")


def variable_coefficients_example1():
    """alpha_i(x, y), beta_i(x, y) of the second setting of Example 1 (Section 4)."""
    alpha = (lambda x, y: 1.0 + x * x, lambda x, y: 2.0 + x * y)
    beta = (lambda x, y: 2.0 - x, lambda x, y: 1.0 + y)
    return alpha, beta


def manufactured_variable_2d(N: int, k: float = 4.0) -> Problem:
    """u = sin(k pi x + k pi y) with the coefficients of the second setting of
    Example 1; s = -alpha_1 u_xx - alpha_2 u_yy + beta_1 u_x + beta_2 u_y."""
    alpha, beta = variable_coefficients_example1()
    X, Y = _grid2(N)
    w = k * np.pi
    u = np.sin(w * X + w * Y)
    du = w * np.cos(w * X + w * Y)          # u_x = u_y
    d2u = -w * w * u                        # u_xx = u_yy
    s = (-alpha[0](X, Y) * d2u - alpha[1](X, Y) * d2u + beta[0](X, Y) * du + beta[1](X, Y) * du)
    return Problem(2, N, alpha, beta, s, _boundary_only(u), u, name=f"variable2d_k{k}_N{N}")


def variable_coefficients_example4():
    """alpha_i(x, y, z), beta_i(x, y, z) of the second setting of Example 4 (Section 4)."""
    alpha = (lambda x, y, z: 1.0 + x * x, lambda x, y, z: 2.0 + x * y, lambda x, y, z: 3.0 - x * y * z)
    beta = (lambda x, y, z: 2.0 - x, lambda x, y, z: 1.0 + y, lambda x, y, z: 2.0 - x + y * z)
    return alpha, beta


def manufactured_variable_3d(N: int, k: float = 4.0) -> Problem:
    """u = sin(k pi (x + y + z)) with the coefficients of the second setting of
    Example 4; s = sum_i (-alpha_i u_{x_i x_i} + beta_i u_{x_i}).  Grids [z, y, x]."""
    alpha, beta = variable_coefficients_example4()
    X, Y, Z = _grid3(N)
    w = k * np.pi
    u = np.sin(w * (X + Y + Z))
    du = w * np.cos(w * (X + Y + Z))        # every first derivative
    d2u = -w * w * u                        # every second derivative
    s = sum(-alpha[a](X, Y, Z) * d2u + beta[a](X, Y, Z) * du for a in range(3))
    return Problem(3, N, alpha, beta, s, _boundary_only(u), u, name=f"variable3d_k{k}_N{N}")


def polynomial_2d(N: int, alpha=(1.0, 1.0), beta=(1.0, 1.0),
                  p=(0.3, -1.2, 2.0), q=(1.1, 0.7, -1.5)) -> Problem:
    """u = p(x) q(y), p and q quadratics (coefficients low to high order)."""
    X, Y = _grid2(N)
    ax, ay = alpha
    bx, by = beta
    P = p[0] + p[1] * X + p[2] * X**2
    Px = p[1] + 2 * p[2] * X
    Pxx = 2 * p[2] + 0 * X
    Q = q[0] + q[1] * Y + q[2] * Y**2
    Qy = q[1] + 2 * q[2] * Y
    Qyy = 2 * q[2] + 0 * Y
    u = P * Q
    s = -ax * Pxx * Q - ay * P * Qyy + bx * Px * Q + by * P * Qy
    return Problem(2, N, tuple(alpha), tuple(beta), s, _boundary_only(u), u,
                   name=f"poly2d_N{N}")


def random_coefficients(rng: np.random.Generator, d: int, beta_max: float):
    alpha = tuple(float(a) for a in 10.0 ** rng.uniform(-2.0, 0.0, d))
    beta = tuple(float(b) for b in rng.uniform(-beta_max, beta_max, d))
    return alpha, beta


def random_fourier_2d(N: int, seed: int, modes: int = 16, kmax: int = 32,
                      beta_max: float = 10.0) -> Problem:
    """alpha_i log-uniform in [1e-2,1], beta_i ~ U(-beta_max, beta_max),
    s = sum_m a_m sin(k_m pi x) sin(l_m pi y), a_m ~ N(0,1), k_m,l_m ~ U{1..kmax}, g = 0."""
    rng = np.random.default_rng(seed)
    alpha, beta = random_coefficients(rng, 2, beta_max)
    a = rng.normal(size=modes)
    k = rng.integers(1, kmax + 1, modes)
    l = rng.integers(1, kmax + 1, modes)
    x = np.linspace(0.0, 1.0, N)
    sx = np.sin(np.pi * np.outer(k, x))      # [m, x]
    sy = np.sin(np.pi * np.outer(l, x))      # [m, y]
    s = np.einsum("m,my,mx->yx", a, sy, sx)
    g = np.zeros((N, N))
    return Problem(2, N, alpha, beta, s, g, None, name=f"fourier2d_N{N}_seed{seed}",
                   meta={"a": a, "k": k, "l": l, "seed": seed})


def manufactured_sine_3d(N: int, alpha=(1.0, 1.0, 1.0), beta=(1.0, 1.0, 1.0)) -> Problem:
    X, Y, Z = _grid3(N)
    ax, ay, az = alpha
    bx, by, bz = beta
    pi = np.pi
    sx, sy, sz = np.sin(pi * X), np.sin(pi * Y), np.sin(pi * Z)
    cx, cy, cz = np.cos(pi * X), np.cos(pi * Y), np.cos(pi * Z)
    u = sx * sy * sz
    s = (ax + ay + az) * pi**2 * u + pi * (bx * cx * sy * sz + by * sx * cy * sz + bz * sx * sy * cz)
    return Problem(3, N, tuple(alpha), tuple(beta), s, _boundary_only(u), u, name=f"sine3d_N{N}")


def random_sine_3d(N: int, seed: int, beta_max: float = 5.0) -> Problem:
    """Random alpha_i log-uniform in [1e-2,1], beta_i ~ U(-beta_max, beta_max), u = prod sin(pi x_i)."""
    rng = np.random.default_rng(seed)
    alpha, beta = random_coefficients(rng, 3, beta_max)
    p = manufactured_sine_3d(N, alpha, beta)
    p.name = f"randsine3d_N{N}_seed{seed}"
    p.meta["seed"] = seed
    return p


def batch_sizes(count: int, seed: int, choices=(129, 257, 513, 1025, 2049)):
    rng = np.random.default_rng(seed)
    return [int(c) for c in rng.choice(np.asarray(choices), size=count)]


def batch_hole(N: int) -> int:
    """Hole size n (fine intervals per coarse interval) of a batch instance:
    32, but at least 16 coarse intervals per axis on the small grids (with 4,
    strongly advective 129 x 129 instances stagnate in FP64 and mixed alike)."""
    return min(32, (N - 1) // 16)


def batch_problems(count: int = 64, seed: int = 0, choices=(129, 257, 513, 1025, 2049), seed0: int = 1000):
    """The uneven-size batch: sizes drawn from `choices`, instance i a
    random-Fourier problem (random_fourier_2d with seed seed0 + i), and its
    coarse interval count mc = (N - 1) / batch_hole(N)."""
    sizes = batch_sizes(count, seed, choices)
    probs = [random_fourier_2d(N, seed0 + i) for i, N in enumerate(sizes)]
    mcs = [(N - 1) // batch_hole(N) for N in sizes]
    return probs, mcs
