"""FP64 CPU oracle for 2D ASDSM with coefficients that vary in space
(K. Trotti, arXiv 2303.01163, Section 4, Example 1, second setting).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: only ``tests/`` do.  It shares no code with the CUDA path, which
solves constant-coefficient problems only.

eq. (1.1) with alpha_i = alpha_i(x, y), beta_i = beta_i(x, y):
    sum_i (-alpha_i(x, y) u_{x_i x_i} + beta_i(x, y) u_{x_i}) = s.
Algorithms 1-4 are those of ``asdsm2d`` unchanged: they use only the
operators of the four meshes, the projectors, the splines and the hole
solves; this module rebuilds the operators and right-hand sides and inherits
the rest.

Reading (the paper gives no discretisation for this case):

R29 Every (sub)mesh takes the centred differences of Section 2.3 with its own
    spacing and the coefficients sampled at the point itself (the
    non-divergence form of eq. (1.1)); Dirichlet lifting as R5 with the
    point's own coefficients.  With constant functions the operators are
    those of ``asdsm2d``.  A hole block of A_ff is still the hole's own
    operator (Remark 2.4), so Proposition 3.1 holds as before.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import asdsm2d as orc


def _coefs(points, M, hx, hy, alpha, beta):
    """Stencil weights at each point of a mesh (fine indices (i, j), spacing hx, hy):
    centre, west, east, south, north of A u."""
    x, y = points[:, 0] / M, points[:, 1] / M
    a1, a2 = alpha[0](x, y), alpha[1](x, y)
    b1, b2 = beta[0](x, y), beta[1](x, y)
    cc = 2.0 * a1 / hx**2 + 2.0 * a2 / hy**2
    cw, ce = -a1 / hx**2 - b1 / (2 * hx), -a1 / hx**2 + b1 / (2 * hx)
    cs, cn = -a2 / hy**2 - b2 / (2 * hy), -a2 / hy**2 + b2 / (2 * hy)
    return cc, cw, ce, cs, cn


def operator_2d_var(xs, ys, hx, hy, M, alpha, beta) -> sp.csr_matrix:
    """A on the product mesh xs x ys (fine indices, x fastest, R2) with spacing
    hx, hy: row of point p holds its own weights; neighbours outside the mesh
    are boundary points (their terms go to the right-hand side)."""
    nx, ny = len(xs), len(ys)
    pts = orc.Meshes2D._product(xs, ys)
    cc, cw, ce, cs, cn = _coefs(pts, M, hx, hy, alpha, beta)
    p = np.arange(nx * ny)
    ix, iy = p % nx, p // nx
    rows, cols, vals = [p], [p], [cc]
    for ok, off, w in ((ix > 0, -1, cw), (ix < nx - 1, 1, ce), (iy > 0, -nx, cs), (iy < ny - 1, nx, cn)):
        rows.append(p[ok])
        cols.append(p[ok] + off)
        vals.append(w[ok])
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(nx * ny, nx * ny))


def rhs_on_mesh_var(points, hx, hy, M, alpha, beta, s_grid, g_grid) -> np.ndarray:
    """Samples of s plus the lifting of the boundary neighbours (R29); grids [y, x]."""
    i, j = points[:, 0], points[:, 1]
    sx, sy = int(round(hx * M)), int(round(hy * M))
    _, cw, ce, cs, cn = _coefs(points, M, hx, hy, alpha, beta)
    b = np.array(s_grid[j, i], dtype=np.float64)
    b -= np.where(i - sx == 0, cw * g_grid[j, 0], 0.0)
    b -= np.where(i + sx == M, ce * g_grid[j, M], 0.0)
    b -= np.where(j - sy == 0, cs * g_grid[0, i], 0.0)
    b -= np.where(j + sy == M, cn * g_grid[M, i], 0.0)
    return b


class Discretisation2DVar(orc.Discretisation2D):
    """The linear systems of eq. (2.4) with variable coefficients; Algorithms
    1-4 (skeleton, filler, initial_guess, correction, asdsm) as in asdsm2d.

    alpha, beta: pairs of functions of (x, y) (numpy arrays in, arrays out)."""

    def __init__(self, N: int, mc: int, alpha, beta):
        self.m = orc.Meshes2D(N, mc)
        m = self.m
        self.alpha_fn, self.beta_fn = tuple(alpha), tuple(beta)
        h, H, M = m.h, m.H, m.M
        fine = np.arange(1, M)
        coarse = np.arange(1, m.mc) * m.n
        op = lambda xs, ys, hx, hy: operator_2d_var(xs, ys, hx, hy, M, self.alpha_fn, self.beta_fn)
        self.A_ff = op(fine, fine, h, h)
        self.A_fc = op(fine, coarse, h, H)
        self.A_cf = op(coarse, fine, H, h)
        self.A_cc = op(coarse, coarse, H, H)
        self.P_ff_fc = orc.projector(m.fc, m.ff, N)
        self.P_ff_cf = orc.projector(m.cf, m.ff, N)
        self.P_ff_cc = orc.projector(m.cc, m.ff, N)
        self.P_ff_holes = orc.projector(m.holes, m.ff, N)
        self.P_fc_cc = orc.projector(m.cc, m.fc, N)
        self.P_cf_cc = orc.projector(m.cc, m.cf, N)
        self.P_ff_skel = orc.projector(m.skeleton, m.ff, N)
        self.lu_fc = spla.splu(self.A_fc.tocsc())
        self.lu_cf = spla.splu(self.A_cf.tocsc())
        self.lu_cc = spla.splu(self.A_cc.tocsc())
        self.lu_holes = spla.splu((self.P_ff_holes @ self.A_ff @ self.P_ff_holes.T).tocsc())
        self._lu_ff = None
        self.knots = np.linspace(0.0, 1.0, m.mc + 1)
        self.fine_x = np.arange(1, M) * h

    def rhs(self, s_grid, g_grid):
        """b_ff, b_fc, b_cf, b_cc (R29)."""
        m = self.m
        h, H, M = m.h, m.H, m.M
        f = lambda pts, hx, hy: rhs_on_mesh_var(pts, hx, hy, M, self.alpha_fn, self.beta_fn, s_grid, g_grid)
        return f(m.ff, h, h), f(m.fc, h, H), f(m.cf, H, h), f(m.cc, H, H)


def residual_grid_var(N, alpha, beta, s_grid, u_grid):
    """r = b_ff - A_ff u on the interior from the full grid u (its boundary is g)."""
    M = N - 1
    h = 1.0 / M
    fine = np.arange(1, M)
    A = operator_2d_var(fine, fine, h, h, M, alpha, beta)
    b = rhs_on_mesh_var(orc.Meshes2D._product(fine, fine), h, h, M, alpha, beta, s_grid, u_grid)
    return b - A @ orc.interior(u_grid), b
