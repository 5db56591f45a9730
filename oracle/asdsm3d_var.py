"""FP64 CPU oracle for the 3D extension with coefficients that vary in space
(K. Trotti, arXiv 2303.01163, Section 4, Example 4, second setting).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: only ``tests/`` do.  It shares no code with the CUDA path, which
solves constant-coefficient problems only.

eq. (1.1) in 3D with alpha_i = alpha_i(x, y, z), beta_i = beta_i(x, y, z).
Reading R29 of ``asdsm2d_var`` in 3D: the 7-point centred differences on
every (sub)mesh with its own spacing per axis and the coefficients sampled at
the point itself; lifting with the point's own weights.  Algorithms 1-4 (the
merge R21-R23, the cube-hole Filler, GCR) are those of ``asdsm3d``, which
this module inherits; only the operators and right-hand sides change.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import asdsm3d as o3


def _weights(points, M, spacing, alpha, beta):
    """Centre and (lower, upper) neighbour weights per axis of A u at each point."""
    x, y, z = points[:, 0] / M, points[:, 1] / M, points[:, 2] / M
    cc = np.zeros(len(points))
    lo, up = [], []
    for a in range(3):
        h = spacing[a]
        al, be = alpha[a](x, y, z), beta[a](x, y, z)
        cc = cc + 2.0 * al / h**2
        lo.append(-al / h**2 - be / (2 * h))
        up.append(-al / h**2 + be / (2 * h))
    return cc, lo, up


def operator_3d_var(axes, spacing, M, alpha, beta) -> sp.csr_matrix:
    """A on the product mesh axes[0] x axes[1] x axes[2] (fine indices, x
    fastest) with the given spacing per axis; neighbours outside the mesh are
    boundary points (their terms go to the right-hand side)."""
    nx, ny, nz = (len(v) for v in axes)
    pts = o3.Meshes3D._product(*axes)
    cc, lo, up = _weights(pts, M, spacing, alpha, beta)
    p = np.arange(nx * ny * nz)
    idx = (p % nx, (p // nx) % ny, p // (nx * ny))
    stride = (1, nx, nx * ny)
    size = (nx, ny, nz)
    rows, cols, vals = [p], [p], [cc]
    for a in range(3):
        for ok, off, w in ((idx[a] > 0, -stride[a], lo[a]), (idx[a] < size[a] - 1, stride[a], up[a])):
            rows.append(p[ok])
            cols.append(p[ok] + off)
            vals.append(w[ok])
    n = nx * ny * nz
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, n))


def rhs_on_mesh_var3(points, spacing, M, alpha, beta, s_grid, g_grid) -> np.ndarray:
    """Samples of s plus the lifting of the boundary neighbours; grids [z, y, x]."""
    i, j, l = points[:, 0], points[:, 1], points[:, 2]
    _, lo, up = _weights(points, M, spacing, alpha, beta)
    b = np.array(s_grid[l, j, i], dtype=np.float64)
    idx = (i, j, l)
    for a in range(3):
        st = int(round(spacing[a] * M))
        q = list(idx)
        q[a] = np.zeros_like(i)
        b -= np.where(idx[a] - st == 0, lo[a] * g_grid[q[2], q[1], q[0]], 0.0)
        q[a] = np.full_like(i, M)
        b -= np.where(idx[a] + st == M, up[a] * g_grid[q[2], q[1], q[0]], 0.0)
    return b


class Discretisation3DVar(o3.Discretisation3D):
    """The 3D systems with variable coefficients; Algorithms 1-4 as in asdsm3d.

    alpha, beta: three functions of (x, y, z) each (numpy arrays in and out)."""

    def __init__(self, N: int, mc: int, alpha, beta):
        self.m = o3.Meshes3D(N, mc)
        m = self.m
        self.alpha_fn, self.beta_fn = tuple(alpha), tuple(beta)

        def op(coarse_axes):
            axes = [m.coarse if a in coarse_axes else m.fine for a in range(3)]
            return operator_3d_var(axes, o3._spacing(m, coarse_axes), m.M, self.alpha_fn, self.beta_fn)

        self.A_ff = op(())
        self.A_plane = {f: op((self.AX[f],)) for f in o3.FAMILIES}
        self.A_line = {f: op(tuple(a for a in range(3) if a != self.AX[f])) for f in o3.FAMILIES}
        self.A_cc = op((0, 1, 2))
        self.P_plane = {f: o3.projector(m.plane[f], m.ff, N) for f in o3.FAMILIES}
        self.P_holes = o3.projector(m.holes, m.ff, N)
        self.P_skel = o3.projector(m.skeleton, m.ff, N)
        self.lu_plane = {f: spla.splu(self.A_plane[f].tocsc()) for f in o3.FAMILIES}
        self.lu_line = {f: spla.splu(self.A_line[f].tocsc()) for f in o3.FAMILIES}
        self.lu_cc = spla.splu(self.A_cc.tocsc())
        self.lu_holes = spla.splu((self.P_holes @ self.A_ff @ self.P_holes.T).tocsc())
        self._lu_ff = None
        self.knots = np.linspace(0.0, 1.0, mc + 1)
        self.fine_x = m.fine * m.h

    def rhs(self, s_grid, g_grid):
        """b_ff, the plane, line and coarse right-hand sides (dicts by family)."""
        m = self.m
        f = lambda pts, coarse_axes: rhs_on_mesh_var3(pts, o3._spacing(m, coarse_axes), m.M, self.alpha_fn,
                                                      self.beta_fn, s_grid, g_grid)
        b_ff = f(m.ff, ())
        b_p = {q: f(m.plane[q], (self.AX[q],)) for q in o3.FAMILIES}
        b_l = {q: f(m.line[q], tuple(x for x in range(3) if x != self.AX[q])) for q in o3.FAMILIES}
        b_c = f(m.cc, (0, 1, 2))
        return b_ff, b_p, b_l, b_c
