"""FP64 CPU oracle for the 3D extension of the Anisotropic Submeshes Domain
Splitting Method (K. Trotti, arXiv 2303.01163, Section "Extension to the 3D
case").

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: only ``tests/`` (and the test-only entry points named in the 2D
oracle) do.  It shares no code with the CUDA path.

The paper extends ASDSM to 3D by iterating over the three strongly anisotropic
plane families Omega^{H,h,h}, Omega^{h,H,h}, Omega^{h,h,H} (coarse in one axis,
fine in the other two) with Omega^{H,H,H} as the coarse intersection mesh, and
by extrapolating the other intersection points too, since Omega^{H,H,H} no
longer holds all of them (the lines where two plane families meet).  What this
module computes, in the paper's order:

* meshes: the fine mesh Omega^{h,h,h}; the plane families P_x = Omega^{H,h,h}
  (x on the coarse knots), P_y, P_z; the line families L_x = Omega^{h,H,H}
  (fine in x only), L_y, L_z; the coarse mesh C = Omega^{H,H,H}.  The holes are
  the cubes between planes; the skeleton is the union of the planes.
* the 7-point centred finite differences of eq. (1.1) on every (sub)mesh, each
  with its own spacing per axis, in Kronecker form, and Dirichlet lifting.
* Algorithm 1 in 3D: the plane solutions (for the initial guess also the line
  and coarse solutions), merged by Algorithm 2 in 3D, filled by Algorithm 3
  (cube holes with Dirichlet data on their six faces).
* Algorithm 4 as in 2D: residual, projections of r on the three plane families,
  Algorithm 1 on them, optimal step (or GCR(m), R15 of the 2D oracle), update.

Library primitives used as single steps: ``scipy.sparse.linalg.splu`` for
every "(A)^{-1} b" and ``scipy.interpolate.CubicSpline`` for "Spline".

Readings (the 2D readings R1-R18 of ``asdsm2d`` carry over):

R20 Meshes and ordering: points (i, j, l) in fine indices (x = i h, y = j h,
    z = l h), listed x fastest, then y, then z; full grids are arrays [z, y, x].
R21 Extrapolation at intersection points (the extrapolation of Algorithm 2
    in 3D, by the combination technique): at knots (points of C)
        u_hat = u_Px + u_Py + u_Pz - u_Lx - u_Ly - u_Lz + u_C,
    and at the other points of a line where two plane families meet (e.g.
    x = kH, y = lH, z fine: P_x and P_y meet on L_z)
        u_hat = u_Px + u_Py - u_Lz.
    This is why the initial guess also solves the line meshes.
R22 Random choice of Algorithm 2 in 3D: one draw per call, uniform over
    the three plane families (SplitMix64 output mod 3, same counter as R8); a
    line point outside the chosen family takes the value of the next family
    in the cyclic order x -> y -> z -> x that contains it.
R23 Spline correction of Algorithm 2 on a plane in 3D: on the plane of
    P_x the errors are known on its lines y = lH and z = mH (where it meets P_y
    and P_z); the correction is the Boolean sum (transfinite interpolation)
        S_y e + S_z e - S_y S_z e
    of the not-a-knot cubic splines (R10) along the plane's two fine axes.
    It equals e on every line of the plane.
R24 Normalisation of Algorithm 1 in 3D: each plane solution by its own
    Euclidean norm; a zero vector stays zero.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.interpolate import CubicSpline

from .asdsm2d import L_matrix, D_matrix, splitmix64, _GOLDEN_GAMMA, _MASK64, hole_fix_due

FAMILIES = ("x", "y", "z")          # plane family P_a: coordinate a on the coarse knots


def choice3(seed: int, k: int) -> int:
    """Family drawn by the random choice of Algorithm 2 at ASDSM sweep k (R22): 0, 1 or 2."""
    return splitmix64((seed + (k + 1) * _GOLDEN_GAMMA) & _MASK64) % 3


# ---------------------------------------------------------------------------
# Meshes (R20).
# ---------------------------------------------------------------------------
class Meshes3D:
    """Fine, plane, line and coarse meshes for N points per side and mc coarse intervals."""

    def __init__(self, N: int, mc: int):
        M = N - 1
        if N < 3 or mc < 2 or M % mc != 0:
            raise ValueError("eq. (2.1) needs (N-1) % mc == 0 with mc >= 2")
        self.N, self.M, self.mc = N, M, mc
        self.n = M // mc
        self.Nf, self.Nc = M - 1, mc - 1
        self.h, self.H = 1.0 / M, 1.0 / mc
        fine = np.arange(1, M)
        coarse = np.arange(1, mc) * self.n
        self.fine, self.coarse = fine, coarse
        P = self._product
        self.ff = P(fine, fine, fine)
        self.plane = {"x": P(coarse, fine, fine), "y": P(fine, coarse, fine), "z": P(fine, fine, coarse)}
        self.line = {"x": P(fine, coarse, coarse), "y": P(coarse, fine, coarse), "z": P(coarse, coarse, fine)}
        self.cc = P(coarse, coarse, coarse)
        on = self.ff % self.n == 0
        self.holes = self.ff[~on.any(axis=1)]
        self.skeleton = self.ff[on.any(axis=1)]

    @staticmethod
    def _product(xs, ys, zs):
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")        # z slowest, x fastest
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def flat(self, points):
        """Index of each point in a full N^3 grid stored [z, y, x]."""
        N = self.N
        return (points[:, 2] * N + points[:, 1]) * N + points[:, 0]


def projector(rows_mesh, cols_mesh, N: int) -> sp.csr_matrix:
    """P with P[m, q] = 1 iff point m of rows_mesh equals point q of cols_mesh (Definition 2.2)."""
    where = np.full(N * N * N, -1, dtype=np.int64)
    where[(cols_mesh[:, 2] * N + cols_mesh[:, 1]) * N + cols_mesh[:, 0]] = np.arange(len(cols_mesh))
    c = where[(rows_mesh[:, 2] * N + rows_mesh[:, 1]) * N + rows_mesh[:, 0]]
    if np.any(c < 0):
        raise ValueError("rows_mesh is not a subset of cols_mesh")
    r = np.arange(len(rows_mesh))
    return sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(len(rows_mesh), len(cols_mesh)))


# ---------------------------------------------------------------------------
# 7-point operator and right-hand sides (Section 2.3 in 3D).
# ---------------------------------------------------------------------------
def operator_3d(nx, hx, ny, hy, nz, hz, alpha, beta) -> sp.csr_matrix:
    """sum_a alpha_a L_a/h_a^2 + beta_a D_a/(2 h_a), Kronecker form, x fastest (R20)."""
    ax, ay, az = alpha
    bx, by, bz = beta
    Ix, Iy, Iz = (sp.identity(k, format="csr") for k in (nx, ny, nz))
    kx = lambda T: sp.kron(Iz, sp.kron(Iy, T))
    ky = lambda T: sp.kron(Iz, sp.kron(T, Ix))
    kz = lambda T: sp.kron(T, sp.kron(Iy, Ix))
    A = (ax * kx(L_matrix(nx) / hx**2) + ay * ky(L_matrix(ny) / hy**2) + az * kz(L_matrix(nz) / hz**2)
         + bx * kx(D_matrix(nx) / (2 * hx)) + by * ky(D_matrix(ny) / (2 * hy)) + bz * kz(D_matrix(nz) / (2 * hz)))
    return A.tocsr()


def rhs_on_mesh(points, spacing, alpha, beta, s_grid, g_grid, M: int) -> np.ndarray:
    """Samples of s plus the Dirichlet lifting with the mesh's own spacing (R5).

    A neighbour that falls on the boundary moves its stencil coefficient times
    g there to the right-hand side.  Grids are [z, y, x]."""
    i, j, l = points[:, 0], points[:, 1], points[:, 2]
    b = np.array(s_grid[l, j, i], dtype=np.float64)
    idx = (i, j, l)
    for a in range(3):
        h = spacing[a]
        st = int(round(h * M))
        lo = alpha[a] / h**2 + beta[a] / (2 * h)          # coefficient of the lower neighbour, moved
        hi = alpha[a] / h**2 - beta[a] / (2 * h)          # upper neighbour
        q = list(idx)
        q[a] = np.zeros_like(i)
        at_lo = idx[a] - st == 0
        b += np.where(at_lo, lo * g_grid[q[2], q[1], q[0]], 0.0)
        q[a] = np.full_like(i, M)
        at_hi = idx[a] + st == M
        b += np.where(at_hi, hi * g_grid[q[2], q[1], q[0]], 0.0)
    return b


def _spacing(m: Meshes3D, coarse_axes):
    return tuple(m.H if a in coarse_axes else m.h for a in range(3))


def _sizes(m: Meshes3D, coarse_axes):
    return tuple(m.Nc if a in coarse_axes else m.Nf for a in range(3))


class Discretisation3D:
    """The linear systems of the 3D extension and Algorithms 1-4 for one problem."""

    AX = {"x": 0, "y": 1, "z": 2}

    def __init__(self, N: int, mc: int, alpha, beta):
        self.m = Meshes3D(N, mc)
        m = self.m
        self.alpha = tuple(float(a) for a in alpha)
        self.beta = tuple(float(b) for b in beta)
        if len(self.alpha) != 3 or len(self.beta) != 3 or min(self.alpha) <= 0:
            raise ValueError("three alpha_i > 0 and three beta_i")
        op = lambda coarse_axes: operator_3d(*[v for a in range(3) for v in (
            _sizes(m, coarse_axes)[a], _spacing(m, coarse_axes)[a])], self.alpha, self.beta)
        self.A_ff = op(())
        self.A_plane = {f: op((self.AX[f],)) for f in FAMILIES}
        self.A_line = {f: op(tuple(a for a in range(3) if a != self.AX[f])) for f in FAMILIES}
        self.A_cc = op((0, 1, 2))
        self.P_plane = {f: projector(m.plane[f], m.ff, N) for f in FAMILIES}
        self.P_holes = projector(m.holes, m.ff, N)
        self.P_skel = projector(m.skeleton, m.ff, N)
        self.lu_plane = {f: spla.splu(self.A_plane[f].tocsc()) for f in FAMILIES}
        self.lu_line = {f: spla.splu(self.A_line[f].tocsc()) for f in FAMILIES}
        self.lu_cc = spla.splu(self.A_cc.tocsc())
        self.lu_holes = spla.splu((self.P_holes @ self.A_ff @ self.P_holes.T).tocsc())
        self._lu_ff = None
        self.knots = np.linspace(0.0, 1.0, mc + 1)
        self.fine_x = m.fine * m.h

    # -- right-hand sides ---------------------------------------------------
    def rhs(self, s_grid, g_grid):
        """b_ff, the plane, line and coarse right-hand sides (dicts by family)."""
        m, a, be = self.m, self.alpha, self.beta
        b_ff = rhs_on_mesh(m.ff, _spacing(m, ()), a, be, s_grid, g_grid, m.M)
        b_p = {f: rhs_on_mesh(m.plane[f], _spacing(m, (self.AX[f],)), a, be, s_grid, g_grid, m.M) for f in FAMILIES}
        b_l = {f: rhs_on_mesh(m.line[f], _spacing(m, tuple(x for x in range(3) if x != self.AX[f])), a, be,
                              s_grid, g_grid, m.M) for f in FAMILIES}
        b_c = rhs_on_mesh(m.cc, _spacing(m, (0, 1, 2)), a, be, s_grid, g_grid, m.M)
        return b_ff, b_p, b_l, b_c

    def solve_fine(self, b_ff):
        if self._lu_ff is None:
            self._lu_ff = spla.splu(self.A_ff.tocsc())
        return self._lu_ff.solve(b_ff)

    # -- helpers on full grids ------------------------------------------------
    def to_full(self, points, values):
        G = np.zeros(self.m.N ** 3)
        G[self.m.flat(points)] = values
        return G.reshape(self.m.N, self.m.N, self.m.N)

    def _masks(self):
        """Full-grid masks: which plane families contain each grid point."""
        m = self.m
        N, n = m.N, m.n
        g = np.arange(N)
        interior = (g > 0) & (g < N - 1)
        onc = interior & (g % n == 0)
        Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
        inner = interior[X] & interior[Y] & interior[Z]
        return {"x": inner & onc[X], "y": inner & onc[Y], "z": inner & onc[Z]}

    # -- Algorithm 2 in 3D ------------------------------------------------------
    def plane_correction(self, f, E):
        """Boolean sum of R23 on every plane of family f.

        E: full grid [z, y, x] holding the errors on the lines of the planes of
        family f (other entries ignored).  Returns the correction on every
        point of those planes (full grid, zero elsewhere)."""
        m = self.m
        a = self.AX[f]
        b, c = [x for x in range(3) if x != a]         # the plane's two fine axes, b < c
        out = np.zeros_like(E)
        co, fi = m.coarse, m.fine

        def spline_along(vals_on_knots, axis):
            # vals: array with the knot axis of length mc+1 at position `axis`
            return CubicSpline(self.knots, vals_on_knots, axis=axis, bc_type="not-a-knot")(self.fine_x)

        for k in co:                                    # one plane a = k
            P = np.take(E, k, axis=2 - a)               # 2D array over the other two axes, [.., ..] in grid order
            # grid order [z, y, x] minus axis a: remaining axes in order (c, b) as array dims (slow, fast)
            # P[u, v]: u indexes axis c, v indexes axis b
            nb = np.zeros((m.N, m.mc + 1))              # S_b: along b, for every u (axis c)
            nb[:, 1:-1] = P[:, co]
            Sb = np.zeros_like(P)
            Sb[:, fi] = spline_along(nb, 1)             # S_b e on every row u
            nc = np.zeros((m.mc + 1, m.N))
            nc[1:-1, :] = P[co, :]
            Sc = np.zeros_like(P)
            Sc[fi, :] = spline_along(nc, 0)             # S_c e on every column v
            # S_b S_c e: S_b applied to (S_c e) sampled on the knots of b
            nbc = np.zeros((m.N, m.mc + 1))
            nbc[:, 1:-1] = Sc[:, co]
            Sbc = np.zeros_like(P)
            Sbc[:, fi] = spline_along(nbc, 1)
            C = Sb + Sc - Sbc
            sl = [slice(None)] * 3
            sl[2 - a] = k
            mask = np.zeros_like(P, dtype=bool)
            mask[np.ix_(fi, fi)] = True
            Cm = np.where(mask, C, 0.0)
            out[tuple(sl)] = Cm
        return out

    def skeleton(self, U_plane, U_line=None, U_cc=None, choice=0):
        """Algorithm 2 in 3D (R21-R23).

        U_plane: dict family -> full grid with that family's (normalised)
        solution on its points; U_line, U_cc: full grids of the line and coarse
        solutions (initial guess, R21) or None (random choice, R22).
        Returns the merged skeleton on the fine interior (vector, zero in the holes)."""
        msk = self._masks()
        Mx, My, Mz = msk["x"], msk["y"], msk["z"]
        cnt = Mx.astype(int) + My + Mz
        inter = cnt >= 2                                               # lines and knots
        Ux, Uy, Uz = U_plane["x"], U_plane["y"], U_plane["z"]
        if U_line is not None:                                         # extrapolation (R21)
            knot = cnt == 3
            u_hat = np.where(knot, Ux + Uy + Uz - U_line["x"] - U_line["y"] - U_line["z"] + U_cc, 0.0)
            u_hat = np.where(Mx & My & ~knot, Ux + Uy - U_line["z"], u_hat)
            u_hat = np.where(My & Mz & ~knot, Uy + Uz - U_line["x"], u_hat)
            u_hat = np.where(Mx & Mz & ~knot, Ux + Uz - U_line["y"], u_hat)
        else:                                                          # random choice (R22)
            order = [FAMILIES[(choice + t) % 3] for t in range(3)]
            u_hat = np.zeros_like(Ux)
            taken = np.zeros_like(inter)
            for f in order:
                sel = inter & msk[f] & ~taken
                u_hat = np.where(sel, U_plane[f], u_hat)
                taken |= sel
        # each plane moved onto u_hat along its lines by the Boolean-sum spline of its mismatch (R23)
        corrected = {}
        for f in FAMILIES:
            E = np.where(inter & msk[f], u_hat - U_plane[f], 0.0)
            corrected[f] = U_plane[f] + self.plane_correction(f, E)
        # the union of the corrected planes (they agree on the lines)
        S = np.zeros_like(Ux)
        for f in FAMILIES:
            S = np.where(msk[f], corrected[f], S)
        return S[1:-1, 1:-1, 1:-1].reshape(-1), corrected, u_hat

    # -- Algorithm 3 ------------------------------------------------------------
    def filler(self, u_t, b_ff):
        """Algorithm 3 for the cube holes: u_holes += A_hh^{-1} P_holes (b_ff - A_ff u_t),
        which zeroes the residual at every hole point (Prop. 3.1 in 3D)."""
        v = self.lu_holes.solve(self.P_holes @ (b_ff - self.A_ff @ u_t))
        return u_t + self.P_holes.T @ v

    # -- Algorithm 1 in 3D --------------------------------------------------------
    def initial_guess(self, b_ff, b_plane, b_line=None, b_cc=None, choice=0):
        """Algorithm 1 in 3D: the three plane families solved exactly; for the
        first iterate (b_line, b_cc given) also the line families and the coarse
        mesh, which the extrapolating merge needs (R21); for a sweep's
        correction each plane solution normalised by its own norm (R24) and
        merged by the random choice (R22); then the cube-hole Filler."""
        m = self.m
        U_plane = {}
        for f in FAMILIES:
            u = self.lu_plane[f].solve(b_plane[f])
            if b_line is None:
                nrm = np.linalg.norm(u)
                if nrm > 0:
                    u = u / nrm
            U_plane[f] = self.to_full(m.plane[f], u)
        U_line = U_cc = None
        if b_line is not None:
            U_line = {f: self.to_full(m.line[f], self.lu_line[f].solve(b_line[f])) for f in FAMILIES}
            U_cc = self.to_full(m.cc, self.lu_cc.solve(b_cc))
        u_t, _, _ = self.skeleton(U_plane, U_line, U_cc, choice)
        return self.filler(u_t, b_ff)

    def residual(self, b_ff, u):
        return b_ff - self.A_ff @ u


def asdsm(disc: Discretisation3D, b, *, tol=1e-10, max_sweeps=200, accel_m=1, seed=0,
          stagnation_window=10, stagnation_factor=1e-3, hole_fix_ratio=0.25, hole_fix_growth=4.0, u0=None):
    """Algorithm 4 in 3D with the readings R13-R15 and R18 of the 2D oracle
    (R18: a Filler pass on the cube holes replaces a sweep when rounding has
    left a hole residual above hole_fix_ratio of the whole residual and above
    hole_fix_growth times its size after the previous pass).

    b = (b_ff, b_plane, b_line, b_cc) from Discretisation3D.rhs."""
    b_ff, b_p, b_l, b_c = b
    sk = disc.P_skel
    u = disc.initial_guess(b_ff, b_p, b_l, b_c) if u0 is None else np.array(u0, dtype=np.float64)
    nb = np.linalg.norm(b_ff)
    hist, steps, choices, kinds = [], [], [], []
    Z, Q = [], []
    hole_ref = 0.0
    status = "max_sweeps"
    k = 0
    while True:
        r = disc.residual(b_ff, u)
        rel = np.linalg.norm(r) / nb if nb > 0 else np.linalg.norm(r)
        hist.append(rel)
        if rel <= tol:
            status = "converged"
            break
        if k >= max_sweeps:
            break
        if (len(hist) > stagnation_window and
                hist[-1] > (1 - stagnation_factor) * hist[-1 - stagnation_window]):
            status = "stagnated"
            break
        if hole_fix_due(np.linalg.norm(disc.P_holes @ r), np.linalg.norm(r), hole_ref, hole_fix_ratio,
                        hole_fix_growth):
            u = disc.filler(u, b_ff)
            hole_ref = np.linalg.norm(disc.P_holes @ disc.residual(b_ff, u))
            Z, Q = [], []
            kinds.append("hole_fix")
            choices.append(-1)
            steps.append(1.0)
            k += 1
            continue
        ch = choice3(seed, k)
        # the correction: Algorithm 1 on the error equations of the plane meshes
        r_p = {f: disc.P_plane[f] @ r for f in FAMILIES}
        e = disc.initial_guess(0.0 * b_ff, r_p, None, None, ch)
        q = sk @ (disc.A_ff @ e)
        rs = sk @ r
        if accel_m == 1:
            qq = q @ q
            s_hat = max(0.0, (rs @ q) / qq) if qq > 0 else 0.0        # R14
            u = u + s_hat * e
            steps.append(s_hat)
        else:
            for zj, qj in zip(Z, Q):                                   # R15
                beta_j = q @ qj
                q = q - beta_j * qj
                e = e - beta_j * zj
            nq = np.linalg.norm(q)
            if nq > 0:
                q, e = q / nq, e / nq
                a = rs @ q
                u = u + a * e
                Z.append(e)
                Q.append(q)
                steps.append(a)
            else:
                steps.append(0.0)
            if len(Z) >= accel_m:
                Z, Q = [], []
        choices.append(ch)
        kinds.append("sweep")
        k += 1
    return u, {"hist": hist, "steps": steps, "choices": choices, "kinds": kinds, "status": status, "sweeps": k}


# ---------------------------------------------------------------------------
# Full-grid helpers ([z, y, x], boundary included).
# ---------------------------------------------------------------------------
def interior(grid3d):
    return np.asarray(grid3d)[1:-1, 1:-1, 1:-1].reshape(-1)


def fine_system3d(N: int, alpha, beta, s_grid, g_grid):
    """A_ff and b_ff of eq. (1.1) in 3D on the fine mesh alone (Section 2.3 in 3D).

    The same operator and lifting as ``Discretisation3D`` builds for its fine
    mesh, without the submesh operators and factorizations, so that a grid of
    257^3 points fits in a few GB and seconds."""
    M = N - 1
    fine = np.arange(1, M)
    A = operator_3d(M - 1, 1.0 / M, M - 1, 1.0 / M, M - 1, 1.0 / M, alpha, beta)
    b = rhs_on_mesh(Meshes3D._product(fine, fine, fine), (1.0 / M,) * 3, alpha, beta, s_grid, g_grid, M)
    return A, b


def residual_grid3d(N: int, alpha, beta, s_grid, u_grid):
    """r = b_ff - A_ff u on the interior, from the full grid u (its boundary is g)."""
    A, b = fine_system3d(N, alpha, beta, s_grid, u_grid)
    return b - A @ interior(u_grid), b


def to_grid(u_ff, g_grid):
    out = np.array(g_grid, dtype=np.float64, copy=True)
    n = out.shape[0] - 2
    out[1:-1, 1:-1, 1:-1] = u_ff.reshape(n, n, n)
    return out
