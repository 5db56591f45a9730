"""FP64 CPU oracle for the 2D Anisotropic Submeshes Domain Splitting Method.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / ``--impl reference`` legs do.  It shares no code with the
CUDA path.

What it computes, in the paper's notation
(K. Trotti, "A domain splitting strategy for solving PDEs", arXiv 2303.01163):

* eq. (2.1)/(2.3): meshes Omega^{h,h}, Omega^{h,H} ("fc"), Omega^{H,h} ("cf"),
  Omega^{H,H} ("cc") and the holes Omega_{i,j}.
* Definition 2.2: the 0/1 selection projectors, built here as explicit sparse
  matrices so every transfer reads exactly as in the paper.
* Section 2.3: second-order centred finite differences in Kronecker form,
  A = alpha (I (x) L/h^2 + L/h^2 (x) I) + beta (I (x) D/(2h) + D/(2h) (x) I),
  with per-axis alpha_i, beta_i.
* Section 3.1: the initial guess (Algorithm 1) from the two anisotropic
  solutions, their merge into one skeleton (Algorithm 2) and the hole solves
  (Algorithm 3), each written as the map it defines rather than as a listing.
* Section 3.2: the ASDSM iteration (Algorithm 4) with the clamped optimal
  scaling s_hat of the correction.

Library primitives used as single steps: ``scipy.sparse.linalg.splu`` for
every "(A)^{-1} b" of the algorithms (each matrix is factored once and reused)
and ``scipy.interpolate.CubicSpline`` for "Spline" in Algorithm 2.

Readings where the paper is silent, ambiguous or garbled:

R1  N and mc.  The API takes N grid points per side including the boundary
    and mc coarse intervals; eq. (2.1) becomes (N-1) % mc == 0, with
    N_f = N-2, N_c = mc-1, n = (N-1)/mc.
R2  Ordering is x fastest (the listed vector of Section 2.2 and the
    Kronecker form), not the index formula of Remark 2.1.
R3  Per-axis coefficients alpha_i, beta_i in A (eq. (1.1) has them).
R4  eq. (1.1) reads sum_i (-alpha_i u_{x_i x_i} + beta_i u_{x_i}) = s,
    matching L = tridiag(-1, 2, -1) and D = tridiag(-1, 0, 1).
R5  Dirichlet data enter the right-hand side of every mesh by the usual
    lifting: a stencil term that reaches a boundary point moves to b with
    that mesh's own spacing.  Error equations have zero boundary data.
R7  The Richardson extrapolation of Algorithm 2 is the 2D combination
    u_hat = P u_fc + P u_cf - u_cc (error C_x h^2 + C_y h^2 after the
    combination when each mesh carries C_x h_x^2 + C_y h_y^2).
R8  The random choice of Algorithm 2 is one draw per call for the
    whole coarse vector, taken from the counter-based SplitMix64 generator
    (choice_bit below), so the CUDA path draws the same sequence.
R9  The normalisation of Algorithm 1 is by the Euclidean norm of the
    whole submesh vector; a zero vector stays zero.
R10 "Spline ... with zero BCs" is the not-a-knot cubic spline through the
    knots x = 0, H, ..., 1 with zero values at x = 0 and x = 1.
R11 Cross points of the merged skeleton take the corrected fc value,
    which is what the assembly of Algorithm 2 writes.
R13 The loop runs while ||r||/||b|| > tol, k < max_sweeps and the residual
    has not stagnated (||r_k|| > (1 - 1e-3) ||r_{k-10}||).
R14 s_hat = max(0, <r, A e>/<A e, A e>), least squares over the skeleton
    rows, where A e is non-zero (Prop. 3.1; Section 3.3, first two remarks).
R15 Refinement to tight tolerances: with accel_m > 1 the correction e of
    Algorithm 4 is used as a flexible preconditioner inside
    restarted GCR(m): the new A e is orthogonalised against the cycle's
    previous ones and the step is the unconstrained least-squares
    coefficient.  accel_m = 1 is exactly the paper's clamped optimal step.
R18 Hole residual.  In exact arithmetic the residual vanishes in the holes
    (Prop. 3.1).  When rounding has made its hole part exceed both
    hole_fix_ratio * ||r|| and hole_fix_growth times its value just after
    the last such correction (zero before the first one), the sweep is
    replaced by Algorithm 3 applied to the current iterate, which solves
    the hole systems with the hole part of the current residual and zeroes
    it (down to rounding).  The GCR cycle
    restarts afterwards.
R27 Residual smoothing (Example 2 of Section 4, where the paper reports that
    an unspecified artificial smoothing of the residual lowers the point where
    plain ASDSM stagnates).  Two readings, both off by default: "knots"
    replaces the projected residual at every cross point of a line by the
    mean of its two fine-axis neighbours on that line (the irregularity the
    paper shows sits at the coarse points); "lines" filters every projected
    line with [1, 2, 1]/4 along its fine axis (zero beyond the boundary).
R28 Extra anisotropic meshes for the extrapolation (the remark after
    Algorithm 2, meshes Omega^{kh,H} and Omega^{H,kh}), with k = 2: the
    samples f2, c2 of the solutions on Omega^{2h,H} and Omega^{H,2h} at the
    coarse points remove each family's own fine-axis h^2 term,
        u_hat = (4 fc - f2)/3 + (4 cf - c2)/3 - cc,
    which extrapolates towards the continuous solution rather than towards
    the fine discrete solution that ASDSM converges to.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy.interpolate import CubicSpline

# ---------------------------------------------------------------------------
# Counter-based random choice (R8): SplitMix64 (Steele, Lea, Flood 2014).
# ---------------------------------------------------------------------------
_MASK64 = (1 << 64) - 1
_GOLDEN_GAMMA = 0x9E3779B97F4A7C15


def splitmix64(state: int) -> int:
    """Output of SplitMix64 for the given (already advanced) 64-bit state."""
    z = state & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def splitmix64_stream(seed: int, count: int) -> list:
    """The first ``count`` outputs of a SplitMix64 generator seeded with ``seed``."""
    return [splitmix64((seed + (k + 1) * _GOLDEN_GAMMA) & _MASK64) for k in range(count)]


def choice_bit(seed: int, k: int) -> int:
    """Coin of the random choice of Algorithm 2 at ASDSM sweep k: the top bit of output k."""
    return splitmix64((seed + (k + 1) * _GOLDEN_GAMMA) & _MASK64) >> 63


# ---------------------------------------------------------------------------
# Section 2.1: meshes.
# ---------------------------------------------------------------------------
class Meshes2D:
    """Meshes of eq. (2.3) for N points per side (R1) and mc coarse intervals.

    Every mesh is an integer array of its points (i, j) in fine-grid indices
    (x = i h, y = j h), listed x fastest (R2)."""

    def __init__(self, N: int, mc: int):
        M = N - 1
        if N < 3 or mc < 2 or M % mc != 0:
            raise ValueError("eq. (2.1) needs (N-1) % mc == 0 with mc >= 2")
        self.N, self.M, self.mc = N, M, mc
        self.n = M // mc                 # fine intervals per coarse interval
        self.Nf = M - 1                  # fine interior points per axis
        self.Nc = mc - 1                 # coarse interior points per axis
        self.h = 1.0 / M
        self.H = 1.0 / mc
        fine = np.arange(1, M)
        coarse = np.arange(1, mc) * self.n
        self.ff = self._product(fine, fine)         # Omega^{h,h}
        self.fc = self._product(fine, coarse)       # Omega^{h,H}: fine in x, coarse in y
        self.cf = self._product(coarse, fine)       # Omega^{H,h}
        self.cc = self._product(coarse, coarse)     # Omega^{H,H}
        in_hole = (self.ff[:, 0] % self.n != 0) & (self.ff[:, 1] % self.n != 0)
        self.holes = self.ff[in_hole]               # union of the holes Omega_{i,j}
        self.skeleton = self.ff[~in_hole]           # Omega^{h,H} U Omega^{H,h}

    @staticmethod
    def _product(xs, ys):
        I, J = np.meshgrid(xs, ys)                  # J varies slowest: x fastest
        return np.stack([I.ravel(), J.ravel()], axis=1)

    def hole_of(self, points):
        """Index (bi, bj) of the hole Omega_{bi,bj} containing each point."""
        return points[:, 0] // self.n, points[:, 1] // self.n


# ---------------------------------------------------------------------------
# Definition 2.2: projectors as explicit 0/1 matrices.
# ---------------------------------------------------------------------------
def projector(rows_mesh, cols_mesh, N: int) -> sp.csr_matrix:
    """P with P[m, q] = 1 iff point m of rows_mesh equals point q of cols_mesh."""
    where = np.full(N * N, -1, dtype=np.int64)
    where[cols_mesh[:, 1] * N + cols_mesh[:, 0]] = np.arange(len(cols_mesh))
    c = where[rows_mesh[:, 1] * N + rows_mesh[:, 0]]
    if np.any(c < 0):
        raise ValueError("rows_mesh is not a subset of cols_mesh")
    r = np.arange(len(rows_mesh))
    return sp.csr_matrix((np.ones(len(r)), (r, c)), shape=(len(rows_mesh), len(cols_mesh)))


# ---------------------------------------------------------------------------
# Section 2.3: discretisation.
# ---------------------------------------------------------------------------
def L_matrix(n: int) -> sp.csr_matrix:
    return sp.diags([-np.ones(n - 1), 2.0 * np.ones(n), -np.ones(n - 1)], [-1, 0, 1], format="csr")


def D_matrix(n: int) -> sp.csr_matrix:
    return sp.diags([-np.ones(n - 1), np.ones(n - 1)], [-1, 1], format="csr")


def operator_2d(nx: int, hx: float, ny: int, hy: float, alpha, beta) -> sp.csr_matrix:
    """A = a_x I(x)L/hx^2 + a_y L/hy^2(x)I + b_x I(x)D/(2hx) + b_y D/(2hy)(x)I (x fastest, R3)."""
    ax, ay = alpha
    bx, by = beta
    Ix, Iy = sp.identity(nx, format="csr"), sp.identity(ny, format="csr")
    A = (ax * sp.kron(Iy, L_matrix(nx) / hx**2) + ay * sp.kron(L_matrix(ny) / hy**2, Ix)
         + bx * sp.kron(Iy, D_matrix(nx) / (2 * hx)) + by * sp.kron(D_matrix(ny) / (2 * hy), Ix))
    return A.tocsr()


def rhs_on_mesh(points, hx: float, hy: float, alpha, beta, s_grid, g_grid, M: int) -> np.ndarray:
    """b on a uniform (sub)mesh: samples of s plus the Dirichlet lifting (R5).

    points are fine-grid indices (i, j); the mesh spacing is hx, hy, so a
    point's neighbours sit hx*M and hy*M fine indices away.  A neighbour on
    the boundary moves its stencil coefficient times g to the right side."""
    ax, ay = alpha
    bx, by = beta
    sx, sy = int(round(hx * M)), int(round(hy * M))
    cw, ce = ax / hx**2 + bx / (2 * hx), ax / hx**2 - bx / (2 * hx)
    cs, cn = ay / hy**2 + by / (2 * hy), ay / hy**2 - by / (2 * hy)
    i, j = points[:, 0], points[:, 1]
    b = np.array(s_grid[j, i], dtype=np.float64)
    b += np.where(i - sx == 0, cw * g_grid[j, 0], 0.0)
    b += np.where(i + sx == M, ce * g_grid[j, M], 0.0)
    b += np.where(j - sy == 0, cs * g_grid[0, i], 0.0)
    b += np.where(j + sy == M, cn * g_grid[M, i], 0.0)
    return b


class Discretisation2D:
    """Linear systems of eq. (2.4) and the algorithms of Section 3 for one problem."""

    def __init__(self, N: int, mc: int, alpha, beta):
        self.m = Meshes2D(N, mc)
        m = self.m
        self.alpha, self.beta = tuple(float(a) for a in alpha), tuple(float(b) for b in beta)
        if min(self.alpha) <= 0:
            raise ValueError("alpha_i must be positive (eq. (1.1))")
        h, H, Nf, Nc = m.h, m.H, m.Nf, m.Nc
        self.A_ff = operator_2d(Nf, h, Nf, h, self.alpha, self.beta)
        self.A_fc = operator_2d(Nf, h, Nc, H, self.alpha, self.beta)
        self.A_cf = operator_2d(Nc, H, Nf, h, self.alpha, self.beta)
        self.A_cc = operator_2d(Nc, H, Nc, H, self.alpha, self.beta)
        # Definition 2.2 projectors (their transposes map back).
        self.P_ff_fc = projector(m.fc, m.ff, N)
        self.P_ff_cf = projector(m.cf, m.ff, N)
        self.P_ff_cc = projector(m.cc, m.ff, N)
        self.P_ff_holes = projector(m.holes, m.ff, N)
        self.P_fc_cc = projector(m.cc, m.fc, N)
        self.P_cf_cc = projector(m.cc, m.cf, N)
        self.P_ff_skel = projector(m.skeleton, m.ff, N)
        # Factorisations, each computed once (library primitive).
        self.lu_fc = spla.splu(self.A_fc.tocsc())
        self.lu_cf = spla.splu(self.A_cf.tocsc())
        self.lu_cc = spla.splu(self.A_cc.tocsc())
        A_holes = (self.P_ff_holes @ self.A_ff @ self.P_ff_holes.T).tocsc()
        self.lu_holes = spla.splu(A_holes)
        self._lu_ff = None
        self.knots = np.linspace(0.0, 1.0, m.mc + 1)
        self.fine_x = np.arange(1, m.M) * h

    # -- right-hand sides ---------------------------------------------------
    def rhs(self, s_grid, g_grid):
        """b_ff, b_fc, b_cf, b_cc (R5)."""
        m = self.m
        h, H, M = m.h, m.H, m.M
        a, be = self.alpha, self.beta
        return (rhs_on_mesh(m.ff, h, h, a, be, s_grid, g_grid, M),
                rhs_on_mesh(m.fc, h, H, a, be, s_grid, g_grid, M),
                rhs_on_mesh(m.cf, H, h, a, be, s_grid, g_grid, M),
                rhs_on_mesh(m.cc, H, H, a, be, s_grid, g_grid, M))

    def solve_fine(self, b_ff):
        """u_ff = (A_ff)^{-1} b_ff, the discrete solution ASDSM converges to."""
        if self._lu_ff is None:
            self._lu_ff = spla.splu(self.A_ff.tocsc())
        return self._lu_ff.solve(b_ff)

    # -- Section 3.1, Algorithm 2: one skeleton from the two anisotropic solutions
    def spline_fc(self, e_cc):
        """Spline(e, Omega^{h,H}): along x on every coarse line (R10)."""
        m = self.m
        E = e_cc.reshape(m.Nc, m.Nc)                 # [line j][knot i]
        vals = np.zeros((m.Nc, m.mc + 1))
        vals[:, 1:-1] = E
        out = CubicSpline(self.knots, vals, axis=1, bc_type="not-a-knot")(self.fine_x)
        return out.reshape(-1)                       # [line j][fine x], x fastest

    def spline_cf(self, e_cc):
        """Spline(e, Omega^{H,h}): along y on every coarse column (R10)."""
        m = self.m
        E = e_cc.reshape(m.Nc, m.Nc)                 # [knot j][column i]
        vals = np.zeros((m.mc + 1, m.Nc))
        vals[1:-1, :] = E
        out = CubicSpline(self.knots, vals, axis=0, bc_type="not-a-knot")(self.fine_x)
        return out.reshape(-1)                       # [fine y][column i], x fastest

    def skeleton(self, u_fc, u_cf, u_cc=None, choice=0):
        """Algorithm 2 (Skeleton Builder) as one map from (u_fc, u_cf) to a fine grid.

        Both families sample the coarse mesh Omega^{H,H}.  Their common value
        there, u_hat, is the extrapolated combination of R7 when u_cc is given,
        otherwise the samples of the family the coin picked (R8).  Each family
        is then moved onto u_hat at the coarse points by adding the spline
        (R10) of its mismatch along its fine axis; the two corrected families
        now agree at the cross points, and together they cover the skeleton
        Omega^{h,H} U Omega^{H,h}, holes left at zero (R11)."""
        at_cc = (self.P_fc_cc @ u_fc, self.P_cf_cc @ u_cf)
        u_hat = at_cc[choice] if u_cc is None else extrapolate_knots(at_cc[0], at_cc[1], u_cc)
        fc = u_fc + self.spline_fc(u_hat - at_cc[0])
        cf = u_cf + self.spline_cf(u_hat - at_cc[1])
        # Cross points belong to both families; they are written once, from fc.
        cf_without_cross = cf - self.P_cf_cc.T @ (self.P_cf_cc @ cf)
        return self.P_ff_fc.T @ fc + self.P_ff_cf.T @ cf_without_cross

    # -- Section 3.1, Algorithm 3: independent hole solves -------------------
    def filler(self, u_t, b_ff):
        """Algorithm 3 (Filler): every hole of Remark 2.4 solved with Dirichlet
        data from the skeleton of u_t.  Since A_ff restricted to the holes is the
        block-diagonal A_hh, the hole values are corrected by
            u_holes += A_hh^{-1} P_holes (b_ff - A_ff u_t),
        which makes the residual vanish at every hole point (Prop. 3.1)."""
        v = self.lu_holes.solve(self.P_ff_holes @ (b_ff - self.A_ff @ u_t))
        return u_t + self.P_ff_holes.T @ v

    # -- Section 3.1, Algorithm 1 ----------------------------------------------
    def initial_guess(self, b_ff, b_fc, b_cf, b_cc=None, choice=0):
        """Algorithm 1 (Initial Guess Builder): the anisotropic systems of
        eq. (2.4) solved exactly, merged by Algorithm 2 and completed by
        Algorithm 3.  With b_cc (the first iterate) the coarse system is solved
        too and the merge extrapolates; without it (the correction of a sweep)
        the two solutions are normalised per family (R9) and merged by the coin."""
        u_fc = self.lu_fc.solve(b_fc)
        u_cf = self.lu_cf.solve(b_cf)
        if b_cc is None:
            u_fc, u_cf = normalised_families(u_fc, u_cf)
            u_t = self.skeleton(u_fc, u_cf, None, choice)
        else:
            u_t = self.skeleton(u_fc, u_cf, self.lu_cc.solve(b_cc))
        return self.filler(u_t, b_ff)

    def correction(self, r, choice, smoothing=None):
        """The ASDSM correction of a sweep (Section 3.2): Algorithm 1 applied to
        the error equations, i.e. right-hand sides P_fc r and P_cf r on the two
        anisotropic meshes, zero boundary data and zero source in the holes;
        with `smoothing` the projections are smoothed first (R27)."""
        r_fc, r_cf = self.P_ff_fc @ r, self.P_ff_cf @ r
        if smoothing is not None:
            r_fc, r_cf = smooth_projections(self.m, r_fc, r_cf, smoothing)
        return self.initial_guess(np.zeros_like(r), r_fc, r_cf, None, choice)

    def residual(self, b_ff, u):
        return b_ff - self.A_ff @ u


def smooth_projections(m: Meshes2D, r_fc, r_cf, mode: str):
    """R27: the projected residuals smoothed along each line's fine axis.

    r_fc lists Omega^{h,H} x fastest (one row per coarse line y = jH), r_cf
    lists Omega^{H,h} x fastest (one row per fine y), so the fine axis is the
    second axis of the first and the first axis of the second."""
    F = np.array(r_fc, dtype=np.float64).reshape(m.Nc, m.Nf)
    C = np.array(r_cf, dtype=np.float64).reshape(m.Nf, m.Nc).T      # one row per coarse column x = iH
    out = []
    for V in (F, C):
        P = np.pad(V, ((0, 0), (1, 1)))                              # zero beyond the boundary
        if mode == "knots":
            W = V.copy()
            cross = np.arange(1, m.mc) * m.n - 1                     # positions of x = kH on the fine axis
            W[:, cross] = 0.5 * (P[:, cross] + P[:, cross + 2])
        elif mode == "lines":
            W = 0.25 * P[:, :-2] + 0.5 * V + 0.25 * P[:, 2:]
        else:
            raise ValueError(f"unknown smoothing {mode!r}")
        out.append(W)
    return out[0].reshape(-1), out[1].T.reshape(-1)


def extrapolate_knots(fc, cf, cc, f2=None, c2=None):
    """u_hat at the coarse points: R7 from the samples of u_fc, u_cf and u_cc,
    or R28 when the samples f2, c2 of the Omega^{2h,H}, Omega^{H,2h} solutions
    are given too."""
    if f2 is None:
        return fc + cf - cc
    return (4.0 * fc - f2) / 3.0 + (4.0 * cf - c2) / 3.0 - cc


def normalised_families(u_fc, u_cf):
    """R9: each anisotropic solution divided by its own Euclidean norm (a zero
    vector stays zero), so that neither family dominates the merge by size."""
    out = []
    for v in (u_fc, u_cf):
        nv = np.linalg.norm(v)
        out.append(v / nv if nv > 0 else v)
    return out[0], out[1]


def hole_fix_due(hole_norm, r_norm, hole_ref, ratio, growth):
    """R18: rounding has left a hole residual worth a Filler pass when it is
    both a sizeable part of the whole residual (ratio) and has grown past
    `growth` times its size right after the previous pass (0 before any)."""
    return hole_norm > ratio * r_norm and hole_norm > growth * hole_ref


def stagnated(hist, window, factor):
    """R13: the residual of the last `window` sweeps fell by less than `factor`."""
    return len(hist) > window and hist[-1] > (1 - factor) * hist[-1 - window]


def asdsm(disc: Discretisation2D, b, *, tol=1e-10, max_sweeps=200, accel_m=1, seed=0,
          hole_fix_ratio=0.25, hole_fix_growth=4.0, stagnation_window=10,
          stagnation_factor=1e-3,
          u0=None, record_iterates=False, smoothing=None):
    """Algorithm 4 (ASDSM) with the readings R13-R15 and R18.

    The iterate starts from Algorithm 1 (or u0).  Each sweep takes the fine
    residual r = b_ff - A_ff u, builds the correction e from it (Section 3.2)
    and moves u along e by a least-squares step on the skeleton rows, where
    A e can be non-zero (Prop. 3.1): the clamped optimal scaling s_hat >= 0 of
    Section 3.2 when accel_m = 1, restarted GCR(accel_m) otherwise (R15);
    `smoothing` selects a reading of R27 for the projected residuals.

    b = (b_ff, b_fc, b_cf, b_cc).  Returns (u, info); info holds the relative
    residual history (entry k is the residual of iterate k), the choice bits,
    the step lengths, what each sweep did and why the loop stopped."""
    b_ff, b_fc, b_cf, b_cc = b
    sk = disc.P_ff_skel
    u = disc.initial_guess(b_ff, b_fc, b_cf, b_cc) if u0 is None else np.array(u0, dtype=np.float64)
    nb = np.linalg.norm(b_ff)
    hist, steps, bits, kinds, iterates = [], [], [], [], []
    Z, Q = [], []                    # GCR cycle: directions and their A-images on the skeleton
    hole_ref = 0.0                   # hole residual norm right after the last Filler pass (R18)
    status = "max_sweeps"
    k = 0
    while True:
        r = disc.residual(b_ff, u)
        rel = np.linalg.norm(r) / nb if nb > 0 else np.linalg.norm(r)
        hist.append(rel)
        if record_iterates:
            iterates.append(u.copy())
        if rel <= tol:
            status = "converged"
            break
        if k >= max_sweeps:
            break
        if stagnated(hist, stagnation_window, stagnation_factor):
            status = "stagnated"
            break
        if hole_fix_due(np.linalg.norm(disc.P_ff_holes @ r), np.linalg.norm(r), hole_ref,
                        hole_fix_ratio, hole_fix_growth):
            u = disc.filler(u, b_ff)
            hole_ref = np.linalg.norm(disc.P_ff_holes @ disc.residual(b_ff, u))
            Z, Q = [], []
            kinds.append("hole_fix")
            bits.append(-1)
            steps.append(1.0)
            k += 1
            continue
        bit = choice_bit(seed, k)
        e = disc.correction(r, bit, smoothing)
        q = sk @ (disc.A_ff @ e)     # A e on the skeleton rows
        rs = sk @ r
        if accel_m == 1:
            qq = q @ q
            s_hat = max(0.0, (rs @ q) / qq) if qq > 0 else 0.0     # R14
            u = u + s_hat * e
            steps.append(s_hat)
        else:
            # R15: orthogonalise A e against the cycle's earlier images, then the
            # least-squares coefficient along the new unit image.
            for zj, qj in zip(Z, Q):
                beta_j = q @ qj
                q = q - beta_j * qj
                e = e - beta_j * zj
            nq = np.linalg.norm(q)
            if nq > 0:
                q = q / nq
                e = e / nq
                a = rs @ q
                u = u + a * e
                Z.append(e)
                Q.append(q)
                steps.append(a)
            else:
                steps.append(0.0)
            if len(Z) >= accel_m:
                Z, Q = [], []
        kinds.append("sweep")
        bits.append(bit)
        k += 1
    info = {"hist": hist, "steps": steps, "bits": bits, "kinds": kinds,
            "status": status, "sweeps": k}
    if record_iterates:
        info["iterates"] = iterates
    return u, info


# ---------------------------------------------------------------------------
# Convenience wrappers on full-grid arrays ([y, x], boundary included).
# ---------------------------------------------------------------------------
def interior(grid2d):
    return np.asarray(grid2d)[1:-1, 1:-1].reshape(-1)


def to_grid(u_ff, g_grid):
    out = np.array(g_grid, dtype=np.float64, copy=True)
    n = out.shape[0] - 2
    out[1:-1, 1:-1] = u_ff.reshape(n, n)
    return out


def solve_problem(N, mc, alpha, beta, s_grid, g_grid, **kw):
    """ASDSM on full-grid inputs; returns the full grid (boundary = g), info, disc, b."""
    disc = Discretisation2D(N, mc, alpha, beta)
    b = disc.rhs(s_grid, g_grid)
    u, info = asdsm(disc, b, **kw)
    return to_grid(u, g_grid), info, disc, b


def fine_system(N, alpha, beta, s_grid, g_grid):
    """A_ff and b_ff of the fine uniform mesh alone (no coarse mesh needed)."""
    M = N - 1
    h = 1.0 / M
    fine = np.arange(1, M)
    pts = Meshes2D._product(fine, fine)
    A = operator_2d(M - 1, h, M - 1, h, alpha, beta)
    b = rhs_on_mesh(pts, h, h, alpha, beta, s_grid, g_grid, M)
    return A, b


def residual_grid(N, alpha, beta, s_grid, u_grid):
    """r = b_ff - A_ff u on the interior, from the full grid u (its boundary is g)."""
    A, b = fine_system(N, alpha, beta, s_grid, u_grid)
    return b - A @ interior(u_grid), b
