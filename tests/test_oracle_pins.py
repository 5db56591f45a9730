"""Pins of the FP64 CPU oracle against facts fixed by the paper and by mathematics.

Each test names the passage it checks.  None of them re-types the formula it
checks: they compare against brute force, closed forms, exactness properties,
published reference values or the paper's propositions.  Several tests plant a
mistake in the oracle (monkeypatched, on the CPU) and check a pin catches it.
"""
import os

import numpy as np
import pytest

from oracle import asdsm2d as o
from paper_2303_01163_gb300 import workloads as w

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------------------
# Counter-based generator (reading R8): published SplitMix64 outputs.
# ---------------------------------------------------------------------------
def _golden_splitmix():
    out = {}
    with open(os.path.join(HERE, "golden", "splitmix64.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            seed, vals = line.split(":")
            out[int(seed)] = [int(v) for v in vals.split()]
    return out


def test_splitmix64_matches_published_outputs():
    for seed, vals in _golden_splitmix().items():
        assert o.splitmix64_stream(seed, len(vals)) == vals


def test_choice_bits_are_balanced_and_seeded():
    bits = [o.choice_bit(7, k) for k in range(4000)]
    assert 0.45 < np.mean(bits) < 0.55
    assert bits != [o.choice_bit(8, k) for k in range(4000)]


# ---------------------------------------------------------------------------
# Section 2.3: the operator against a brute-force stencil assembly.
# ---------------------------------------------------------------------------
def _brute_force_operator(nx, hx, ny, hy, alpha, beta):
    """Dense matrix assembled point by point from the centred differences of
    -a u'' + b u' on each axis (independent of the Kronecker construction)."""
    ax, ay = alpha
    bx, by = beta
    n = nx * ny
    A = np.zeros((n, n))
    for j in range(ny):
        for i in range(nx):
            row = j * nx + i
            A[row, row] = 2 * ax / hx**2 + 2 * ay / hy**2
            for di, dj, coef in ((-1, 0, -ax / hx**2 - bx / (2 * hx)),
                                 (1, 0, -ax / hx**2 + bx / (2 * hx)),
                                 (0, -1, -ay / hy**2 - by / (2 * hy)),
                                 (0, 1, -ay / hy**2 + by / (2 * hy))):
                ii, jj = i + di, j + dj
                if 0 <= ii < nx and 0 <= jj < ny:
                    A[row, jj * nx + ii] = coef
    return A


@pytest.mark.parametrize("dims", [(5, 5), (7, 3), (3, 9)])
def test_operator_matches_brute_force(dims):
    nx, ny = dims
    alpha, beta = (0.7, 1.9), (-3.0, 5.5)
    A = o.operator_2d(nx, 1 / (nx + 1), ny, 0.25, alpha, beta).toarray()
    B = _brute_force_operator(nx, 1 / (nx + 1), ny, 0.25, alpha, beta)
    np.testing.assert_allclose(A, B, rtol=1e-14, atol=0)


def test_quadratic_solution_has_zero_residual_on_every_mesh():
    """Centred differences are exact for u = p(x) q(y) with quadratic p, q, so
    the sampled exact solution solves every system of eq. (2.4), including the
    Dirichlet lifting (R5).  A wrong sign, spacing or axis fails this."""
    N, mc = 25, 4
    prob = w.polynomial_2d(N, alpha=(0.8, 1.7), beta=(2.5, -4.0))
    disc = o.Discretisation2D(N, mc, prob.alpha, prob.beta)
    b_ff, b_fc, b_cf, b_cc = disc.rhs(prob.s, prob.g)
    m = disc.m
    ue = prob.u_exact
    for A, mesh, bb in ((disc.A_ff, m.ff, b_ff), (disc.A_fc, m.fc, b_fc),
                        (disc.A_cf, m.cf, b_cf), (disc.A_cc, m.cc, b_cc)):
        u = ue[mesh[:, 1], mesh[:, 0]]
        r = bb - A @ u
        assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(bb)


def test_closed_form_discrete_poisson_eigenfunction():
    """beta = 0, s = sin(k pi x) sin(l pi y), g = 0: the discrete solution is
    s / (a_x lam_k + a_y lam_l) with lam_k = 4/h^2 sin^2(k pi h / 2)."""
    N = 33
    h = 1.0 / (N - 1)
    x = np.linspace(0, 1, N)
    k, l = 3, 5
    S = np.outer(np.sin(l * np.pi * x), np.sin(k * np.pi * x))
    alpha = (0.6, 1.3)
    lam = lambda q: 4 / h**2 * np.sin(q * np.pi * h / 2) ** 2
    A, b = o.fine_system(N, alpha, (0.0, 0.0), S, np.zeros((N, N)))
    import scipy.sparse.linalg as spla
    u = spla.spsolve(A.tocsc(), b)
    expect = o.interior(S) / (alpha[0] * lam(k) + alpha[1] * lam(l))
    np.testing.assert_allclose(u, expect, rtol=1e-11, atol=1e-14)


def test_second_order_convergence():
    """The fine discrete solution converges as O(h^2) to the smooth solution."""
    errs = []
    for N in (17, 33, 65, 129):
        p = w.manufactured_sine_2d(N, alpha=(1.0, 0.5), beta=(2.0, -1.0))
        A, b = o.fine_system(N, p.alpha, p.beta, p.s, p.g)
        import scipy.sparse.linalg as spla
        u = spla.spsolve(A.tocsc(), b)
        errs.append(np.abs(u - o.interior(p.u_exact)).max())
    ratios = [errs[i] / errs[i + 1] for i in range(len(errs) - 1)]
    assert all(3.8 < r < 4.2 for r in ratios[1:]), ratios


# ---------------------------------------------------------------------------
# Section 2.1-2.2: mesh relations and projector properties.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,mc", [(9, 2), (17, 4), (33, 8), (25, 3)])
def test_prop_2_1_mesh_relations(N, mc):
    m = o.Meshes2D(N, mc)
    ff = {tuple(p) for p in m.ff}
    fc = {tuple(p) for p in m.fc}
    cf = {tuple(p) for p in m.cf}
    cc = {tuple(p) for p in m.cc}
    holes = {tuple(p) for p in m.holes}
    assert fc <= ff and cf <= ff                       # a)
    assert cc <= ff and cc <= cf and cc <= fc          # b)
    assert holes == ff - (fc | cf)                     # d)
    bi, bj = m.hole_of(m.holes)                        # c): every hole has (n-1)^2 points
    counts = np.bincount(bj * m.mc + bi, minlength=m.mc * m.mc)
    assert np.all(counts == (m.n - 1) ** 2)
    assert len(holes) == m.mc ** 2 * (m.n - 1) ** 2
    assert len(fc | cf) == 2 * m.Nc * m.Nf - m.Nc ** 2


def test_prop_2_3_projectors_are_partial_identities():
    disc = o.Discretisation2D(33, 4, (1.0, 1.0), (0.0, 0.0))
    for P in (disc.P_ff_fc, disc.P_ff_cf, disc.P_ff_cc, disc.P_ff_holes, disc.P_fc_cc, disc.P_cf_cc):
        I = (P @ P.T).toarray()
        np.testing.assert_array_equal(I, np.eye(P.shape[0]))
        assert abs(P).sum(axis=1).max() == 1 and abs(P).sum(axis=0).max() == 1


def test_remark_2_4_hole_blocks_are_diagonal_sub_blocks():
    """P A P^T splits into identical blocks, each the operator of one hole."""
    N, mc = 17, 2
    disc = o.Discretisation2D(N, mc, (0.9, 1.4), (3.0, -2.0))
    m = disc.m
    Ah = (disc.P_ff_holes @ disc.A_ff @ disc.P_ff_holes.T).toarray()
    bi, bj = m.hole_of(m.holes)
    hid = bj * m.mc + bi
    assert np.all(Ah[hid[:, None] != hid[None, :]] == 0)
    block = o.operator_2d(m.n - 1, m.h, m.n - 1, m.h, disc.alpha, disc.beta).toarray()
    for h in range(m.mc * m.mc):
        sel = np.flatnonzero(hid == h)
        np.testing.assert_allclose(Ah[np.ix_(sel, sel)], block, rtol=1e-15)


# ---------------------------------------------------------------------------
# Algorithm 2: the spline of reading R10.
# ---------------------------------------------------------------------------
def test_spline_reproduces_cubics_vanishing_at_the_boundary():
    """A not-a-knot cubic spline reproduces any cubic, so knot values of
    c(x) = x (1 - x) (a + b x) interpolate back to c on every fine point."""
    N, mc = 49, 6
    disc = o.Discretisation2D(N, mc, (1.0, 1.0), (0.0, 0.0))
    m = disc.m
    knots = np.arange(1, mc) * m.H
    rng = np.random.default_rng(3)
    coef = rng.normal(size=(m.Nc, 2))                    # one cubic per coarse line
    cub = lambda t, c: t * (1 - t) * (c[0] + c[1] * t)
    E = np.array([[cub(t, coef[j]) for t in knots] for j in range(m.Nc)])    # [line][knot]
    out = disc.spline_fc(E.reshape(-1)).reshape(m.Nc, m.Nf)
    fine = np.arange(1, m.M) * m.h
    expect = np.array([cub(fine, coef[j]) for j in range(m.Nc)])
    np.testing.assert_allclose(out, expect, atol=1e-13)
    out2 = disc.spline_cf(E.T.reshape(-1)).reshape(m.Nf, m.Nc)
    np.testing.assert_allclose(out2, expect.T, atol=1e-13)


def test_spline_with_one_coarse_point_is_the_parabola():
    disc = o.Discretisation2D(9, 2, (1.0, 1.0), (0.0, 0.0))
    out = disc.spline_fc(np.array([1.0]))
    t = np.arange(1, 8) / 8
    np.testing.assert_allclose(out, 4 * t * (1 - t), atol=1e-14)


# ---------------------------------------------------------------------------
# Algorithms 1-3 and Proposition 3.1.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N,mc", [(25, 4), (33, 8), (37, 6)])
def test_initial_guess_is_exact_for_quadratic_solutions(N, mc):
    """With u = p(x) q(y) every submesh solution is exact, RE and the spline
    see no error and Algorithm 1 returns u_ff: this pins lifting on every mesh,
    the RE combination, the merge and the Filler together."""
    prob = w.polynomial_2d(N, alpha=(0.8, 1.7), beta=(2.5, -4.0))
    disc = o.Discretisation2D(N, mc, prob.alpha, prob.beta)
    b = disc.rhs(prob.s, prob.g)
    u0 = disc.initial_guess(*b)
    np.testing.assert_allclose(u0, o.interior(prob.u_exact), rtol=0, atol=1e-11)


def test_prop_3_1_1_filler_of_the_exact_skeleton_is_exact():
    p = w.random_fourier_2d(65, 5)
    disc = o.Discretisation2D(65, 4, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    uff = disc.solve_fine(b[0])
    skel_only = disc.P_ff_skel.T @ (disc.P_ff_skel @ uff)
    out = disc.filler(skel_only, b[0])
    assert np.abs(out - uff).max() <= 1e-12 * np.abs(uff).max()


@pytest.mark.parametrize("m", [1, 4])
def test_prop_3_1_2_residual_vanishes_in_the_holes_every_iterate(m):
    p = w.manufactured_shifted_sine_2d(65, alpha=(1.0, 1.0), beta=(1.0, 1.0), k=1.0)
    disc = o.Discretisation2D(65, 8, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    u, info = o.asdsm(disc, b, tol=1e-14, max_sweeps=12, accel_m=m, record_iterates=True,
                      stagnation_window=1000)
    nb = np.linalg.norm(b[0])
    for it in info["iterates"]:
        r = disc.residual(b[0], it)
        assert np.abs(disc.P_ff_holes @ r).max() <= 1e-12 * nb
        assert np.abs(disc.P_ff_skel @ r).max() > 0


def test_paper_step_6_never_increases_the_residual():
    """Remark after Algorithm 4: the scaling cannot make ASDSM diverge."""
    p = w.random_fourier_2d(65, 2)
    disc = o.Discretisation2D(65, 8, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    _, info = o.asdsm(disc, b, tol=1e-14, max_sweeps=25, accel_m=1, stagnation_window=1000)
    h = np.array(info["hist"])
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-12))


def test_fixed_point_is_the_fine_solution():
    """ASDSM started at u_ff stops at once: its residual is already at rounding level."""
    p = w.manufactured_sine_2d(33)
    disc = o.Discretisation2D(33, 4, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    uff = disc.solve_fine(b[0])
    u, info = o.asdsm(disc, b, tol=1e-13, u0=uff, max_sweeps=5)
    assert info["status"] == "converged" and info["sweeps"] == 0


def test_asdsm_converges_to_the_dense_brute_force_solution():
    """Tiny grid: GCR-refined ASDSM reaches the solution of the dense system
    assembled point by point (independent of every sparse construction)."""
    N, mc = 17, 4
    p = w.random_fourier_2d(N, 11, kmax=4)
    disc = o.Discretisation2D(N, mc, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    u, info = o.asdsm(disc, b, tol=1e-13, max_sweeps=400, accel_m=8)
    assert info["status"] == "converged"
    m = disc.m
    A = _brute_force_operator(m.Nf, m.h, m.Nf, m.h, p.alpha, p.beta)
    ue = np.linalg.solve(A, b[0])
    assert np.abs(u - ue).max() <= 1e-10 * np.abs(ue).max()


# ---------------------------------------------------------------------------
# Section 4 qualitative statements (Example 1, setting 1).
# ---------------------------------------------------------------------------
def test_richardson_initial_guess_beats_random_choice_and_first_sweep_drops():
    p = w.manufactured_shifted_sine_2d(129, k=1.0)
    disc = o.Discretisation2D(129, 8, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    nb = np.linalg.norm(b[0])
    with_re = disc.initial_guess(*b)
    no_re = disc.initial_guess(b[0], b[1], b[2], None, 0)    # normalised + chosen, no b_cc
    r_re = np.linalg.norm(disc.residual(b[0], with_re)) / nb
    r_no = np.linalg.norm(disc.residual(b[0], no_re)) / nb
    assert r_re < 1e-2 * r_no
    _, info = o.asdsm(disc, b, tol=1e-14, max_sweeps=3, accel_m=1, stagnation_window=1000)
    assert info["hist"][1] < 0.5 * info["hist"][0]


# ---------------------------------------------------------------------------
# Planted mistakes (on the CPU, in the oracle): the pins above catch them.
# ---------------------------------------------------------------------------
def test_planted_wrong_richardson_sign_is_caught(monkeypatch):
    prob = w.polynomial_2d(25, alpha=(0.8, 1.7), beta=(2.5, -4.0))
    disc = o.Discretisation2D(25, 4, prob.alpha, prob.beta)
    b = disc.rhs(prob.s, prob.g)
    orig = o.Discretisation2D.skeleton

    def bad(self, u_fc, u_cf, u_cc=None, choice=0):
        return orig(self, u_fc, u_cf, None if u_cc is None else -u_cc, choice)
    monkeypatch.setattr(o.Discretisation2D, "skeleton", bad)
    u0 = disc.initial_guess(*b)
    assert np.abs(u0 - o.interior(prob.u_exact)).max() > 1e-3


def test_planted_transposed_advection_is_caught(monkeypatch):
    orig = o.D_matrix
    monkeypatch.setattr(o, "D_matrix", lambda n: orig(n).T)
    prob = w.polynomial_2d(25, alpha=(0.8, 1.7), beta=(2.5, -4.0))
    disc = o.Discretisation2D(25, 4, prob.alpha, prob.beta)
    b_ff = disc.rhs(prob.s, prob.g)[0]
    u = o.interior(prob.u_exact)
    assert np.linalg.norm(b_ff - disc.A_ff @ u) > 1e-3 * np.linalg.norm(b_ff)


def test_planted_spline_knot_shift_is_caught(monkeypatch):
    disc = o.Discretisation2D(49, 6, (1.0, 1.0), (0.0, 0.0))
    disc.fine_x = disc.fine_x + disc.m.h          # evaluate one fine point off
    m = disc.m
    knots = np.arange(1, m.mc) * m.H
    E = np.array([[t * (1 - t) for t in knots] for _ in range(m.Nc)])
    out = disc.spline_fc(E.reshape(-1)).reshape(m.Nc, m.Nf)
    fine = np.arange(1, m.M) * m.h
    assert np.abs(out - fine * (1 - fine)).max() > 1e-4
