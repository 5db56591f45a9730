"""Pins of the 3D oracle (oracle/asdsm3d.py) against what the paper and the
mathematics fix, independently of the oracle's own formulas:

* the 7-point operator on every mesh, by discrete eigenfunctions (closed-form
  eigenvalues with the mesh's own spacing per axis);
* Dirichlet lifting and operator signs, by linear fields (second differences
  vanish, centred first differences are exact);
* second-order accuracy of the fine solution of the manufactured problem;
* the combination weights of R21 and the Boolean-sum correction of R23: when
  every (sub)mesh solution samples the same function the merged skeleton
  reproduces it; the Boolean sum reproduces tensor-product cubics that vanish
  on the boundary on the whole plane, and any data on the plane's lines;
* the Filler (cube holes, six faces), by fields the discrete operator maps to a
  constant;
* the normalisation of each plane solution (R24), by the invariance of a
  sweep's correction under per-family scaling of the residual;
* Algorithm 4 in 3D: GCR(m) reaches 1e-10 and the direct fine solution; the
  paper's step (m = 1) never increases the skeleton residual.

Each pin fails for at least one plausible mistake in the oracle (a wrong
combination weight or line mesh, a dropped Boolean-sum term, the fine spacing
on a coarse axis, a lifting or first-difference sign, no normalisation, a
Filler sign, a transposed spline axis).
"""
import numpy as np
import pytest

from oracle import asdsm3d as o3
from paper_2303_01163_gb300 import workloads as wl


def _lam(k, h):
    return 4.0 / h**2 * np.sin(k * np.pi * h / 2) ** 2


def test_operator_eigenfunctions_on_fine_plane_and_line_meshes():
    disc = o3.Discretisation3D(17, 4, alpha=(0.7, 1.3, 0.4), beta=(0.0, 0.0, 0.0))
    m = disc.m
    kx, ky, kz = 2, 3, 1
    for name, A, pts, coarse_axes in [
        ("ff", disc.A_ff, m.ff, ()),
        ("plane x", disc.A_plane["x"], m.plane["x"], (0,)),
        ("plane z", disc.A_plane["z"], m.plane["z"], (2,)),
        ("line y", disc.A_line["y"], m.line["y"], (0, 2)),
        ("coarse", disc.A_cc, m.cc, (0, 1, 2)),
    ]:
        xyz = pts * m.h
        v = np.sin(kx * np.pi * xyz[:, 0]) * np.sin(ky * np.pi * xyz[:, 1]) * np.sin(kz * np.pi * xyz[:, 2])
        hs = [m.H if a in coarse_axes else m.h for a in range(3)]
        lam = sum(al * _lam(k, h) for al, k, h in zip(disc.alpha, (kx, ky, kz), hs))
        assert np.linalg.norm(A @ v - lam * v) <= 1e-12 * lam * np.linalg.norm(v), name


def test_lifting_and_signs_by_linear_fields():
    N, mc = 17, 4
    alpha, beta = (0.8, 1.7, 0.5), (2.5, -4.0, 1.5)
    disc = o3.Discretisation3D(N, mc, alpha, beta)
    x = np.linspace(0.0, 1.0, N)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    c = (0.3, -1.2, 2.0, 0.7)
    w = c[0] + c[1] * X + c[2] * Y + c[3] * Z
    s = np.full_like(w, beta[0] * c[1] + beta[1] * c[2] + beta[2] * c[3])   # -alpha Lap w + beta . grad w
    b_ff, b_p, b_l, b_c = disc.rhs(s, w)
    assert np.allclose(disc.solve_fine(b_ff), o3.interior(w), rtol=0, atol=1e-11)
    # every submesh's own system has the samples of w as its solution too (lifting with its spacing)
    for f in o3.FAMILIES:
        pts = disc.m.plane[f]
        want = w[pts[:, 2], pts[:, 1], pts[:, 0]]
        assert np.allclose(disc.lu_plane[f].solve(b_p[f]), want, rtol=0, atol=1e-11), f
        pts = disc.m.line[f]
        want = w[pts[:, 2], pts[:, 1], pts[:, 0]]
        assert np.allclose(disc.lu_line[f].solve(b_l[f]), want, rtol=0, atol=1e-11), f
    pts = disc.m.cc
    assert np.allclose(disc.lu_cc.solve(b_c), w[pts[:, 2], pts[:, 1], pts[:, 0]], rtol=0, atol=1e-11)


def test_fine_solution_is_second_order():
    alpha, beta = (1.0, 0.6, 1.4), (1.0, -2.0, 0.5)
    errs = []
    for N in (9, 17, 33):
        disc = o3.Discretisation3D(N, 2, alpha, beta)
        p = wl.manufactured_sine_3d(N, alpha, beta)
        u, s = p.u_exact, p.s
        b = disc.rhs(s, np.zeros_like(u))
        errs.append(np.max(np.abs(disc.solve_fine(b[0]) - o3.interior(u))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.5 < r1 < 4.5 and 3.7 < r2 < 4.3, errs


def test_merge_reproduces_a_common_field():
    """If planes, lines and coarse solutions all sample one function, R21's
    weights (3 - 3 + 1 at knots, 2 - 1 on lines) give it back, the errors vanish
    and the skeleton is that function on every plane point."""
    N, mc = 17, 4
    disc = o3.Discretisation3D(N, mc, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    x = np.linspace(0.0, 1.0, N)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    w = np.sin(2 * X) * np.cos(Y + 0.3) * (1 + Z ** 2)
    msk = disc._masks()
    U_plane = {f: np.where(msk[f], w, 0.0) for f in o3.FAMILIES}
    m = disc.m
    U_line = {f: disc.to_full(m.line[f], w[m.line[f][:, 2], m.line[f][:, 1], m.line[f][:, 0]]) for f in o3.FAMILIES}
    U_cc = disc.to_full(m.cc, w[m.cc[:, 2], m.cc[:, 1], m.cc[:, 0]])
    skel, _, _ = disc.skeleton(U_plane, U_line, U_cc)
    sk = disc.P_skel
    assert np.allclose(sk @ skel, sk @ o3.interior(w), rtol=0, atol=1e-13)
    for choice in (0, 1, 2):                     # random choice: equal plane values, nothing to correct
        skel, _, _ = disc.skeleton(U_plane, None, None, choice)
        assert np.allclose(sk @ skel, sk @ o3.interior(w), rtol=0, atol=1e-13)


def test_boolean_sum_reproduces_boundary_vanishing_cubics_and_line_data():
    N, mc = 33, 4
    disc = o3.Discretisation3D(N, mc, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    x = np.linspace(0.0, 1.0, N)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    p = lambda t: t * (1 - t) * (t - 0.3)          # cubic, zero at 0 and 1
    q = lambda t: t * (1 - t) * (t + 0.5)
    msk = disc._masks()
    cnt = msk["x"].astype(int) + msk["y"] + msk["z"]
    lines = cnt >= 2
    for f, e in (("x", p(Y) * q(Z) + 2 * q(Y) * p(Z)), ("y", p(X) * q(Z)), ("z", q(X) * p(Y) - p(X) * q(Y))):
        C = disc.plane_correction(f, np.where(lines & msk[f], e, 0.0))
        assert np.allclose(C[msk[f]], e[msk[f]], rtol=0, atol=1e-13), f
    rng = np.random.default_rng(1)
    R = rng.normal(size=(N, N, N))
    for f in o3.FAMILIES:
        C = disc.plane_correction(f, np.where(lines & msk[f], R, 0.0))
        sel = lines & msk[f]
        assert np.allclose(C[sel], R[sel], rtol=0, atol=1e-12), f


def test_filler_on_cube_holes_recovers_linear_fields():
    N, mc = 17, 4
    alpha, beta = (0.8, 1.7, 0.5), (2.5, -4.0, 1.5)
    disc = o3.Discretisation3D(N, mc, alpha, beta)
    x = np.linspace(0.0, 1.0, N)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    w = 1.0 + 0.5 * X - 2.0 * Y + 0.25 * Z
    s = np.full_like(w, 0.5 * beta[0] - 2.0 * beta[1] + 0.25 * beta[2])
    b_ff = disc.rhs(s, w)[0]
    u_t = o3.interior(w).copy()
    u_t[disc.P_holes.T @ np.ones(disc.P_holes.shape[0]) > 0] = 123.0       # garbage in the holes
    got = disc.filler(u_t, b_ff)
    assert np.allclose(got, o3.interior(w), rtol=0, atol=1e-11)


@pytest.mark.parametrize("N,mc", [(17, 4), (17, 2)])
def test_asdsm3d_gcr_reaches_the_fine_solution(N, mc):
    alpha, beta = (1.0, 0.5, 0.8), (1.5, -1.0, 0.5)
    disc = o3.Discretisation3D(N, mc, alpha, beta)
    p = wl.manufactured_sine_3d(N, alpha, beta)
    u_ex, s = p.u_exact, p.s
    b = disc.rhs(s, np.zeros_like(u_ex))
    u, info = o3.asdsm(disc, b, tol=1e-10, max_sweeps=300, accel_m=8)
    assert info["status"] == "converged", info["status"]
    assert info["hist"][-1] <= 1e-10
    uf = disc.solve_fine(b[0])
    assert np.linalg.norm(u - uf) / np.linalg.norm(uf) <= 1e-8


def test_asdsm3d_paper_step_never_increases_the_skeleton_residual():
    N, mc = 17, 4
    alpha, beta = (1.0, 0.5, 0.8), (1.5, -1.0, 0.5)
    disc = o3.Discretisation3D(N, mc, alpha, beta)
    p = wl.manufactured_sine_3d(N, alpha, beta)
    u_ex, s = p.u_exact, p.s
    b = disc.rhs(s, np.zeros_like(u_ex))
    u, info = o3.asdsm(disc, b, tol=1e-14, max_sweeps=12, accel_m=1, stagnation_window=10**9)
    h = np.array(info["hist"])
    assert np.all(np.array(info["steps"]) >= 0.0)
    # the step minimises the skeleton part of the residual, and the Filler keeps the hole part at rounding
    assert np.all(h[1:] <= h[:-1] * (1 + 1e-9)), h
    assert h[-1] < h[0]


def test_sweep_correction_is_invariant_to_per_family_scaling():
    """R24: each plane solution is normalised by its own norm before the merge,
    so scaling one family's right-hand side by a positive factor changes nothing."""
    N, mc = 17, 4
    disc = o3.Discretisation3D(N, mc, (1.0, 0.5, 0.8), (1.5, -1.0, 0.5))
    rng = np.random.default_rng(4)
    r = rng.normal(size=disc.m.Nf ** 3)
    r_p = {f: disc.P_plane[f] @ r for f in o3.FAMILIES}
    scaled = {f: c * r_p[f] for f, c in zip(o3.FAMILIES, (2.0, 5.0, 0.5))}
    zero = np.zeros_like(r)
    for choice in (0, 1, 2):
        e1 = disc.initial_guess(zero, r_p, None, None, choice)
        e2 = disc.initial_guess(zero, scaled, None, None, choice)
        assert np.allclose(e1, e2, rtol=0, atol=1e-12 * np.abs(e1).max())


def test_filler_pass_in_3d_removes_the_hole_residual_and_keeps_the_skeleton():
    """R18 in 3D: a start whose residual sits mostly in the cube holes gets a
    Filler pass first, which zeroes the hole residual (Prop. 3.1 on the cube
    holes) and leaves the skeleton as it was."""
    N, mc = 17, 4
    p = wl.random_sine_3d(N, 6)
    disc = o3.Discretisation3D(N, mc, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    u_ff = disc.solve_fine(b[0])
    u0 = u_ff + np.random.default_rng(3).normal(size=u_ff.size) * np.abs(u_ff).max()
    r0 = disc.residual(b[0], u0)
    assert np.linalg.norm(disc.P_holes @ r0) > 0.25 * np.linalg.norm(r0)
    u1, info = o3.asdsm(disc, b, tol=0.0, max_sweeps=1, accel_m=4, u0=u0, stagnation_window=10**9)
    assert info["kinds"] == ["hole_fix"]
    r1 = disc.residual(b[0], u1)
    assert np.linalg.norm(disc.P_holes @ r1) <= 1e-12 * np.linalg.norm(r0)
    np.testing.assert_array_equal(disc.P_skel @ u1, disc.P_skel @ u0)


def test_fine_only_residual_matches_the_full_discretisation_and_vanishes_on_quadratics():
    """residual_grid3d (the fine system alone, for grids too large for the
    submesh factorizations) against Discretisation3D on a small grid, and
    exactly zero on a quadratic field: centred second and first differences
    are exact for quadratics, so the field solves the discrete system."""
    N, mc = 17, 4
    alpha, beta = (0.8, 1.7, 0.5), (2.5, -4.0, 1.5)
    rng = np.random.default_rng(3)
    s, u = rng.standard_normal((N, N, N)), rng.standard_normal((N, N, N))
    disc = o3.Discretisation3D(N, mc, alpha, beta)
    b_ff = disc.rhs(s, u)[0]
    r, b = o3.residual_grid3d(N, alpha, beta, s, u)
    assert np.allclose(b, b_ff, rtol=1e-14, atol=0)
    assert np.allclose(r, disc.residual(b_ff, o3.interior(u)), rtol=1e-13, atol=1e-10)

    N = 33
    x = np.linspace(0.0, 1.0, N)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    w = 1.0 + X * X - 2.0 * Y * Z + 3.0 * Z * Z - X * Y
    # -alpha . (w_xx, w_yy, w_zz) + beta . grad w
    s = (-(alpha[0] * 2.0 + alpha[2] * 6.0)
         + beta[0] * (2.0 * X - Y) + beta[1] * (-2.0 * Z - X) + beta[2] * (-2.0 * Y + 6.0 * Z))
    r, b = o3.residual_grid3d(N, alpha, beta, s, w)
    assert np.linalg.norm(r) <= 1e-10 * np.linalg.norm(b)
    # a wrong sign of one first-difference term is visible
    r_bad, _ = o3.residual_grid3d(N, alpha, (beta[0], -beta[1], beta[2]), s, w)
    assert np.linalg.norm(r_bad) > 1e-3 * np.linalg.norm(b)


def test_extrapolation_weights_per_axis_under_the_error_model():
    """R21's weights axis by axis: when each mesh's solution carries its own
    error a hx^2 + b hy^2 + c hz^2 (hx, hy, hz its spacings), the combination
    at the knots and at the other line points is u + (a + b + c) h^2, the fine
    mesh's value.  Exact fields (a = b = c = 0) only check that the weights sum
    to one; here each axis's coefficient must come out h^2, so a wrong sign or
    one line family in place of another fails."""
    N, mc = 17, 4
    disc = o3.Discretisation3D(N, mc, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    h, H = disc.m.h, disc.m.H
    a, b, c = 0.7, -1.9, 2.6
    x = np.linspace(0.0, 1.0, N)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    u = np.sin(X + 2.0 * Y) * np.cos(Z)
    val = lambda sx, sy, sz: u + a * sx**2 + b * sy**2 + c * sz**2
    U_plane = {"x": val(H, h, h), "y": val(h, H, h), "z": val(h, h, H)}     # P_a coarse in a
    U_line = {"x": val(h, H, H), "y": val(H, h, H), "z": val(H, H, h)}      # L_a fine in a only
    _, _, u_hat = disc.skeleton(U_plane, U_line, val(H, H, H))
    msk = disc._masks()
    inter = (msk["x"].astype(int) + msk["y"] + msk["z"]) >= 2
    want = u + (a + b + c) * h**2
    assert inter.sum() > 0
    assert np.allclose(u_hat[inter], want[inter], rtol=0, atol=1e-13)
