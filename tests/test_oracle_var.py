"""Pins of the variable-coefficient oracle (oracle/asdsm2d_var.py, reading
R29), independent of its own formulas:

* with constant functions every operator and right-hand side equals the
  constant-coefficient oracle's (itself pinned in test_oracle_pins);
* quadratic fields solve the discrete system on all four meshes with
  coefficients that vary in space (centred differences are exact for
  quadratics, so a coefficient sampled at the wrong point, a lifting with the
  wrong weight or a wrong sign fails);
* second-order accuracy of the fine solution on Example 1's second setting;
* Proposition 3.1 (zero residual in the holes after Algorithm 3) and GCR
  refinement to the direct fine solution, both unchanged by the coefficients.
"""
import numpy as np
import scipy.sparse.linalg as spla
import pytest

from oracle import asdsm2d as orc
from oracle import asdsm2d_var as ov
from paper_2303_01163_gb300 import workloads as wl


def test_constant_functions_give_the_constant_coefficient_systems():
    N, mc = 33, 4
    alpha, beta = (0.8, 1.7), (2.5, -4.0)
    fa = (lambda x, y: np.full_like(x, alpha[0]), lambda x, y: np.full_like(x, alpha[1]))
    fb = (lambda x, y: np.full_like(x, beta[0]), lambda x, y: np.full_like(x, beta[1]))
    dv = ov.Discretisation2DVar(N, mc, fa, fb)
    dc = orc.Discretisation2D(N, mc, alpha, beta)
    for name in ("A_ff", "A_fc", "A_cf", "A_cc"):
        diff = abs(getattr(dv, name) - getattr(dc, name)).max()
        assert diff <= 1e-12 * abs(getattr(dc, name)).max(), name
    rng = np.random.default_rng(4)
    s, g = rng.standard_normal((N, N)), rng.standard_normal((N, N))
    for bv, bc in zip(dv.rhs(s, g), dc.rhs(s, g)):
        assert np.allclose(bv, bc, rtol=1e-13, atol=1e-12 * np.abs(bc).max())


def test_quadratic_fields_solve_every_mesh_with_variable_coefficients():
    N, mc = 33, 4
    alpha, beta = wl.variable_coefficients_example1()
    d = ov.Discretisation2DVar(N, mc, alpha, beta)
    x = np.linspace(0.0, 1.0, N)
    Y, X = np.meshgrid(x, x, indexing="ij")
    q = 1.0 + 0.5 * X - 0.3 * Y + X * X - 1.5 * X * Y + 0.8 * Y * Y
    qx, qy = 0.5 + 2.0 * X - 1.5 * Y, -0.3 - 1.5 * X + 1.6 * Y
    s = -alpha[0](X, Y) * 2.0 - alpha[1](X, Y) * 1.6 + beta[0](X, Y) * qx + beta[1](X, Y) * qy
    m = d.m
    for A, pts, b in zip((d.A_ff, d.A_fc, d.A_cf, d.A_cc), (m.ff, m.fc, m.cf, m.cc), d.rhs(s, q)):
        r = b - A @ q[pts[:, 1], pts[:, 0]]
        assert np.abs(r).max() <= 1e-9 * np.abs(b).max()
    # coefficients sampled one point to the east are visible
    shifted = (lambda x, y: alpha[0](x + 1.0 / (N - 1), y), alpha[1])
    d2 = ov.Discretisation2DVar(N, mc, shifted, beta)
    r = d2.rhs(s, q)[0] - d2.A_ff @ orc.interior(q)
    assert np.abs(r).max() > 1e-3


def test_fine_solution_is_second_order_on_example_1_setting_2():
    errs = []
    for N in (65, 129, 257):
        p = wl.manufactured_variable_2d(N)
        r, b = ov.residual_grid_var(N, p.alpha, p.beta, p.s, p.g)      # b - A g: b with the lifting
        M = N - 1
        fine = np.arange(1, M)
        A = ov.operator_2d_var(fine, fine, 1.0 / M, 1.0 / M, M, p.alpha, p.beta)
        u = spla.spsolve(A.tocsc(), b)
        errs.append(np.abs(u - orc.interior(p.u_exact)).max())
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.6 <= q <= 4.4 for q in ratios), (errs, ratios)


def test_filler_zeroes_the_hole_residual_and_gcr_reaches_the_fine_solution():
    N, mc = 65, 8
    p = wl.manufactured_variable_2d(N)
    d = ov.Discretisation2DVar(N, mc, p.alpha, p.beta)
    b = d.rhs(p.s, p.g)
    rng = np.random.default_rng(9)
    u_t = d.P_ff_skel.T @ rng.standard_normal(d.P_ff_skel.shape[0])     # any skeleton, holes empty
    r = d.residual(b[0], d.filler(u_t, b[0]))
    assert np.abs(d.P_ff_holes @ r).max() <= 1e-9 * np.abs(b[0]).max()
    u, info = orc.asdsm(d, b, tol=1e-10, max_sweeps=300, accel_m=8)
    assert info["status"] == "converged", info["status"]
    u_ff = d.solve_fine(b[0])
    assert np.linalg.norm(u - u_ff) <= 1e-7 * np.linalg.norm(u_ff)
