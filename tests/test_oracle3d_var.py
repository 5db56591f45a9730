"""Pins of the 3D variable-coefficient oracle (oracle/asdsm3d_var.py, R29 in
3D), independent of its own formulas:

* with constant functions every operator and right-hand side equals the
  constant-coefficient 3D oracle's (itself pinned in test_oracle3d_pins);
* quadratic fields solve the fine, plane, line and coarse systems with
  Example 4's coefficients (a coefficient sampled one point off fails);
* second-order accuracy of the fine solution with Example 4's coefficients;
* the cube-hole Filler zeroes the hole residual and GCR reaches the direct
  fine solution.
"""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import asdsm3d as o3
from oracle import asdsm3d_var as ov3
from paper_2303_01163_gb300 import workloads as wl


def _grid(N):
    x = np.linspace(0.0, 1.0, N)
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    return X, Y, Z


def test_constant_functions_give_the_constant_coefficient_systems():
    N, mc = 17, 4
    alpha, beta = (0.8, 1.7, 0.5), (2.5, -4.0, 1.5)
    const = lambda c: (lambda x, y, z: np.full_like(x, c))
    dv = ov3.Discretisation3DVar(N, mc, [const(a) for a in alpha], [const(b) for b in beta])
    dc = o3.Discretisation3D(N, mc, alpha, beta)
    mats = [("A_ff", dv.A_ff, dc.A_ff), ("A_cc", dv.A_cc, dc.A_cc)]
    mats += [(f"A_plane {f}", dv.A_plane[f], dc.A_plane[f]) for f in o3.FAMILIES]
    mats += [(f"A_line {f}", dv.A_line[f], dc.A_line[f]) for f in o3.FAMILIES]
    for name, A, B in mats:
        assert abs(A - B).max() <= 1e-12 * abs(B).max(), name
    rng = np.random.default_rng(6)
    s, g = rng.standard_normal((N, N, N)), rng.standard_normal((N, N, N))
    bv, bc = dv.rhs(s, g), dc.rhs(s, g)
    assert np.allclose(bv[0], bc[0], rtol=1e-13, atol=1e-12 * np.abs(bc[0]).max())
    for q in (1, 2):
        for f in o3.FAMILIES:
            assert np.allclose(bv[q][f], bc[q][f], rtol=1e-13, atol=1e-12 * np.abs(bc[q][f]).max())
    assert np.allclose(bv[3], bc[3], rtol=1e-13, atol=1e-12 * np.abs(bc[3]).max())


def test_quadratic_fields_solve_every_mesh_with_example_4_coefficients():
    N, mc = 17, 4
    alpha, beta = wl.variable_coefficients_example4()
    d = ov3.Discretisation3DVar(N, mc, alpha, beta)
    X, Y, Z = _grid(N)
    q = 1.0 + 0.4 * X - 0.7 * Y + 0.2 * Z + X * X - 1.2 * X * Y + 0.6 * Y * Z + 0.9 * Z * Z
    grads = (0.4 + 2.0 * X - 1.2 * Y, -0.7 - 1.2 * X + 0.6 * Z, 0.2 + 0.6 * Y + 1.8 * Z)
    second = (2.0, 0.0, 1.8)
    s = sum(-alpha[a](X, Y, Z) * second[a] + beta[a](X, Y, Z) * grads[a] for a in range(3))
    b_ff, b_p, b_l, b_c = d.rhs(s, q)
    m = d.m
    samp = lambda pts: q[pts[:, 2], pts[:, 1], pts[:, 0]]
    checks = [(d.A_ff, m.ff, b_ff), (d.A_cc, m.cc, b_c)]
    checks += [(d.A_plane[f], m.plane[f], b_p[f]) for f in o3.FAMILIES]
    checks += [(d.A_line[f], m.line[f], b_l[f]) for f in o3.FAMILIES]
    for A, pts, b in checks:
        assert np.abs(b - A @ samp(pts)).max() <= 1e-9 * np.abs(b).max()
    shifted = (alpha[0], alpha[1], lambda x, y, z: alpha[2](x, y, z + 1.0 / (N - 1)))
    d2 = ov3.Discretisation3DVar(N, mc, shifted, beta)
    assert np.abs(d2.rhs(s, q)[0] - d2.A_ff @ samp(m.ff)).max() > 1e-3


def test_fine_solution_is_second_order_with_example_4_coefficients():
    alpha, beta = wl.variable_coefficients_example4()
    errs = []
    for N in (9, 17, 33):
        p = wl.manufactured_variable_3d(N, k=1.0)
        M = N - 1
        fine = np.arange(1, M)
        A = ov3.operator_3d_var([fine] * 3, (1.0 / M,) * 3, M, alpha, beta)
        b = ov3.rhs_on_mesh_var3(o3.Meshes3D._product(fine, fine, fine), (1.0 / M,) * 3, M, alpha, beta, p.s, p.g)
        u = spla.spsolve(A.tocsc(), b)
        errs.append(np.abs(u - o3.interior(p.u_exact)).max())
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(3.5 <= r <= 4.5 for r in ratios), (errs, ratios)


def test_filler_and_gcr_with_example_4_coefficients():
    N, mc = 17, 4
    p = wl.manufactured_variable_3d(N)
    d = ov3.Discretisation3DVar(N, mc, p.alpha, p.beta)
    b = d.rhs(p.s, p.g)
    rng = np.random.default_rng(2)
    u_t = d.P_skel.T @ rng.standard_normal(d.P_skel.shape[0])
    r = d.residual(b[0], d.filler(u_t, b[0]))
    assert np.abs(d.P_holes @ r).max() <= 1e-9 * np.abs(b[0]).max()
    u, info = o3.asdsm(d, b, tol=1e-10, max_sweeps=400, accel_m=16)
    assert info["status"] == "converged", info["status"]
    u_ff = d.solve_fine(b[0])
    assert np.linalg.norm(u - u_ff) <= 1e-7 * np.linalg.norm(u_ff)
