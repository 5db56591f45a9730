"""Pins of the skeleton-only oracle (oracle/asdsm2d_skel.py, Section 3.3's
remarks on residual sparsity and storage): its sweeps are those of the
full-grid oracle, which keeps every hole value, so the iterates and the
residual histories must agree to rounding; it stores the skeleton and the ring
only, O(N_c N_f) values; and it reaches the fine discrete solution.
"""
import numpy as np
import pytest

from oracle import asdsm2d as orc
from oracle import asdsm2d_skel as osk
from paper_2303_01163_gb300 import workloads as wl


def _case(kind):
    if kind == "sine":
        return wl.manufactured_shifted_sine_2d(65, (1.0, 1.0), (1.0, 1.0), 4.0), 8
    return wl.random_fourier_2d(65, 5), 8


@pytest.mark.parametrize("kind", ["sine", "fourier"])
@pytest.mark.parametrize("m,sweeps", [(1, 6), (4, 10)])
def test_skeleton_only_sweeps_equal_the_full_grid_sweeps(kind, m, sweeps):
    p, mc = _case(kind)
    disc = orc.Discretisation2D(p.N, mc, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    kw = dict(tol=1e-30, max_sweeps=sweeps, accel_m=m, seed=2, stagnation_window=10**9)
    u_full, info_full = orc.asdsm(disc, b, **kw)
    assert "hole_fix" not in info_full["kinds"]
    u_sk, info_sk = osk.asdsm_skeleton_only(disc, b, **kw)
    assert info_sk["sweeps"] == info_full["sweeps"] == sweeps
    assert np.linalg.norm(u_sk - u_full) <= 1e-11 * np.linalg.norm(u_full)
    np.testing.assert_allclose(info_sk["hist"], info_full["hist"], rtol=1e-7)
    np.testing.assert_allclose(info_sk["steps"], info_full["steps"], rtol=1e-7, atol=1e-14)


def test_storage_is_the_skeleton_and_its_ring():
    N, mc = 65, 8
    n, Nf, Nc = (N - 1) // mc, N - 2, mc - 1
    p = wl.manufactured_shifted_sine_2d(N, (1.0, 1.0), (1.0, 1.0), 1.0)
    disc = orc.Discretisation2D(N, mc, p.alpha, p.beta)
    _, info = osk.asdsm_skeleton_only(disc, disc.rhs(p.s, p.g), tol=1e-30, max_sweeps=1)
    skeleton = 2 * Nc * Nf - Nc * Nc
    ring = mc * mc * (4 * (n - 1) - 4)        # each hole's border, corners once
    assert info["stored"] == skeleton + ring
    assert info["full"] == Nf * Nf


def test_skeleton_only_gcr_reaches_the_fine_solution():
    p, mc = _case("fourier")
    disc = orc.Discretisation2D(p.N, mc, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    u, info = osk.asdsm_skeleton_only(disc, b, tol=1e-10, max_sweeps=300, accel_m=8)
    assert info["status"] == "converged", info["status"]
    r = b[0] - disc.A_ff @ u
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b[0])       # holes filled at the end: r = 0 there
    u_ff = disc.solve_fine(b[0])
    h = 1.0 / (p.N - 1)
    kappa = 4.0 / (np.pi**2 * h**2) * max(p.alpha) / min(p.alpha)
    assert np.linalg.norm(u - u_ff) <= kappa * 1.01e-10 * np.linalg.norm(u_ff)
