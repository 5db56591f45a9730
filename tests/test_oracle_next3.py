"""The follow-up readings R27 (residual smoothing, Example 2 of Section 4) and
R28 (extra anisotropic meshes for the extrapolation, the remark after
Algorithm 2) in the 2D oracle: each pinned by a brute-force or closed-form
check, and the two measurements that decided they stay out of the CUDA path.

* R27: the smoothed projections against a point-by-point loop over the full
  grid (a transposed family or a shifted cross point fails it); the "knots"
  reading maps a residual on the cross points to zero; on the paper's Example
  2 problem (alpha = beta = 1, u = sin(pi x + pi y)) neither reading lowers
  the level at which plain ASDSM (m = 1) stagnates, and both slow GCR(8).
* R28: on samples that follow the error model u + a h_x^2 + b h_y^2 exactly,
  R7 returns the fine discrete value u + (a + b) h^2 and R28 the continuous
  value u; on the Example 1 problem R28's knots are further from the fine
  discrete solution than R7's.
"""
import numpy as np
import pytest

from oracle import asdsm2d as orc
from paper_2303_01163_gb300 import workloads as wl


@pytest.mark.parametrize("mode", ["knots", "lines"])
def test_smoothed_projections_match_a_pointwise_loop(mode):
    N, mc = 17, 4
    m = orc.Meshes2D(N, mc)
    rng = np.random.default_rng(5)
    R = np.zeros((N, N))                    # [y, x], zero on the boundary
    R[1:-1, 1:-1] = rng.standard_normal((N - 2, N - 2))
    disc = orc.Discretisation2D(N, mc, (1.0, 1.0), (0.0, 0.0))
    r = orc.interior(R)
    got_fc, got_cf = orc.smooth_projections(m, disc.P_ff_fc @ r, disc.P_ff_cf @ r, mode)

    def smooth(val, prev, nxt, at_cross):
        if mode == "knots":
            return 0.5 * (prev + nxt) if at_cross else val
        return 0.25 * prev + 0.5 * val + 0.25 * nxt

    want_fc = [smooth(R[j, i], R[j, i - 1], R[j, i + 1], i % m.n == 0) for i, j in m.fc]
    want_cf = [smooth(R[j, i], R[j - 1, i], R[j + 1, i], j % m.n == 0) for i, j in m.cf]
    assert np.allclose(got_fc, want_fc, rtol=0, atol=1e-15)
    assert np.allclose(got_cf, want_cf, rtol=0, atol=1e-15)


def test_knot_smoothing_discards_a_residual_on_the_cross_points():
    """The "knots" reading has a kernel: a residual that lives only on the
    cross points projects to zero, so no correction can remove it."""
    N, mc = 33, 4
    m = orc.Meshes2D(N, mc)
    disc = orc.Discretisation2D(N, mc, (1.0, 1.0), (0.0, 0.0))
    r = disc.P_ff_cc.T @ np.random.default_rng(1).standard_normal(len(m.cc))
    r_fc, r_cf = orc.smooth_projections(m, disc.P_ff_fc @ r, disc.P_ff_cf @ r, "knots")
    assert not r_fc.any() and not r_cf.any()


def test_gcr_with_smoothing_falls_behind_the_plain_correction():
    """GCR(8) on the Example 1 problem at N = 65, mc = 8: 22 sweeps to 1e-10
    without smoothing; with either reading the residual is still above 1e-9
    after 60 sweeps (the smoothed correction is a worse preconditioner, and
    the "knots" reading cannot see cross-point residuals at all)."""
    N, mc = 65, 8
    p = wl.manufactured_shifted_sine_2d(N, (1.0, 1.0), (1.0, 1.0), 1.0)
    disc = orc.Discretisation2D(N, mc, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    _, info = orc.asdsm(disc, b, tol=1e-10, max_sweeps=60, accel_m=8)
    assert info["status"] == "converged" and info["sweeps"] <= 30, info["sweeps"]
    for mode in ("knots", "lines"):
        _, info = orc.asdsm(disc, b, tol=1e-10, max_sweeps=60, accel_m=8, smoothing=mode)
        assert info["status"] != "converged" and min(info["hist"]) > 1e-9, (mode, min(info["hist"]))


def test_smoothing_does_not_lower_the_stagnation_level_of_plain_asdsm():
    """Example 2, first problem, at N = 129 with mc = 8 and 40 sweeps of the
    paper's step: the smallest relative residual reached without smoothing is
    4.8e-9, with "knots" 1.1e-8 and with "lines" 1.8e-8."""
    N, mc = 129, 8
    p = wl.manufactured_shifted_sine_2d(N, (1.0, 1.0), (1.0, 1.0), 1.0)
    disc = orc.Discretisation2D(N, mc, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    floor = {}
    for mode in (None, "knots", "lines"):
        _, info = orc.asdsm(disc, b, tol=1e-14, max_sweeps=40, accel_m=1, stagnation_window=1000,
                            smoothing=mode)
        floor[mode] = min(info["hist"])
    print({k: f"{v:.2e}" for k, v in floor.items()})
    assert floor["knots"] >= floor[None] and floor["lines"] >= floor[None]


def test_extrapolation_readings_on_the_error_model():
    rng = np.random.default_rng(2)
    u, a, b = rng.standard_normal((3, 9))
    h, H = 1.0 / 64, 1.0 / 8
    sample = lambda hx, hy: u + a * hx**2 + b * hy**2
    fc, cf, cc = sample(h, H), sample(H, h), sample(H, H)
    f2, c2 = sample(2 * h, H), sample(H, 2 * h)
    assert np.allclose(orc.extrapolate_knots(fc, cf, cc), u + (a + b) * h**2, rtol=0, atol=1e-14)
    assert np.allclose(orc.extrapolate_knots(fc, cf, cc, f2, c2), u, rtol=0, atol=1e-14)


def test_extra_meshes_move_the_knots_away_from_the_fine_solution():
    """Example 1, first setting, N = 257, mc = 16: max |u_hat - u_ff| over the
    coarse points is 6.4e-6 with R7 and 1.7e-5 with R28."""
    N, mc = 257, 16
    p = wl.manufactured_shifted_sine_2d(N, (1.0, 1.0), (1.0, 1.0), 1.0)
    d = orc.Discretisation2D(N, mc, p.alpha, p.beta)
    b = d.rhs(p.s, p.g)
    u_ff = d.P_ff_cc @ d.solve_fine(b[0])
    fc, cf, cc = d.P_fc_cc @ d.lu_fc.solve(b[1]), d.P_cf_cc @ d.lu_cf.solve(b[2]), d.lu_cc.solve(b[3])
    N2 = (N - 1) // 2 + 1                 # Omega^{2h,H} and Omega^{H,2h}: the same mc on half the fine points
    p2 = wl.manufactured_shifted_sine_2d(N2, (1.0, 1.0), (1.0, 1.0), 1.0)
    d2 = orc.Discretisation2D(N2, mc, p2.alpha, p2.beta)
    b2 = d2.rhs(p2.s, p2.g)
    f2, c2 = d2.P_fc_cc @ d2.lu_fc.solve(b2[1]), d2.P_cf_cc @ d2.lu_cf.solve(b2[2])
    e7 = np.abs(orc.extrapolate_knots(fc, cf, cc) - u_ff).max()
    e28 = np.abs(orc.extrapolate_knots(fc, cf, cc, f2, c2) - u_ff).max()
    print(f"R7 {e7:.2e}, R28 {e28:.2e}")
    assert e28 > e7
