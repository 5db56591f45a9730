"""CPU pins of two readings of the 2D oracle that decide what a sweep does.

* R9, the normalisation of the two anisotropic solutions of a sweep's
  correction (Algorithm 1 without b_cc): each family is divided by its own
  Euclidean norm.  Pinned by (a) the merge of Algorithm 2 passing two
  families through untouched when, so normalised, they already agree at the
  cross points (the mismatch it splines is then zero), and (b) the
  correction's invariance under scaling either family's right-hand side.
* R18, when rounding has left enough residual in the holes for a Filler pass
  to replace a sweep.  Pinned by Prop. 3.1 (the pass leaves no hole residual
  and does not touch the skeleton) and by where the trigger sits: just above
  and just below hole_fix_ratio of the whole residual.

Planted mistakes (in the oracle, on the CPU), each caught by a pin here: no
normalisation, one common norm for both families, the max norm, and a
trigger comparing squared norms against the unsquared ratio.
"""
import numpy as np
import pytest

from oracle import asdsm2d as o
from paper_2303_01163_gb300 import workloads as w


def _disc(N=33, mc=4):
    return o.Discretisation2D(N, mc, (0.7, 1.3), (2.0, -1.5))


def _agreeing_families(disc):
    """Two anisotropic fields, of different norms and different max norms, whose
    unit-2-norm versions agree at the cross points Omega^{H,H}."""
    m = disc.m
    fld = lambda x, y: np.sin(np.pi * x) * np.sin(2 * np.pi * y) + 3 * x * y * (1 - x) * (1 - y)
    xf, yf = m.fc[:, 0] * m.h, m.fc[:, 1] * m.h
    xc, yc = m.cf[:, 0] * m.h, m.cf[:, 1] * m.h
    # psi and phi vanish on the coarse points (y = k H on cf, x = k H on fc):
    # psi changes v_cf's norm and max norm, phi then restores equal norms.
    v_cf = fld(xc, yc) + 1.5 * np.sin(m.mc * np.pi * yc) * (1 + xc)
    v_fc = fld(xf, yf)
    phi = np.sin(m.mc * np.pi * xf) * (1 + yf)
    roots = np.roots([phi @ phi, 2 * (v_fc @ phi), v_fc @ v_fc - v_cf @ v_cf])
    assert np.all(np.isreal(roots))
    v_fc = v_fc + float(np.real(roots).max()) * phi
    assert np.isclose(np.linalg.norm(v_cf), np.linalg.norm(v_fc), rtol=1e-13)
    assert abs(np.abs(v_cf).max() - np.abs(v_fc).max()) > 0.05 * np.abs(v_fc).max()
    return v_fc, v_cf


def test_normalised_families_that_agree_at_cross_points_merge_untouched():
    disc = _disc()
    v_fc, v_cf = _agreeing_families(disc)
    # Right-hand sides whose solutions are 2 v_fc and 7 v_cf: the scales differ,
    # so only a per-family normalisation makes the two agree at the cross points.
    r_fc, r_cf = disc.A_fc @ (2.0 * v_fc), disc.A_cf @ (7.0 * v_cf)
    unit = v_fc / np.linalg.norm(v_fc), v_cf / np.linalg.norm(v_cf)
    for choice in (0, 1):
        e = disc.initial_guess(np.zeros(disc.m.Nf ** 2), r_fc, r_cf, None, choice)
        np.testing.assert_allclose(disc.P_ff_fc @ e, unit[0], rtol=0, atol=1e-12)
        np.testing.assert_allclose(disc.P_ff_cf @ e, unit[1], rtol=0, atol=1e-12)


def test_sweep_correction_is_invariant_to_per_family_scaling():
    disc = _disc()
    r = np.random.default_rng(5).normal(size=disc.m.Nf ** 2)
    r_fc, r_cf = disc.P_ff_fc @ r, disc.P_ff_cf @ r
    zero = np.zeros_like(r)
    for choice in (0, 1):
        e1 = disc.initial_guess(zero, r_fc, r_cf, None, choice)
        e2 = disc.initial_guess(zero, 3.0 * r_fc, 0.25 * r_cf, None, choice)
        np.testing.assert_allclose(e2, e1, rtol=0, atol=1e-12 * np.abs(e1).max())


# ---------------------------------------------------------------------------
# R18: the hole-residual Filler pass.
# ---------------------------------------------------------------------------
def _problem(N=33, mc=4):
    p = w.random_fourier_2d(N, 3)
    disc = o.Discretisation2D(N, mc, p.alpha, p.beta)
    return disc, disc.rhs(p.s, p.g)


def test_filler_pass_removes_the_hole_residual_and_keeps_the_skeleton():
    disc, b = _problem()
    u_ff = disc.solve_fine(b[0])
    u0 = u_ff + np.random.default_rng(2).normal(size=u_ff.size) * np.abs(u_ff).max()
    r0 = disc.residual(b[0], u0)
    assert np.linalg.norm(disc.P_ff_holes @ r0) > 0.25 * np.linalg.norm(r0)
    u1, info = o.asdsm(disc, b, tol=0.0, max_sweeps=1, accel_m=8, u0=u0, stagnation_window=10**9)
    assert info["kinds"] == ["hole_fix"]
    r1 = disc.residual(b[0], u1)
    assert np.linalg.norm(disc.P_ff_holes @ r1) <= 1e-12 * np.linalg.norm(r0)     # Prop. 3.1
    np.testing.assert_array_equal(disc.P_ff_skel @ u1, disc.P_ff_skel @ u0)


def _iterate_with_hole_ratio(disc, b, rho):
    """An iterate whose hole residual is rho times its whole residual: a filled
    iterate (zero hole residual, Prop. 3.1) plus t times a hole perturbation d,
    t chosen so that ||P_h r|| = rho ||r|| with r = r_a - t A d."""
    rng = np.random.default_rng(7)
    u_ff = disc.solve_fine(b[0])
    u_a = disc.filler(u_ff + disc.P_ff_skel.T @ rng.normal(size=disc.P_ff_skel.shape[0]), b[0])
    r_a = disc.residual(b[0], u_a)
    d = disc.P_ff_holes.T @ rng.normal(size=disc.P_ff_holes.shape[0])
    Ad = disc.A_ff @ d
    p2 = np.linalg.norm(disc.P_ff_holes @ Ad) ** 2
    # t^2 p2 = rho^2 (|r_a|^2 - 2 t <r_a, Ad> + t^2 |Ad|^2)
    roots = np.roots([p2 - rho**2 * (Ad @ Ad), 2 * rho**2 * (r_a @ Ad), -rho**2 * (r_a @ r_a)])
    t = max(float(np.real(x)) for x in roots if abs(np.imag(x)) == 0 and np.real(x) > 0)
    u = u_a + t * d
    r = disc.residual(b[0], u)
    assert np.isclose(np.linalg.norm(disc.P_ff_holes @ r) / np.linalg.norm(r), rho, rtol=1e-9)
    return u


@pytest.mark.parametrize("rho,kind", [(0.25 * (1 + 1e-6), "hole_fix"), (0.25 * (1 - 1e-6), "sweep")])
def test_hole_fix_trigger_sits_at_the_ratio(rho, kind):
    disc, b = _problem()
    u0 = _iterate_with_hole_ratio(disc, b, rho)
    _, info = o.asdsm(disc, b, tol=0.0, max_sweeps=1, accel_m=8, u0=u0, stagnation_window=10**9,
                      hole_fix_ratio=0.25, hole_fix_growth=4.0)
    assert info["kinds"] == [kind]


def test_hole_fix_growth_rule():
    """With ratio 0 only the growth rule decides: the first hole residual above
    zero triggers a pass (nothing was filled before), an infinite growth never."""
    disc, b = _problem()
    u0 = _iterate_with_hole_ratio(disc, b, 0.01)
    _, info = o.asdsm(disc, b, tol=0.0, max_sweeps=1, accel_m=8, u0=u0, stagnation_window=10**9,
                      hole_fix_ratio=0.0, hole_fix_growth=4.0)
    assert info["kinds"] == ["hole_fix"]
    _, info = o.asdsm(disc, b, tol=0.0, max_sweeps=3, accel_m=8, u0=u0, stagnation_window=10**9,
                      hole_fix_ratio=0.0, hole_fix_growth=np.inf)
    assert info["kinds"] == ["sweep"] * 3


# ---------------------------------------------------------------------------
# Planted mistakes.
# ---------------------------------------------------------------------------
def _unnormalised(u_fc, u_cf):
    return u_fc, u_cf


def _common_norm(u_fc, u_cf):
    n = np.sqrt(u_fc @ u_fc + u_cf @ u_cf)
    return u_fc / n, u_cf / n


def _max_norm(u_fc, u_cf):
    return u_fc / np.abs(u_fc).max(), u_cf / np.abs(u_cf).max()


@pytest.mark.parametrize("plant", [_unnormalised, _common_norm, _max_norm])
def test_planted_normalisation_mistakes_are_caught(monkeypatch, plant):
    monkeypatch.setattr(o, "normalised_families", plant)
    with pytest.raises(AssertionError):
        test_normalised_families_that_agree_at_cross_points_merge_untouched()


def test_planted_squared_trigger_is_caught(monkeypatch):
    monkeypatch.setattr(o, "hole_fix_due", lambda hn, rn, ref, ratio, growth:
                        hn**2 > ratio * rn**2 and hn > growth * ref)
    with pytest.raises(AssertionError):
        test_hole_fix_trigger_sits_at_the_ratio(0.25 * (1 + 1e-6), "hole_fix")
