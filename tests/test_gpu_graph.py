"""Device-driven sweeps (CUDA graphs) against host-driven sweeps.

Both paths launch the same kernels; only where the decisions between sweeps
are taken differs (a single-thread controller kernel vs the host), in the same
FP64 operations.  The two may differ by FMA contraction in that scalar
arithmetic, so histories agree to rounding, and for the FP64 path the final
iterates to 1e-10 relative.
"""
import numpy as np
import pytest

from oracle import asdsm2d as orc
from paper_2303_01163_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_01163_gb300 import asdsm
    return asdsm


def _dev(a):
    import torch
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _relerr(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


def _solve(lib, p, mc, prec, graph, **kw):
    with lib.Solver(p.N, mc, p.alpha, p.beta, precision=prec, sweep_graph=graph, **kw) as sv:
        u = _dev(p.g)
        res = sv.solve(_dev(p.s), u)
        return res, u.cpu().numpy()


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
@pytest.mark.parametrize("m", [1, 4, 8])
def test_graph_sweeps_follow_host_sweeps(lib, prec_name, m):
    p = wl.random_fourier_2d(129, 7)
    prec = lib.FP64 if prec_name == "fp64" else lib.MIXED
    kw = dict(tol=1e-10, max_sweeps=300, accel_m=m, seed=5)
    rh, uh = _solve(lib, p, 16, prec, 0, **kw)
    rg, ug = _solve(lib, p, 16, prec, 1, **kw)
    assert rg.status == rh.status
    assert abs(rg.stats["sweeps"] - rh.stats["sweeps"]) <= 2, (rg.stats, rh.stats)
    assert rg.stats["hole_fixes"] == rh.stats["hole_fixes"]
    n = min(len(rg.history), len(rh.history), 20)
    np.testing.assert_allclose(rg.history[:n], rh.history[:n], rtol=1e-4)
    if prec == lib.FP64 and rg.stats["sweeps"] == rh.stats["sweeps"]:
        assert _relerr(orc.interior(ug), orc.interior(uh)) <= 1e-10
    if rh.status == lib.OK:             # plain ASDSM (m = 1) stagnates above 1e-10 on this problem
        r, bb = orc.residual_grid(p.N, p.alpha, p.beta, p.s, ug)
        assert np.linalg.norm(r) / np.linalg.norm(bb) <= 1e-10 * 1.01
    assert rg.stats["launches"] > 0


def test_graph_matches_oracle_iterates(lib):
    """Fixed sweep counts, FP64: the graph path's iterates are the oracle's."""
    p = wl.random_fourier_2d(65, 4, kmax=8)
    disc = orc.Discretisation2D(65, 8, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    for sweeps in (1, 3, 9, 17):        # inside one graph launch, at its end and across launches
        uo, info = orc.asdsm(disc, b, tol=1e-30, max_sweeps=sweeps, accel_m=4, seed=2, stagnation_window=10**9)
        res, u = _solve(lib, p, 8, lib.FP64, 1, tol=1e-30, max_sweeps=sweeps, accel_m=4, seed=2, stagnation_window=0)
        assert res.stats["sweeps"] == info["sweeps"]
        assert _relerr(orc.interior(u), uo) <= 1e-12, (sweeps, _relerr(orc.interior(u), uo))
        np.testing.assert_allclose(res.history, info["hist"], rtol=1e-6, atol=1e-11)


def test_hole_correction_branch_in_the_graph(lib):
    """Thresholds of zero make every sweep a hole correction (the branch of the
    switch node for iterate buffer 0); a low threshold mixes corrections into
    the sweeps (either buffer).  The graph takes the branches the host takes."""
    p = wl.random_fourier_2d(129, 3)
    for prec in (lib.FP64, lib.MIXED):
        kw = dict(tol=1e-30, max_sweeps=5, accel_m=8, hole_fix_ratio=0.0, hole_fix_growth=0.0)
        rh, uh = _solve(lib, p, 16, prec, 0, **kw)
        rg, ug = _solve(lib, p, 16, prec, 1, **kw)
        assert rh.stats["hole_fixes"] == rg.stats["hole_fixes"] == 5
        assert _relerr(orc.interior(ug), orc.interior(uh)) <= 1e-12
        kw = dict(tol=1e-10, max_sweeps=200, accel_m=8, hole_fix_ratio=1e-4, hole_fix_growth=1.0)
        rh, uh = _solve(lib, p, 16, prec, 0, **kw)
        rg, ug = _solve(lib, p, 16, prec, 1, **kw)
        assert rg.stats["hole_fixes"] == rh.stats["hole_fixes"]
        assert rg.status == rh.status
        assert abs(rg.stats["sweeps"] - rh.stats["sweeps"]) <= 2


def test_graph_is_reused_and_rebuilt(lib):
    """Repeated solves on one handle replay the cached graph; changing m or the
    precision rebuilds it; results do not depend on what ran before."""
    p = wl.random_fourier_2d(129, 8)
    with lib.Solver(p.N, 16, p.alpha, p.beta, precision=lib.MIXED, tol=1e-10, max_sweeps=300, accel_m=8) as sv:
        s = _dev(p.s)
        outs = []
        for opts in ({}, {}, {"accel_m": 4}, {"precision": lib.FP64}, {"accel_m": 8, "precision": lib.MIXED}):
            if opts:
                sv.set_opts(**opts)
            u = _dev(p.g)
            res = sv.solve(s, u)
            assert res.status == lib.OK
            outs.append((res.stats["sweeps"], u.cpu().numpy()))
        assert outs[0][0] == outs[1][0] == outs[4][0]
        assert np.array_equal(outs[0][1], outs[1][1])
        assert np.array_equal(outs[0][1], outs[4][1])


def test_graph_max_sweeps_and_stagnation(lib):
    p = wl.random_fourier_2d(129, 2)
    res, _ = _solve(lib, p, 16, lib.MIXED, 1, tol=1e-30, max_sweeps=13, accel_m=8)
    assert res.status == lib.NOT_CONVERGED and res.stats["sweeps"] == 13
    assert len(res.history) == 14
    res, _ = _solve(lib, p, 16, lib.FP64, 1, tol=1e-30, max_sweeps=400, accel_m=1, stagnation_window=5,
                    stagnation_factor=0.5)
    assert res.status == lib.STAGNATED
    h = res.history
    assert h[-1] > 0.5 * h[-6]


@pytest.mark.parametrize("prec_name", ["fp64", "mixed"])
def test_autotuned_shapes_keep_parity(lib, prec_name):
    """After asdsm_autotune the level products may sum in another order; the
    solves still meet the parity bars (FP64 iterates vs the oracle, mixed
    convergence to the fine solution)."""
    p = wl.random_fourier_2d(129, 7)
    prec = lib.FP64 if prec_name == "fp64" else lib.MIXED
    disc = orc.Discretisation2D(p.N, 16, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    if prec == lib.FP64:
        uo, info = orc.asdsm(disc, b, tol=1e-30, max_sweeps=6, accel_m=4, seed=1, stagnation_window=10**9)
        kw = dict(tol=1e-30, max_sweeps=6, accel_m=4, seed=1, stagnation_window=0)
    else:
        kw = dict(tol=1e-10, max_sweeps=300, accel_m=8)
    with lib.Solver(p.N, 16, p.alpha, p.beta, precision=prec, **kw) as sv:
        sv.autotune()
        u = _dev(p.g)
        res = sv.solve(_dev(p.s), u)
        U = u.cpu().numpy()
    if prec == lib.FP64:
        assert _relerr(orc.interior(U), uo) <= 1e-12
    else:
        assert res.status == lib.OK
        r, bb = orc.residual_grid(p.N, p.alpha, p.beta, p.s, U)
        assert np.linalg.norm(r) / np.linalg.norm(bb) <= 1e-10 * 1.01
