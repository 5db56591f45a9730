"""GPU parity of the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances:
* FP64 path: every step and every iterate within 1e-12 relative l2 (the
  oracle and the GPU use different exact solvers - sparse LU vs block cyclic
  reduction - so they differ by rounding amplified by the conditioning of the
  small systems; 1e-12 leaves three orders of margin on these sizes).
* Mixed path (FP32 solves/merge/fill, exact residual and accumulation): the
  solve must reach ||b - A u||/||b|| <= 1e-10 as measured by the oracle in
  FP64, and u must agree with the oracle's direct solution u_ff within
  kappa * 1e-10 with kappa = ||A|| ||A^-1|| <= 8 (N-1)^2 / pi^2 (the bound that
  relative residual tol implies).  Single FP32 steps agree to 2e-5 relative.
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


CASES = [
    ("sine65", lambda: wl.manufactured_sine_2d(65), 8),
    ("fourier129", lambda: wl.random_fourier_2d(129, 7), 16),
    ("poly33_mc2", lambda: wl.polynomial_2d(33, alpha=(0.8, 1.7), beta=(2.5, -4.0)), 2),
    ("fourier65_n2", lambda: wl.random_fourier_2d(65, 4, kmax=8), 32),
    ("shift_osc129", lambda: wl.manufactured_shifted_sine_2d(129, alpha=(0.3, 1.2), beta=(-6.0, 3.0), k=4.0), 8),
]


@pytest.mark.parametrize("name,make,mc", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_submesh_solves_match_oracle(lib, name, make, mc, precision):
    import torch
    p = make()
    prec = lib.FP64 if precision == "fp64" else lib.MIXED
    tol = 1e-12 if precision == "fp64" else 2e-5
    disc = orc.Discretisation2D(p.N, mc, p.alpha, p.beta)
    m = disc.m
    rng = np.random.default_rng(1)
    with lib.Solver(p.N, mc, p.alpha, p.beta, precision=prec) as sv:
        for mesh, A, size in ((lib.MESH_FC, disc.A_fc, m.Nc * m.Nf), (lib.MESH_CF, disc.A_cf, m.Nc * m.Nf),
                              (lib.MESH_CC, disc.A_cc, m.Nc * m.Nc)):
            f = rng.normal(size=size)
            ref = disc.lu_fc.solve(f) if mesh == lib.MESH_FC else (disc.lu_cf.solve(f) if mesh == lib.MESH_CF else disc.lu_cc.solve(f))
            out = torch.zeros(size, dtype=torch.float64, device="cuda")
            sv.submesh_solve(mesh, _dev(f), out)
            assert _relerr(out.cpu().numpy(), ref) <= tol, (mesh, _relerr(out.cpu().numpy(), ref))
        # holes: rhs on hole points of a full grid
        F = np.zeros((p.N, p.N))
        F[1:-1, 1:-1] = rng.normal(size=(m.Nf, m.Nf))
        fh = disc.P_ff_holes @ orc.interior(F)
        ref = disc.lu_holes.solve(fh)
        out = _dev(np.full((p.N, p.N), 7.0))
        sv.submesh_solve(lib.MESH_HOLES, _dev(F), out)
        got = out.cpu().numpy()
        assert _relerr(disc.P_ff_holes @ orc.interior(got), ref) <= tol
        assert np.all(disc.P_ff_skel @ orc.interior(got) == 7.0)        # skeleton untouched


@pytest.mark.parametrize("name,make,mc", CASES)
def test_initial_guess_matches_oracle(lib, name, make, mc):
    import torch
    p = make()
    disc = orc.Discretisation2D(p.N, mc, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    ref = disc.initial_guess(*b)
    # Mixed: FP32 solves with FP64-residual refinement (two steps per submesh
    # system, one for the holes) reach the FP64 result to the refinement's
    # contraction (~1e-6 per step) times the FP32 hole rounding.
    for prec, tol in ((lib.FP64, 1e-12), (lib.MIXED, 1e-10)):
        with lib.Solver(p.N, mc, p.alpha, p.beta, precision=prec) as sv:
            u = _dev(p.g)
            sv.initial_guess(_dev(p.s), u)
            got = u.cpu().numpy()
            assert _relerr(orc.interior(got), ref) <= tol, (prec, _relerr(orc.interior(got), ref))
            ring = np.ones((p.N, p.N), bool)
            ring[1:-1, 1:-1] = False
            assert np.array_equal(got[ring], p.g[ring])                     # ring never written


@pytest.mark.parametrize("name,make,mc", CASES[:3])
def test_residual_matches_oracle(lib, name, make, mc):
    import torch
    p = make()
    rng = np.random.default_rng(5)
    U = p.g.copy()
    U[1:-1, 1:-1] = rng.normal(size=(p.N - 2, p.N - 2))
    r_ref, b = orc.residual_grid(p.N, p.alpha, p.beta, p.s, U)
    with lib.Solver(p.N, mc, p.alpha, p.beta, precision=lib.FP64) as sv:
        r = torch.full((p.N, p.N), 3.0, dtype=torch.float64, device="cuda")
        rel = sv.residual(_dev(p.s), _dev(U), r)
        rg = r.cpu().numpy()
    sten = (2 * p.alpha[0] + 2 * p.alpha[1]) * (p.N - 1) ** 2 * 2 + (abs(p.beta[0]) + abs(p.beta[1])) * (p.N - 1)
    assert np.abs(orc.interior(rg) - r_ref).max() <= 1e-14 * (sten * np.abs(U).max() + np.abs(b).max())
    assert abs(rel - np.linalg.norm(r_ref) / np.linalg.norm(b)) <= 1e-12 * rel
    ring = np.ones((p.N, p.N), bool)
    ring[1:-1, 1:-1] = False
    assert np.all(rg[ring] == 0.0)


@pytest.mark.parametrize("name,make,mc", CASES)
@pytest.mark.parametrize("m", [1, 4])
def test_fp64_iterates_match_oracle(lib, name, make, mc, m):
    """Same choice sequence, same readings: FP64 iterates agree sweep by sweep."""
    p = make()
    disc = orc.Discretisation2D(p.N, mc, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    for sweeps in (1, 5):
        uo, info = orc.asdsm(disc, b, tol=1e-30, max_sweeps=sweeps, accel_m=m, seed=11, stagnation_window=10**9)
        with lib.Solver(p.N, mc, p.alpha, p.beta, precision=lib.FP64, tol=1e-30, max_sweeps=sweeps,
                        accel_m=m, seed=11, stagnation_window=0) as sv:
            u = _dev(p.g)
            res = sv.solve(_dev(p.s), u)
            got = orc.interior(u.cpu().numpy())
        assert res.stats["sweeps"] == info["sweeps"]
        assert _relerr(got, uo) <= 1e-12, (sweeps, _relerr(got, uo))
        # Residual histories: iterates agreeing to 1e-12 give relative residuals that agree to
        # ||A|| ||du|| / ||b|| <= 8 (N-1)^2 |u|/|b| * 1e-12 (a few 1e-11 on these grids).
        np.testing.assert_allclose(res.history, info["hist"], rtol=1e-6, atol=1e-11)


def test_fp64_solves_cfg1_to_1e12_like_the_oracle(lib):
    """65 x 65, alpha = beta = (1,1), sin(pi x) sin(pi y): FP64 ASDSM to 1e-12."""
    p = wl.manufactured_sine_2d(65)
    disc = orc.Discretisation2D(65, 8, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    uo, info = orc.asdsm(disc, b, tol=1e-12, max_sweeps=300, accel_m=8, seed=0)
    with lib.Solver(65, 8, p.alpha, p.beta, precision=lib.FP64, tol=1e-12, max_sweeps=300, accel_m=8) as sv:
        u = _dev(p.g)
        res = sv.solve(_dev(p.s), u)
    assert res.status == lib.OK and info["status"] == "converged"
    # Near the FP64 floor (~4e-13 here) the last sweeps are rounding-driven, so
    # the sweep counts agree only roughly; both iterates sit within kappa*tol of u_ff.
    assert abs(res.stats["sweeps"] - info["sweeps"]) <= 0.25 * info["sweeps"]
    got = orc.interior(u.cpu().numpy())
    kappa = 8 * 64**2 / np.pi**2
    assert _relerr(got, uo) <= 2 * kappa * 1e-12
    r, bb = orc.residual_grid(65, p.alpha, p.beta, p.s, u.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(bb) <= 1e-12


MIXED_CASES = [
    ("fourier129", lambda: wl.random_fourier_2d(129, 7), 16),
    ("fourier257", lambda: wl.random_fourier_2d(257, 2), 16),
    ("sine257", lambda: wl.manufactured_sine_2d(257, alpha=(1.0, 0.25), beta=(3.0, -2.0)), 16),
    ("poly65", lambda: wl.polynomial_2d(65, alpha=(0.8, 1.7), beta=(2.5, -4.0)), 8),
]


@pytest.mark.parametrize("name,make,mc", MIXED_CASES)
def test_mixed_converges_to_the_fine_solution(lib, name, make, mc):
    p = make()
    disc = orc.Discretisation2D(p.N, mc, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    uff = disc.solve_fine(b[0])
    with lib.Solver(p.N, mc, p.alpha, p.beta, precision=lib.MIXED, tol=1e-10, max_sweeps=600, accel_m=8) as sv:
        u = _dev(p.g)
        res = sv.solve(_dev(p.s), u)
    assert res.status == lib.OK, res.stats
    U = u.cpu().numpy()
    r, bb = orc.residual_grid(p.N, p.alpha, p.beta, p.s, U)
    assert np.linalg.norm(r) / np.linalg.norm(bb) <= 1e-10 * 1.01
    kappa = 8 * (p.N - 1) ** 2 / np.pi**2
    assert _relerr(orc.interior(U), uff) <= kappa * 1e-10
    ring = np.ones((p.N, p.N), bool)
    ring[1:-1, 1:-1] = False
    assert np.array_equal(U[ring], p.g[ring])


def test_mixed_and_fp64_take_similar_sweeps(lib):
    p = wl.random_fourier_2d(129, 7)
    out = {}
    for prec in (lib.FP64, lib.MIXED):
        with lib.Solver(129, 16, p.alpha, p.beta, precision=prec, tol=1e-10, max_sweeps=600, accel_m=8) as sv:
            u = _dev(p.g)
            out[prec] = sv.solve(_dev(p.s), u).stats["sweeps"]
    assert out[lib.MIXED] <= 1.5 * out[lib.FP64] + 5, out


def test_invalid_and_degenerate_inputs(lib):
    import torch
    with pytest.raises(Exception):
        lib.Solver(64, 8, (1, 1), (0, 0))
    with pytest.raises(Exception):
        lib.Solver(65, 128, (1, 1), (0, 0))
    # zero source and zero boundary: u = 0 exactly, reported converged at once
    with lib.Solver(17, 4, (1, 1), (1, 1), precision=lib.FP64) as sv:
        u = torch.zeros(17, 17, dtype=torch.float64, device="cuda")
        s = torch.zeros_like(u)
        res = sv.solve(s, u)
        assert torch.count_nonzero(u).item() == 0
    # smallest grid the library takes (N = 9, one coarse line per axis)
    p = wl.manufactured_sine_2d(9, alpha=(1.0, 0.7), beta=(1.0, -2.0))
    disc = orc.Discretisation2D(9, 2, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    uff = disc.solve_fine(b[0])
    with lib.Solver(9, 2, p.alpha, p.beta, precision=lib.FP64, tol=1e-14, max_sweeps=200) as sv:
        u = _dev(p.g)
        res = sv.solve(_dev(p.s), u)
    assert res.status == lib.OK
    assert _relerr(orc.interior(u.cpu().numpy()), uff) <= 1e-12


def test_advection_dominated_tiny_grid_matches_oracle_iterates(lib):
    """Cell Peclet ~ 25 on a 9 x 9 grid: ASDSM converges slowly here (the
    oracle too) and its GCR directions become nearly dependent, which
    amplifies the rounding difference between the GPU's one-pass (classical)
    and the oracle's modified Gram-Schmidt; over the first 10 sweeps the GPU
    iterates still follow the oracle's."""
    p = wl.random_fourier_2d(9, 3, kmax=3)
    disc = orc.Discretisation2D(9, 2, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    uo, info = orc.asdsm(disc, b, tol=1e-30, max_sweeps=10, accel_m=8, stagnation_window=10**9)
    with lib.Solver(9, 2, p.alpha, p.beta, precision=lib.FP64, tol=1e-30, max_sweeps=10, accel_m=8,
                    stagnation_window=0) as sv:
        u = _dev(p.g)
        sv.solve(_dev(p.s), u)
    assert _relerr(orc.interior(u.cpu().numpy()), uo) <= 1e-10


def test_nan_source_is_reported_not_trapped(lib):
    import torch
    with lib.Solver(17, 4, (1, 1), (1, 1), precision=lib.MIXED) as sv:
        s = torch.zeros(17, 17, dtype=torch.float64, device="cuda")
        s[5, 5] = float("nan")
        u = torch.zeros_like(s)
        with pytest.raises(Exception) as ei:
            sv.solve(s, u)
        assert ei.value.code == lib.ERR_NAN


def test_resume_from_a_given_iterate(lib):
    p = wl.random_fourier_2d(129, 9)
    for prec in (lib.FP64, lib.MIXED):
        with lib.Solver(129, 16, p.alpha, p.beta, precision=prec, tol=1e-10, max_sweeps=600) as sv:
            u = _dev(p.g)
            sv.set_opts(max_sweeps=10)
            r1 = sv.solve(_dev(p.s), u)
            sv.set_opts(max_sweeps=600, skip_initial_guess=1)
            r2 = sv.solve(_dev(p.s), u)
            assert r2.status == lib.OK
            assert r2.stats["rel_res0"] <= r1.stats["rel_res"] * 1.5


def test_resume_from_a_zero_interior_rescales_the_accumulator(lib):
    """A resume from a zero interior gives the fixed-point shift no hint of the
    solution's size (max |u*| is about 68 here, while the first shift leaves
    room for |u| < 4): the solve restarts with smaller shifts from the last
    iterate that fitted and still reaches 1e-10, judged by the oracle."""
    p = wl.random_fourier_2d(257, 4)
    s = p.s * 1e4
    with lib.Solver(257, 16, p.alpha, p.beta, precision=lib.MIXED, tol=1e-10, max_sweeps=600,
                    skip_initial_guess=1) as sv:
        u = _dev(p.g)
        res = sv.solve(_dev(s), u)
        assert res.status == lib.OK, res.stats
        assert res.stats["rescales"] >= 1
        hist = sv.history()
        assert len(hist) <= res.stats["sweeps"] + 1 and hist[-1] <= 1e-10
    ug = u.cpu().numpy()
    r, b = orc.residual_grid(257, p.alpha, p.beta, s, ug)
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1.01e-10
    assert abs(res.stats["rel_res_fp64"] - rel) <= 1e-3 * rel


@pytest.mark.parametrize("tm,ks", [(32, 1), (128, 1), (128, 2), (128, 4)])
@pytest.mark.parametrize("name,make,mc", CASES[:3] + [("fourier257", lambda: wl.random_fourier_2d(257, 5), 8),
                                                      ("fourier513_c255", lambda: wl.random_fourier_2d(513, 6), 256)])
def test_tensor_core_level_kernels_match_oracle(lib, name, make, mc, tm, ks):
    """Every level of the FP32 submesh solves forced onto a tensor-core kernel
    (TF32 split products; tm = 32: the mma.sync kernel for A_fc and A_cf,
    tm = 128: the tcgen05 kernel for A_fc, A_cf and A_cc, its reduction split
    over ks CTAs of a cluster): the solves within the FP32 bar, and a mixed
    solve still reaches the fine solution."""
    import torch
    p = make()
    disc = orc.Discretisation2D(p.N, mc, p.alpha, p.beta)
    m = disc.m
    rng = np.random.default_rng(3)
    with lib.Solver(p.N, mc, p.alpha, p.beta, precision=lib.MIXED, tol=1e-10, max_sweeps=600) as sv:
        state = sv.tune_state()
        # layout: per precision [aniso fwd 16, aniso bwd 16, cc fwd 16, cc bwd 16, fill]; FP32 second
        base = 4 * 16 + 1
        for q in range(64 if tm == 128 else 32):
            state[base + q] = (tm << 8) | ks
        sv.set_tune_state(state)
        meshes = [(lib.MESH_FC, m.Nc * m.Nf, disc.lu_fc), (lib.MESH_CF, m.Nc * m.Nf, disc.lu_cf)]
        if tm == 128:
            meshes.append((lib.MESH_CC, m.Nc * m.Nc, disc.lu_cc))
        for mesh, size, lu in meshes:
            f = rng.normal(size=size)
            out = torch.zeros(size, dtype=torch.float64, device="cuda")
            sv.submesh_solve(mesh, _dev(f), out)
            ref = lu.solve(f)
            assert _relerr(out.cpu().numpy(), ref) <= 2e-5, (mesh, _relerr(out.cpu().numpy(), ref))
        u = _dev(p.g)
        res = sv.solve(_dev(p.s), u)
    assert res.status == lib.OK, (name, tm, res.status, res.stats)
    r, bb = orc.residual_grid(p.N, p.alpha, p.beta, p.s, u.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(bb) <= 1e-10 * 1.01


def test_tune_set_rejects_a_bad_entry_and_keeps_the_handle(lib):
    p = wl.random_fourier_2d(129, 2)
    with lib.Solver(129, 8, p.alpha, p.beta, precision=lib.MIXED, tol=1e-10, max_sweeps=400) as sv:
        before = sv.tune_state()
        bad = list(before)
        bad[3] = (48 << 8) | 1
        with pytest.raises(lib.AsdsmError):
            sv.set_tune_state(bad)
        assert sv.tune_state() == before
