"""GPU parity of the 3D extension (Section 3.5) against the FP64 3D oracle.

Layouts on the GPU side (asdsm_submesh_solve with d = 3): a plane family a
is [k][q][p] with (p, q) the two other axes in increasing order; a line
family a is [f][cq][cp] (f the fine coordinate along a); the coarse mesh
[cz][cy][cx]; holes are read and written on N^3 grids.  The oracle lists
every mesh x fastest, then y, then z; the helpers below permute.

Bars: FP64 path 1e-12 relative (single solves, the initial guess and the
iterates, same random choices); FP32 single solves 2e-5; mixed solves
reach 1e-10 judged by the oracle's FP64 residual.
"""
import numpy as np
import pytest

from oracle import asdsm3d as o3
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


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


# oracle order (x fastest, then y, then z, on the mesh's own index ranges) -> GPU order
def _plane_to_gpu(f, v, m):
    Nf, Nc = m.Nf, m.Nc
    if f == "x":
        return v.reshape(Nf, Nf, Nc).transpose(2, 0, 1).reshape(-1)     # [z][y][kx] -> [kx][z][y]
    if f == "y":
        return v.reshape(Nf, Nc, Nf).transpose(1, 0, 2).reshape(-1)     # [z][ky][x] -> [ky][z][x]
    return v.copy()                                                      # [kz][y][x]


def _line_to_gpu(f, v, m):
    Nf, Nc = m.Nf, m.Nc
    if f == "x":
        return v.reshape(Nc, Nc, Nf).transpose(2, 0, 1).reshape(-1)     # [cz][cy][x] -> [x][cz][cy]
    if f == "y":
        return v.reshape(Nc, Nf, Nc).transpose(1, 0, 2).reshape(-1)     # [cz][y][cx] -> [y][cz][cx]
    return v.copy()                                                      # [z][cy][cx]


CASES = [
    ("sine17_mc4", lambda: wl.manufactured_sine_3d(17, (0.7, 1.3, 0.4), (1.5, -1.0, 0.5)), 4),
    ("rand17_mc4", lambda: wl.random_sine_3d(17, 1), 4),
    ("rand33_mc8", lambda: wl.random_sine_3d(33, 2), 8),
    ("rand33_mc4", lambda: wl.random_sine_3d(33, 3), 4),
    ("pe_near1_17", lambda: wl.manufactured_sine_3d(17, (0.1, 0.5, 1.0), (0.8, -3.0, 0.0)), 4),
]


@pytest.mark.parametrize("name,make,mc", CASES)
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_3d_submesh_solves_match_oracle(lib, name, make, mc, precision):
    import torch
    p = make()
    disc = o3.Discretisation3D(p.N, mc, p.alpha, p.beta)
    m = disc.m
    tol = 1e-12 if precision == "fp64" else 2e-5
    prec = lib.FP64 if precision == "fp64" else lib.MIXED
    rng = np.random.default_rng(7)
    with lib.Solver(p.N, mc, p.alpha, p.beta, precision=prec) as sv:
        for a, f in enumerate(o3.FAMILIES):
            rhs = rng.normal(size=len(m.plane[f]))
            want = _plane_to_gpu(f, disc.lu_plane[f].solve(rhs), m)
            out = torch.zeros(want.size, dtype=torch.float64, device="cuda")
            sv.submesh_solve(lib.MESH3_PLANE + a, _dev(_plane_to_gpu(f, rhs, m)), out)
            assert _rel(out.cpu().numpy(), want) <= tol, ("plane", f, _rel(out.cpu().numpy(), want))
            rhs = rng.normal(size=len(m.line[f]))
            want = _line_to_gpu(f, disc.lu_line[f].solve(rhs), m)
            out = torch.zeros(want.size, dtype=torch.float64, device="cuda")
            sv.submesh_solve(lib.MESH3_LINE + a, _dev(_line_to_gpu(f, rhs, m)), out)
            assert _rel(out.cpu().numpy(), want) <= tol, ("line", f, _rel(out.cpu().numpy(), want))
        rhs = rng.normal(size=len(m.cc))
        out = torch.zeros(rhs.size, dtype=torch.float64, device="cuda")
        sv.submesh_solve(lib.MESH3_COARSE, _dev(rhs), out)
        assert _rel(out.cpu().numpy(), disc.lu_cc.solve(rhs)) <= tol
        F = np.zeros((p.N,) * 3)
        F[1:-1, 1:-1, 1:-1] = rng.normal(size=(m.Nf,) * 3)
        want = disc.lu_holes.solve(disc.P_holes @ o3.interior(F))
        out = _dev(np.full((p.N,) * 3, 7.0))
        sv.submesh_solve(lib.MESH3_HOLES, _dev(F), out)
        got = out.cpu().numpy()
        assert _rel(disc.P_holes @ o3.interior(got), want) <= tol
        assert np.all(disc.P_skel @ o3.interior(got) == 7.0)          # skeleton untouched


@pytest.mark.parametrize("name,make,mc", CASES)
def test_3d_initial_guess_matches_oracle(lib, name, make, mc):
    p = make()
    disc = o3.Discretisation3D(p.N, mc, p.alpha, p.beta)
    ref = disc.initial_guess(*disc.rhs(p.s, p.g))
    for prec, tol in ((lib.FP64, 1e-12), (lib.MIXED, 1e-5)):
        with lib.Solver(p.N, mc, p.alpha, p.beta, precision=prec) as sv:
            u = _dev(p.g)
            sv.initial_guess(_dev(p.s), u)
            got = u.cpu().numpy()
        assert _rel(o3.interior(got), ref) <= tol, (prec, _rel(o3.interior(got), ref))
        ring = np.ones((p.N,) * 3, bool)
        ring[1:-1, 1:-1, 1:-1] = False
        assert np.array_equal(got[ring], p.g[ring])


@pytest.mark.parametrize("name,make,mc", CASES[:4])
@pytest.mark.parametrize("m", [1, 4])
def test_3d_fp64_iterates_match_oracle(lib, name, make, mc, m):
    """Same random choices (R22), same readings: the FP64 iterates agree sweep by sweep."""
    p = make()
    disc = o3.Discretisation3D(p.N, mc, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    for sweeps in (1, 5):
        uo, info = o3.asdsm(disc, b, tol=1e-30, max_sweeps=sweeps, accel_m=m, seed=5, stagnation_window=10**9)
        with lib.Solver(p.N, mc, p.alpha, p.beta, precision=lib.FP64, tol=1e-30, max_sweeps=sweeps,
                        accel_m=m, seed=5, stagnation_window=0) as sv:
            u = _dev(p.g)
            res = sv.solve(_dev(p.s), u)
            got = o3.interior(u.cpu().numpy())
        assert res.stats["sweeps"] == info["sweeps"]
        assert _rel(got, uo) <= 1e-12, (sweeps, _rel(got, uo))
        np.testing.assert_allclose(res.history, info["hist"], rtol=1e-6, atol=1e-11)


@pytest.mark.parametrize("N,mc,seed,m", [(33, 8, 2, 16), (33, 4, 3, 64), (65, 8, 4, 256)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_3d_solve_reaches_the_fine_solution(lib, N, mc, seed, m, precision):
    p = wl.random_sine_3d(N, seed)
    disc = o3.Discretisation3D(N, mc, p.alpha, p.beta)
    b = disc.rhs(p.s, p.g)
    prec = lib.FP64 if precision == "fp64" else lib.MIXED
    with lib.Solver(N, mc, p.alpha, p.beta, precision=prec, tol=1e-10, max_sweeps=800, accel_m=m) as sv:
        u = _dev(p.g)
        res = sv.solve(_dev(p.s), u)
        rel_lib = sv.residual(_dev(p.s), u)
    assert res.status == lib.OK, res.stats
    got = o3.interior(u.cpu().numpy())
    rel = np.linalg.norm(b[0] - disc.A_ff @ got) / np.linalg.norm(b[0])
    assert rel <= 1.01e-10, rel
    assert abs(rel_lib - rel) <= 1e-3 * rel
    assert abs(res.stats["rel_res_fp64"] - rel) <= 1e-3 * rel
    if N <= 33:       # a direct sparse solve of the 3D fine system is cheap only on small grids
        u_ff = disc.solve_fine(b[0])
        kappa = 4.0 / (np.pi**2 / (N - 1) ** 2) * max(p.alpha) / min(p.alpha)
        assert _rel(got, u_ff) <= kappa * rel
    print(f"3D {precision} N={N} mc={mc}: {res.stats['sweeps']} sweeps, oracle residual {rel:.2e}")


def test_3d_sizes_are_checked(lib):
    with pytest.raises(lib.AsdsmError):
        lib.Solver(513, 16, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))          # N above 257
    with pytest.raises(lib.AsdsmError):
        lib.Solver(65, 2, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))            # holes of 31 points per side
    with pytest.raises(lib.AsdsmError):
        lib.Solver(33, 4, (1.0, -1.0, 1.0), (0.0, 0.0, 0.0))           # alpha <= 0


@pytest.mark.parametrize("name,make,mc", CASES[:4] + [("rand65_mc4", lambda: wl.random_sine_3d(65, 8), 4)])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_3d_homogeneous_fill_matches_oracle(lib, name, make, mc, precision):
    """Algorithm 3 with zero source as the sweeps apply it (FP32: the product
    with the hole extension operator; FP64: block cyclic reduction per hole)."""
    import torch
    p = make()
    disc = o3.Discretisation3D(p.N, mc, p.alpha, p.beta)
    rng = np.random.default_rng(11)
    Z = np.zeros((p.N,) * 3)
    Z[1:-1, 1:-1, 1:-1] = rng.normal(size=(disc.m.Nf,) * 3)
    skel = disc.P_skel.T @ (disc.P_skel @ o3.interior(Z))            # skeleton values, zero holes
    want = disc.P_holes @ disc.filler(skel, np.zeros_like(skel))
    prec = lib.FP64 if precision == "fp64" else lib.MIXED
    with lib.Solver(p.N, mc, p.alpha, p.beta, precision=prec) as sv:
        out = _dev(np.full((p.N,) * 3, 7.0))
        sv.submesh_solve(lib.MESH3_FILL, _dev(o3.to_grid(skel, np.zeros((p.N,) * 3))), out)
        got = out.cpu().numpy()
    tol = 1e-12 if precision == "fp64" else 2e-5
    assert _rel(disc.P_holes @ o3.interior(got), want) <= tol
    assert np.all(disc.P_skel @ o3.interior(got) == 7.0)
