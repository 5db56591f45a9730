"""CPU checks of the host precomputation for cube holes (the 3D extension):
asdsm_hole_extension_operator_3d (host FP64 banded elimination, no GPU),
pinned against the 3D oracle's Filler (Algorithm 3 with zero source) and
against properties of the discrete Dirichlet problem.

* G z reproduces the oracle's hole values for random skeleton values (1e-12).
* Pure diffusion: rows of G sum to one (a constant on the faces extends to that
  constant) and every entry is nonnegative (discrete maximum principle).
* Isotropic diffusion: G commutes with exchanging x and y (hole points and faces).
"""
import numpy as np
import pytest

from oracle import asdsm3d as o3


@pytest.fixture(scope="module")
def asd():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_01163_gb300 import asdsm
    return asdsm


def _faces(Z, bi, bj, bk, n):
    """The six faces of hole (bi, bj, bk) of the [z, y, x] grid Z, in the operator's order."""
    x0, y0, z0 = bi * n, bj * n, bk * n
    c = slice(1, n)
    west = Z[z0 + 1:z0 + n, y0 + 1:y0 + n, x0]           # [z][y]: y fastest
    east = Z[z0 + 1:z0 + n, y0 + 1:y0 + n, x0 + n]
    south = Z[z0 + 1:z0 + n, y0, x0 + 1:x0 + n]          # [z][x]
    north = Z[z0 + 1:z0 + n, y0 + n, x0 + 1:x0 + n]
    down = Z[z0, y0 + 1:y0 + n, x0 + 1:x0 + n]           # [y][x]
    up = Z[z0 + n, y0 + 1:y0 + n, x0 + 1:x0 + n]
    return np.concatenate([f.reshape(-1) for f in (west, east, south, north, down, up)])


@pytest.mark.parametrize("N,mc,alpha,beta", [
    (17, 4, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0)),
    (17, 4, (0.8, 1.7, 0.5), (2.5, -4.0, 1.5)),
    (33, 4, (1.0, 0.05, 0.6), (30.0, 0.0, -2.0)),      # convection-dominated along x
])
def test_operator_reproduces_the_3d_oracle_filler(asd, N, mc, alpha, beta):
    n = (N - 1) // mc
    C = n - 1
    G = asd.hole_extension_operator_3d(N, mc, alpha, beta)
    assert G.shape == (C ** 3, 6 * C * C)
    rng = np.random.default_rng(N + mc)
    Z = rng.normal(size=(N, N, N))
    Z[0], Z[-1], Z[:, 0], Z[:, -1], Z[:, :, 0], Z[:, :, -1] = 0, 0, 0, 0, 0, 0
    disc = o3.Discretisation3D(N, mc, alpha, beta)
    ref = o3.to_grid(disc.filler(o3.interior(Z), np.zeros((N - 2) ** 3)), np.zeros((N, N, N)))
    for bk in range(mc):
        for bj in range(mc):
            for bi in range(mc):
                mine = G @ _faces(Z, bi, bj, bk, n)
                want = ref[bk * n + 1:bk * n + n, bj * n + 1:bj * n + n, bi * n + 1:bi * n + n].reshape(-1)
                assert np.linalg.norm(mine - want) <= 1e-12 * max(np.linalg.norm(want), 1e-300)


def test_pure_diffusion_rows_sum_to_one_and_are_nonnegative(asd):
    G = asd.hole_extension_operator_3d(257, 16, (0.8, 1.7, 0.4), (0.0, 0.0, 0.0))
    assert G.shape == (15 ** 3, 6 * 15 * 15)
    assert np.allclose(G.sum(axis=1), 1.0, rtol=0, atol=1e-12)
    assert G.min() >= -1e-14


def test_isotropic_operator_commutes_with_exchanging_x_and_y(asd):
    N, mc = 33, 4
    C = (N - 1) // mc - 1
    F = C * C
    G = asd.hole_extension_operator_3d(N, mc, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    # hole point (x, y, z) <-> (y, x, z)
    pts = np.array([(z * C + x) * C + y for z in range(C) for y in range(C) for x in range(C)])
    # faces: west <-> south, east <-> north (their (y, z) and (x, z) layouts match), down/up transpose (x, y)
    tr = np.array([u * C + v for v in range(C) for u in range(C)])        # (x, y) -> (y, x) within a face
    perm = np.concatenate([2 * F + np.arange(F), 3 * F + np.arange(F), 0 * F + np.arange(F), 1 * F + np.arange(F),
                           4 * F + tr, 5 * F + tr])
    assert np.allclose(G[pts][:, perm], G, rtol=0, atol=1e-14)


def test_invalid_3d_descriptions_are_rejected(asd):
    with pytest.raises(asd.AsdsmError):
        asd.hole_extension_operator_3d(100, 8, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0))
    with pytest.raises(asd.AsdsmError):
        asd.hole_extension_operator_3d(17, 4, (1.0, 1.0, 0.0), (0.0, 0.0, 0.0))
