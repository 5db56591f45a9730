"""CPU checks of the host precomputation behind the tensor-core Filler: the
hole extension operator G of Algorithm 3 with zero source
(asdsm_hole_extension_operator, host FP64, no GPU), pinned against the oracle's
Filler and against properties of the discrete Dirichlet problem.

* G z reproduces the oracle's hole values (Algorithm 3 with b = 0) for random
  skeleton values, to 1e-12 relative.
* Pure diffusion (beta = 0): the 5-point operator has zero row sums, so a
  constant ring extends to the same constant (every row of G sums to 1), and
  every entry of G is nonnegative (discrete maximum principle).
* Isotropic diffusion: G is invariant under the transposition of the hole
  (x <-> y swaps the west/south and east/north ring blocks).
"""
import numpy as np
import pytest

from oracle import asdsm2d as orc


@pytest.fixture(scope="module")
def asd():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_01163_gb300 import asdsm
    return asdsm


def _ring(Z, bi, bj, n):
    x0, y0 = bi * n, bj * n
    return np.concatenate([Z[y0 + 1:y0 + n, x0], Z[y0 + 1:y0 + n, x0 + n], Z[y0, x0 + 1:x0 + n], Z[y0 + n, x0 + 1:x0 + n]])


@pytest.mark.parametrize("N,mc,alpha,beta", [
    (33, 2, (1.0, 1.0), (0.0, 0.0)),            # n = 16: the tensor-core Filler's size
    (49, 3, (0.8, 1.7), (2.5, -4.0)),
    (65, 4, (1.0, 0.05), (40.0, 0.0)),          # convection-dominated along x
    (65, 8, (0.3, 1.2), (-6.0, 3.0)),           # n = 8
])
def test_operator_reproduces_the_oracle_filler(asd, N, mc, alpha, beta):
    n = (N - 1) // mc
    G = asd.hole_extension_operator(N, mc, alpha, beta)
    assert G.shape == ((n - 1) ** 2, 4 * (n - 1))
    rng = np.random.default_rng(N + mc)
    Z = rng.normal(size=(N, N))
    Z[0, :] = Z[-1, :] = Z[:, 0] = Z[:, -1] = 0.0
    disc = orc.Discretisation2D(N, mc, alpha, beta)
    ref = orc.to_grid(disc.filler(orc.interior(Z), np.zeros((N - 2) ** 2)), np.zeros((N, N)))
    for bj in range(mc):
        for bi in range(mc):
            mine = (G @ _ring(Z, bi, bj, n)).reshape(n - 1, n - 1)
            want = ref[bj * n + 1:bj * n + n, bi * n + 1:bi * n + n]
            assert np.linalg.norm(mine - want) <= 1e-12 * max(np.linalg.norm(want), 1e-300)


def test_pure_diffusion_rows_sum_to_one_and_are_nonnegative(asd):
    G = asd.hole_extension_operator(4097, 256, (0.8, 1.7), (0.0, 0.0))
    assert np.allclose(G.sum(axis=1), 1.0, rtol=0, atol=1e-13)
    assert G.min() >= -1e-15


def test_isotropic_operator_is_symmetric_under_transposition(asd):
    C = 15
    G = asd.hole_extension_operator(4097, 256, (1.0, 1.0), (0.0, 0.0))
    perm_out = np.array([(x - 1) * C + (y - 1) for y in range(1, C + 1) for x in range(1, C + 1)])
    # ring blocks: west <-> south, east <-> north under x <-> y
    perm_ring = np.concatenate([np.arange(2 * C, 3 * C), np.arange(3 * C, 4 * C), np.arange(0, C), np.arange(C, 2 * C)])
    assert np.allclose(G[perm_out][:, perm_ring], G, rtol=0, atol=1e-14)


def test_invalid_sizes_are_rejected(asd):
    with pytest.raises(asd.AsdsmError):
        asd.hole_extension_operator(100, 8, (1.0, 1.0), (0.0, 0.0))
