"""GPU parity of the Filler with zero source (Algorithm 3 as every sweep of
Algorithm 4 uses it) against the FP64 oracle, through the C ABI
(asdsm_submesh_solve, mesh 4).

For holes of 15 x 15 points (n = 16) the mixed path runs the tensor-core
kernel (a TF32 split-product GEMM of the hole extension operator with the ring
values); other hole sizes, and the tuned state selecting it, run the block
cyclic reduction kernel.  Bars: FP32 results within 2e-5 relative l2 of the
oracle, FP64 within 1e-12; points that are not hole points stay untouched.
At the 4097^2 size the check is per hole: sampled holes are re-solved by the
oracle on a 49^2 grid whose centre hole gets the same ring values, and every
hole's equations are checked through the oracle's residual.
"""
import numpy as np
import pytest

from oracle import asdsm2d as orc
from paper_2303_01163_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FILL_TC, FILL_BCR8 = 16, 8
TUNE_FILL_MIXED = 2 * (4 * 16 + 1) - 1      # the Filler entry of the FP32 half of the tune state


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


def _skeleton_grid(N, seed):
    """Random skeleton values, zero boundary ring (a sweep direction's data)."""
    rng = np.random.default_rng(seed)
    Z = rng.normal(size=(N, N))
    Z[0, :] = Z[-1, :] = Z[:, 0] = Z[:, -1] = 0.0
    return Z


def _oracle_fill(N, mc, alpha, beta, Z):
    disc = orc.Discretisation2D(N, mc, alpha, beta)
    u = disc.filler(orc.interior(Z), np.zeros((N - 2) ** 2))
    return disc, orc.to_grid(u, np.zeros((N, N)))


def _run(lib, N, mc, alpha, beta, Z, precision, fill=None):
    with lib.Solver(N, mc, alpha, beta, precision=precision) as sv:
        if fill is not None:
            state = sv.tune_state()
            state[TUNE_FILL_MIXED] = fill
            sv.set_tune_state(state)
        out = _dev(np.full((N, N), 7.0))
        sv.submesh_solve(lib.MESH_HOLES_HOMOGENEOUS, _dev(Z), out)
        return out.cpu().numpy()


CASES = [
    # (N, mc, alpha, beta): n = 16 unless noted; mc = 4 is a tile of 4 of 128 holes
    (65, 4, (1.0, 1.0), (0.0, 0.0)),
    (129, 8, (0.8, 1.7), (2.5, -4.0)),
    (257, 16, (0.3, 1.2), (-6.0, 3.0)),
    (65, 4, (1.0, 0.05), (40.0, 0.0)),           # strongly anisotropic, convection-dominated
    (129, 16, (1.0, 1.0), (0.0, 0.0)),            # n = 8: block cyclic reduction kernel
]


@pytest.mark.parametrize("N,mc,alpha,beta", CASES)
def test_homogeneous_fill_matches_oracle(lib, N, mc, alpha, beta):
    Z = _skeleton_grid(N, N + mc)
    disc, ref = _oracle_fill(N, mc, alpha, beta, Z)
    holes = disc.P_ff_holes
    for prec, tol in ((lib.MIXED, 2e-5), (lib.FP64, 1e-12)):
        got = _run(lib, N, mc, alpha, beta, Z, prec)
        e = _relerr(holes @ orc.interior(got), holes @ orc.interior(ref))
        assert e <= tol, (prec, e)
        assert np.all(disc.P_ff_skel @ orc.interior(got) == 7.0)      # skeleton untouched
        assert np.all(got[0, :] == 7.0) and np.all(got[:, -1] == 7.0)  # boundary untouched


def test_tensor_core_and_reduction_fill_agree_with_oracle(lib):
    N, mc, alpha, beta = 129, 8, (0.8, 1.7), (2.5, -4.0)
    Z = _skeleton_grid(N, 5)
    disc, ref = _oracle_fill(N, mc, alpha, beta, Z)
    holes = disc.P_ff_holes
    r = holes @ orc.interior(ref)
    tc = holes @ orc.interior(_run(lib, N, mc, alpha, beta, Z, lib.MIXED, FILL_TC))
    bcr = holes @ orc.interior(_run(lib, N, mc, alpha, beta, Z, lib.MIXED, FILL_BCR8))
    assert _relerr(tc, r) <= 2e-5 and _relerr(bcr, r) <= 2e-5
    assert not np.array_equal(tc, bcr)          # two kernels really ran


def test_zero_ring_gives_zero_holes(lib):
    N, mc = 129, 8
    got = _run(lib, N, mc, (1.0, 1.0), (0.0, 0.0), np.zeros((N, N)), lib.MIXED)
    disc = orc.Discretisation2D(N, mc, (1.0, 1.0), (0.0, 0.0))
    assert np.all(disc.P_ff_holes @ orc.interior(got) == 0.0)


def test_full_size_holes_sampled_against_oracle(lib):
    """4097^2, 256 x 256 holes (two tiles of 128 per hole row)."""
    N, mc, alpha, beta = 4097, 256, (0.8, 1.7), (2.5, -4.0)
    Z = _skeleton_grid(N, 11)
    got = _run(lib, N, mc, alpha, beta, Z, lib.MIXED)
    # every hole equation, by the oracle's residual (zero source): r = -A u at hole points
    r, _ = orc.residual_grid(N, alpha, beta, np.zeros((N, N)), np.where(got == 7.0, Z, got))
    R = r.reshape(N - 2, N - 2) if r.ndim == 1 else r
    idx = np.arange(1, N - 1)
    hole_rows = (idx % 16) != 0
    Rh = R[np.ix_(hole_rows, hole_rows)]
    cc = 2.0 * (alpha[0] + alpha[1]) * (N - 1) ** 2
    assert np.max(np.abs(Rh)) <= 1e-5 * cc * np.max(np.abs(Z))
    # sampled holes re-solved by the oracle: the centre hole of a 49^2 grid (mc = 3)
    rng = np.random.default_rng(2)
    picks = [(0, 0), (255, 255), (127, 128), (128, 127)] + [tuple(rng.integers(0, 256, 2)) for _ in range(6)]
    for bi, bj in picks:
        x0, y0 = 16 * bi, 16 * bj
        S = np.zeros((49, 49))
        S[16:33, 16:33] = Z[y0:y0 + 17, x0:x0 + 17]
        S[17:32, 17:32] = 0.0
        # same operator on both grids needs the same h: rescale alpha/beta to the 49^2 spacing
        f = (N - 1) / (49 - 1)
        a2, b2 = (alpha[0] * f * f, alpha[1] * f * f), (beta[0] * f, beta[1] * f)
        disc2 = orc.Discretisation2D(49, 3, a2, b2)
        u2 = orc.to_grid(disc2.filler(orc.interior(S), np.zeros(47 * 47)), np.zeros((49, 49)))
        ref = u2[17:32, 17:32]
        mine = got[y0 + 1:y0 + 16, x0 + 1:x0 + 16]
        assert _relerr(mine, ref) <= 2e-5, (bi, bj, _relerr(mine, ref))
