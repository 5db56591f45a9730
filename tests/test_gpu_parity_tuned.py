"""End-to-end parity of a tuned mixed-precision solve at a production shape.

A 1025 x 1025 instance of the random-coefficient workload with mc = 64 (holes
of 15 x 15, so the sweeps fill them with the tensor-core Filler), launch
shapes autotuned for both precisions as the benchmark does, solved to 1e-10
and judged by the oracle alone: its FP64 fine residual of the returned grid,
and the distance to its direct solve of the fine system (u_ff = A_ff^{-1} b_ff,
the fixed point of ASDSM, Prop. 3.1), bounded by the condition number times
the residual.
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


@pytest.mark.parametrize("seed", [0, 3])
def test_tuned_mixed_solve_at_1025_matches_the_oracle(lib, seed):
    import torch
    N, mc = 1025, 64
    p = wl.random_fourier_2d(N, seed)
    s = torch.tensor(p.s, dtype=torch.float64, device="cuda")
    u = torch.tensor(p.g, dtype=torch.float64, device="cuda")
    with lib.Solver(N, mc, p.alpha, p.beta, precision=lib.MIXED, tol=1e-10, max_sweeps=600) as sv:
        sv.autotune(lib.MIXED)
        sv.autotune(lib.FP64)
        res = sv.solve(s, u)
        assert res.status == lib.OK, res.stats
        lib_fp64 = sv.residual(s, u)
    ug = u.cpu().numpy()
    r, b = orc.residual_grid(N, p.alpha, p.beta, p.s, ug)
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1.01e-10, rel
    assert abs(lib_fp64 - rel) <= 1e-3 * rel          # the library's FP64 residual agrees with the oracle's
    assert abs(res.stats["rel_res_fp64"] - rel) <= 1e-3 * rel   # and so does the solve's own FP64 check
    off = np.arange(1, N - 1) % ((N - 1) // mc) != 0      # fine indices strictly inside the holes
    hole = np.abs(r.reshape(N - 2, N - 2)[np.ix_(off, off)]).max()
    h = 1.0 / (N - 1)
    stencil_scale = 2 * (p.alpha[0] + p.alpha[1]) / h**2 * np.abs(ug).max()   # size of the terms of A u
    assert abs(res.stats["hole_res_max"] - hole) <= 1e-3 * hole + 1e-14 * stencil_scale
    disc = orc.Discretisation2D(N, mc, p.alpha, p.beta)
    u_ff = disc.solve_fine(disc.rhs(p.s, p.g)[0])
    err = np.linalg.norm(orc.interior(ug) - u_ff) / np.linalg.norm(u_ff)
    kappa = 4.0 / (np.pi**2 * h**2) * max(p.alpha) / min(p.alpha)
    print(f"seed {seed}: {res.stats['sweeps']} sweeps, oracle rel residual {rel:.3e}, "
          f"rel error to u_ff {err:.3e} (bound {kappa * rel:.1e})")
    assert err <= kappa * rel
