"""Failure detection on the GPU without a GPU fault.

The tensor-core kernels hand work between warps through mbarriers, and every
wait is bounded: when one runs out the kernel stops, frees its tensor memory
and sets a flag that the solve reports as ASDSM_ERR_CUDA.  Here a self-test
kernel takes tensor memory and waits, with a 20 ms bound, on an mbarrier
that nothing arrives at (no copy or MMA in flight); the test checks that the
status comes back to the host, that it is sticky for the handle, and that the
GPU context still serves a new handle's solve.
"""
import time

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


def test_a_wait_that_runs_out_is_reported_and_the_context_survives(lib):
    p = wl.random_fourier_2d(129, 1)
    raw = lib.load()
    sv = lib.Solver(129, 8, p.alpha, p.beta, precision=lib.MIXED, tol=1e-10, max_sweeps=400)
    t0 = time.time()
    rc = raw.asdsm_selftest_wait_timeout(sv._h, 20_000_000)
    elapsed = time.time() - t0
    assert rc == lib.ERR_CUDA
    assert b"timed out" in raw.asdsm_last_error()
    assert elapsed < 10.0
    assert raw.asdsm_selftest_wait_timeout(sv._h, 0) == lib.ERR_INVALID        # the bound must be positive
    with pytest.raises(lib.AsdsmError) as ei:                                   # sticky for this handle
        sv.solve(_dev(p.s), _dev(p.g))
    assert ei.value.code == lib.ERR_CUDA
    sv.close()
    with lib.Solver(129, 8, p.alpha, p.beta, precision=lib.MIXED, tol=1e-10, max_sweeps=400) as fresh:
        u = _dev(p.g)
        res = fresh.solve(_dev(p.s), u)
    assert res.status == lib.OK
    r, b = orc.residual_grid(129, p.alpha, p.beta, p.s, u.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(b) <= 1.01e-10
