"""GPU test of asdsm_residual_noalloc, the residual entry point that allocates
no device memory (for callers that cannot call cudaMalloc, e.g. during CUDA
graph capture).  It is called through the C ABI and compared with the
existing asdsm_residual on two calls in a row, within the tolerance of the
residual parity test.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _problem(N, seed):
    from paper_2303_01163_gb300 import workloads as wl
    p = wl.manufactured_sine_2d(N, alpha=(0.7, 1.3), beta=(2.0, -3.0)) if seed == 0 else wl.random_fourier_2d(N, seed)
    rng = np.random.default_rng(seed + 10)
    U = p.g.copy()
    U[1:-1, 1:-1] = rng.normal(size=(N - 2, N - 2))
    return p, U


@pytest.mark.parametrize("N,mc,seed", [(65, 8, 0), (257, 16, 3)])
def test_noalloc_residual_matches_the_handle_residual(N, mc, seed):
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_01163_gb300 import asdsm
    lib = asdsm.load()
    p, U = _problem(N, seed)
    s = torch.tensor(p.s, dtype=torch.float64, device="cuda")
    u = torch.tensor(U, dtype=torch.float64, device="cuda")
    with asdsm.Solver(N, mc, p.alpha, p.beta, precision=asdsm.FP64) as sv:
        r_ref = torch.zeros_like(u)
        rel_ref = sv.residual(s, u, r_ref)
    sten = (2 * p.alpha[0] + 2 * p.alpha[1]) * (N - 1) ** 2 * 2 + (abs(p.beta[0]) + abs(p.beta[1])) * (N - 1)
    scale = sten * np.abs(U).max() + np.abs(p.s).max()
    d = asdsm.Desc()
    d.d, d.n = 2, N
    for q in range(2):
        d.alpha[q], d.beta[q] = p.alpha[q], p.beta[q]
    stream = torch.cuda.current_stream()
    for call in range(2):                      # two calls in a row share the static scratch
        r = torch.full_like(u, 5.0)
        rel = ctypes.c_double()
        rc = lib.asdsm_residual_noalloc(ctypes.byref(d), ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(u.data_ptr()),
                                        ctypes.c_void_p(r.data_ptr()), ctypes.byref(rel),
                                        ctypes.c_void_p(stream.cuda_stream))
        assert rc == asdsm.OK, lib.asdsm_noalloc_last_error()
        torch.cuda.synchronize()
        got, ref = r.cpu().numpy(), r_ref.cpu().numpy()
        assert np.abs(got[1:-1, 1:-1] - ref[1:-1, 1:-1]).max() <= 1e-14 * scale
        assert np.all(got[0, :] == 5.0) and np.all(got[:, 0] == 5.0)       # ring untouched
        assert abs(rel.value - rel_ref) <= 1e-12 * rel_ref, (call, rel.value, rel_ref)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_01163_gb300 import asdsm
    lib = asdsm.load()
    d = asdsm.Desc()
    d.d, d.n = 2, 8194                          # one point beyond the stated maximum
    d.alpha[0] = d.alpha[1] = 1.0
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")   # never read: the size check comes first
    rel = ctypes.c_double()
    rc = lib.asdsm_residual_noalloc(ctypes.byref(d), ctypes.c_void_p(buf.data_ptr()), ctypes.c_void_p(buf.data_ptr()),
                                    None, ctypes.byref(rel), None)
    assert rc == asdsm.ERR_INVALID
    assert b"8193" in lib.asdsm_noalloc_last_error()
