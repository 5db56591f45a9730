"""GPU test of asdsm_residual_noalloc, the residual entry point that allocates
no device memory (for callers that cannot call cudaMalloc: services whose
device memory belongs to their own pool allocator, loops that must not stall
on an allocation).  It is called through the C ABI and compared with the
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


@pytest.mark.parametrize("N", [3, 17, 20, 65])
def test_noalloc_residual_3d_matches_the_3d_oracle(N):
    """d = 3: the 7-point residual of the 3D extension against the FP64 3D
    oracle's operator and Dirichlet lifting (N = 3: one interior point;
    N = 20: a size that no coarse mesh divides)."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_01163_gb300 import asdsm
    from oracle import asdsm3d as o3
    alpha, beta = (0.7, 1.3, 0.4), (2.0, -3.0, 1.0)
    rng = np.random.default_rng(N)
    U = rng.normal(size=(N, N, N))
    S = rng.normal(size=(N, N, N))
    M, Nf, h = N - 1, N - 2, 1.0 / (N - 1)
    fine = np.arange(1, M)
    pts = o3.Meshes3D._product(fine, fine, fine)
    b = o3.rhs_on_mesh(pts, (h, h, h), alpha, beta, S, U, M)
    r_ref = b - o3.operator_3d(Nf, h, Nf, h, Nf, h, alpha, beta) @ o3.interior(U)
    rel_ref = np.linalg.norm(r_ref) / np.linalg.norm(b)
    s = torch.tensor(S, dtype=torch.float64, device="cuda")
    u = torch.tensor(U, dtype=torch.float64, device="cuda")
    r = torch.full_like(u, 5.0)
    rel = asdsm.residual_noalloc(N, alpha, beta, s, u, r)
    got = r.cpu().numpy()
    scale = (2 * sum(alpha) / h**2 * 2 + sum(abs(x) for x in beta) / h) * np.abs(U).max() + np.abs(S).max()
    assert np.abs(o3.interior(got) - r_ref).max() <= 1e-14 * scale
    assert abs(rel - rel_ref) <= 1e-12 * rel_ref
    ring = np.ones((N, N, N), dtype=bool)
    ring[1:-1, 1:-1, 1:-1] = False
    assert np.all(got[ring] == 5.0)                    # boundary untouched


def test_noalloc_3d_rejects_invalid_descriptions():
    import torch
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_01163_gb300 import asdsm
    s = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        asdsm.residual_noalloc(2050, (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), s, s)
    with pytest.raises(RuntimeError):
        asdsm.residual_noalloc(17, (1.0, 1.0, 0.0), (0.0, 0.0, 0.0), s, s)
