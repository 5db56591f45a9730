"""CPU pins of the dense tail of the block cyclic reduction (host FP64).

The anisotropic systems of eq. (2.4) are block tridiagonal,
    a x_{i-1} + (d I + T) x_i + c x_{i+1} = f_i,  T = tridiag(tl, td, tu),
and the FP32 solves replace the last levels of their cyclic reduction by one
dense map D over the rt rows i = k (R+1)/(rt+1).  For a right-hand side that
vanishes off those rows, the reduction leaves it unchanged on them, so D must
equal the restriction of the system's inverse to those rows: checked here
against a dense solve of the assembled system (numpy), for diffusion- and
advection-dominated coefficients, several sizes and tail lengths.  A wrong
row spacing, a transposed block or a dropped neighbour term fails it.
"""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as ge
    ge.build()
    from paper_2303_01163_gb300 import asdsm
    return asdsm.load()


def _tail(lib, R, C, coef, rt):
    D = np.zeros((rt * C) ** 2)
    c = np.ascontiguousarray(coef, dtype=np.float64)
    p = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    rc = lib.asdsm_bcr_tail_map(R, C, p(c), rt, p(D))
    return rc, D.reshape(rt * C, rt * C)


def _assemble(R, C, coef):
    a, d, c, tl, td, tu = coef
    T = np.diag(np.full(C, td)) + np.diag(np.full(C - 1, tl), -1) + np.diag(np.full(C - 1, tu), 1)
    A = np.kron(np.eye(R), d * np.eye(C) + T)
    A += np.kron(np.eye(R, k=-1), a * np.eye(C)) + np.kron(np.eye(R, k=1), c * np.eye(C))
    return A


def _coef(alpha_r, beta_r, h, alpha_c, beta_c, H):
    """Rows along a fine axis of spacing h, columns along a coarse axis of spacing H (eq. 2.4)."""
    lo, di, up = -alpha_r / h**2 - beta_r / (2 * h), 2 * alpha_r / h**2, -alpha_r / h**2 + beta_r / (2 * h)
    tl, td, tu = -alpha_c / H**2 - beta_c / (2 * H), 2 * alpha_c / H**2, -alpha_c / H**2 + beta_c / (2 * H)
    return (lo, di, up, tl, td, tu)


@pytest.mark.parametrize("R,C,rt", [(15, 5, 7), (31, 1, 7), (31, 6, 3), (63, 9, 7), (63, 4, 15), (7, 3, 7)])
@pytest.mark.parametrize("kind", ["diffusion", "advection"])
def test_tail_map_is_the_inverse_on_the_tail_rows(lib, R, C, rt, kind):
    h, H = 1.0 / (R + 1), 1.0 / (C + 1)
    coef = _coef(0.7, 0.3, h, 1.3, -0.5, H) if kind == "diffusion" else _coef(0.02, 5.0, h, 0.05, -4.0, H)
    rc, D = _tail(lib, R, C, coef, rt)
    assert rc == 0
    A = _assemble(R, C, coef)
    s0 = (R + 1) // (rt + 1)
    rows = [k * s0 for k in range(1, rt + 1)]                    # 1-based tail rows
    idx = np.concatenate([np.arange((i - 1) * C, i * C) for i in rows])
    rng = np.random.default_rng(R * 100 + C)
    for _ in range(3):
        f = np.zeros(R * C)
        f[idx] = rng.standard_normal(len(idx))
        x = np.linalg.solve(A, f)
        got = D @ f[idx]
        assert np.allclose(got, x[idx], rtol=1e-11, atol=1e-13 * np.abs(x).max())


def test_tail_map_rejects_bad_sizes(lib):
    coef = np.ascontiguousarray(_coef(1.0, 0.0, 1 / 16, 1.0, 0.0, 1 / 4), dtype=np.float64)
    D = np.zeros(100 * 100)                      # room for any map these sizes could describe
    p = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    # rt not of the form 2^t - 1; rt > R; R not 2^L - 1; no columns; no tail rows; a map
    # too large to hold (rt C > 8192)
    for R, C, rt in [(15, 3, 5), (15, 3, 31), (14, 3, 7), (15, 0, 7), (15, 3, 0), (32767, 512, 31)]:
        assert lib.asdsm_bcr_tail_map(R, C, p(coef), rt, p(D)) != 0, (R, C, rt)
