"""CPU pins of the host real Schur form used by the 3D plane-family solves.

The plane systems of the 3D extension (Section 3.5) couple one coarse axis
with two fine ones; the coarse-axis operator T_H (tridiagonal, N_c x N_c) is
brought to real Schur form T_H = Q S Q^T, so that in the basis of Q a plane
system becomes a back-substitution over S's diagonal blocks.  Checked here
against the definition and against numpy's eigenvalue routine: Q orthogonal,
Q S Q^T = A, S quasi upper triangular with 2 x 2 blocks exactly where the
eigenvalues are complex, and the eigenvalues of the blocks equal numpy's
within the Bauer-Fike bound of the eigenvector condition number.
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


def _schur(lib, A):
    n = A.shape[0]
    a = np.ascontiguousarray(A, dtype=np.float64)
    Q = np.zeros((n, n))
    S = np.zeros((n, n))
    p = lambda x: x.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    assert lib.asdsm_real_schur(n, p(a), p(Q), p(S)) == 0
    return Q, S


def _block_eigs(S):
    n = S.shape[0]
    eigs, i, blocks = [], 0, []
    while i < n:
        if i + 1 < n and S[i + 1, i] != 0.0:
            B = S[i:i + 2, i:i + 2]
            tr, det = B[0, 0] + B[1, 1], B[0, 0] * B[1, 1] - B[0, 1] * B[1, 0]
            disc = tr * tr / 4 - det
            assert disc < 0, "a 2 x 2 block with real eigenvalues was left unsplit"
            eigs += [tr / 2 + 1j * np.sqrt(-disc), tr / 2 - 1j * np.sqrt(-disc)]
            blocks.append(2)
            i += 2
        else:
            eigs.append(S[i, i] + 0j)
            blocks.append(1)
            i += 1
    return np.array(eigs), blocks


def _coarse_axis_operator(Nc, alpha, beta):
    H = 1.0 / (Nc + 1)
    lo, di, up = -alpha / H**2 - beta / (2 * H), 2 * alpha / H**2, -alpha / H**2 + beta / (2 * H)
    return np.diag(np.full(Nc, di)) + np.diag(np.full(Nc - 1, lo), -1) + np.diag(np.full(Nc - 1, up), 1)


def _check(lib, A):
    n = A.shape[0]
    Q, S = _schur(lib, A)
    scale = np.abs(A).max()
    assert np.abs(Q.T @ Q - np.eye(n)).max() <= 1e-13 * n
    assert np.abs(Q @ S @ Q.T - A).max() <= 1e-13 * n * scale
    assert np.all(np.tril(S, -2) == 0.0)
    sub = np.diag(S, -1)
    assert not np.any((sub[:-1] != 0) & (sub[1:] != 0)), "two adjacent subdiagonal entries"
    got, _ = _block_eigs(S)
    want, V = np.linalg.eig(A)
    # Both spectra come from backward-stable methods: by Bauer-Fike they agree to
    # about cond(V) * eps * ||A|| (huge for the strongly non-normal operators).
    tol = 1e-13 * n * scale * min(np.linalg.cond(V), 1e12)
    rest = list(want)
    for z in got:                                   # greedy nearest pairing of the two multisets
        k = int(np.argmin([abs(z - w) for w in rest]))
        assert abs(z - rest[k]) <= max(tol, 1e-13 * scale), (z, rest[k], tol)
        rest.pop(k)
    return S


@pytest.mark.parametrize("Nc,alpha,beta", [(15, 1.0, 0.0), (15, 0.5, 3.0), (15, 0.01, 5.0), (15, 0.01, -5.0),
                                            (15, 0.1562, 5.0), (31, 0.05, 2.0), (7, 0.2, -9.0), (63, 0.01, 4.0),
                                            (1, 0.3, 1.0), (2, 0.01, 5.0), (3, 0.02, 1.0)])
def test_schur_of_coarse_axis_operators(lib, Nc, alpha, beta):
    """Cell Peclet numbers beta H / (2 alpha) below 1 (real spectrum), above 1
    (complex pairs) and close to 1 (nearly defective)."""
    S = _check(lib, _coarse_axis_operator(Nc, alpha, beta))
    pe = abs(beta) / (Nc + 1) / (2 * alpha)
    _, blocks = _block_eigs(S)
    if pe < 0.999:
        assert all(b == 1 for b in blocks)          # real eigenvalues only
    if pe > 1.001 and Nc >= 2:
        assert any(b == 2 for b in blocks)


@pytest.mark.parametrize("n,seed", [(2, 0), (3, 1), (5, 2), (12, 3), (40, 4)])
def test_schur_of_random_hessenberg_matrices(lib, n, seed):
    A = np.triu(np.random.default_rng(seed).normal(size=(n, n)), -1)
    _check(lib, A)


def test_planted_wrong_rotation_sign_is_caught(lib):
    """A Schur form whose Q lost a sign flip no longer reconstructs A: the
    reconstruction check is what fixes the orientation of Q."""
    A = _coarse_axis_operator(15, 0.01, 5.0)
    Q, S = _schur(lib, A)
    Qb = Q.copy()
    Qb[:, 3] *= -1.0
    Qb[:, 4] *= -1.0 if S[4, 3] == 0 else 1.0
    assert np.abs(Qb @ S @ Qb.T - A).max() > 1e-6 * np.abs(A).max()
