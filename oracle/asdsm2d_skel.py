"""FP64 CPU oracle for skeleton-only ASDSM in 2D (K. Trotti, arXiv
2303.01163, Section 3.3, the remarks on the sparsity of the residual and on
storing only the skeleton and the points next to it).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import this
module: only ``tests/`` do.  It shares no code with the CUDA path.

After Algorithm 3 the residual vanishes in every hole (Prop. 3.1), and every
later correction is harmonic in the holes (its Filler has zero source), so
the iterate is fixed by its skeleton values u_s: its hole values are
u_h = A_hh^{-1} (b_h - A_hs u_s).  The residual lives on the skeleton rows,
and a skeleton row reaches, besides skeleton points, only the ring (the hole
points next to the skeleton):
    r_s = b_s - A_ss u_s - A_sR u_R,   u_R = the ring rows of u_h.
This module runs Algorithm 4 on (u_s, u_R) alone, O(N_c N_f) values, and
fills the holes once at the end.  Its sweeps are those of ``asdsm2d.asdsm``
in exact arithmetic; the hole-residual correction R18 has nothing to act on
here (no hole values are kept), so it is left out.

Reading:

R30 The ring is every hole point with a skeleton point among its four
    neighbours; the correction's ring values are the ring rows of Algorithm 3
    with zero source applied to the correction's skeleton values.
"""
from __future__ import annotations

import numpy as np

from oracle import asdsm2d as orc


class SkeletonOnly:
    """The skeleton-and-ring operators of one Discretisation2D."""

    def __init__(self, disc: orc.Discretisation2D):
        self.disc = disc
        m = disc.m
        N, n = m.N, m.n
        i, j = m.holes[:, 0], m.holes[:, 1]
        near = (i % n == 1) | (i % n == n - 1) | (j % n == 1) | (j % n == n - 1)
        self.ring = m.holes[near]
        P_skel, P_holes = disc.P_ff_skel, disc.P_ff_holes
        self.P_ring = orc.projector(self.ring, m.ff, N)
        self.P_holes_ring = orc.projector(self.ring, m.holes, N)
        A_s = P_skel @ disc.A_ff                       # skeleton rows of A_ff
        self.A_ss = (A_s @ P_skel.T).tocsr()
        self.A_sR = (A_s @ self.P_ring.T).tocsr()
        self.A_hs = (P_holes @ disc.A_ff @ P_skel.T).tocsr()
        # a skeleton row touches only skeleton and ring points
        rest = A_s - self.A_ss @ P_skel - self.A_sR @ self.P_ring
        assert abs(rest).max() == 0.0 if rest.nnz else True

    def hole_values(self, u_s, b_h):
        """u_h = A_hh^{-1} (b_h - A_hs u_s): Algorithm 3 from the skeleton alone."""
        return self.disc.lu_holes.solve(b_h - self.A_hs @ u_s)

    def ring_values(self, u_s, b_h):
        return self.P_holes_ring @ self.hole_values(u_s, b_h)

    def residual(self, b_s, u_s, u_R):
        return b_s - self.A_ss @ u_s - self.A_sR @ u_R

    def correction(self, r_s, choice):
        """The correction's skeleton and ring values: Algorithms 1-2 on the
        projected residual (zero in the holes), then R30."""
        d = self.disc
        r = d.P_ff_skel.T @ r_s
        u_fc, u_cf = orc.normalised_families(d.lu_fc.solve(d.P_ff_fc @ r), d.lu_cf.solve(d.P_ff_cf @ r))
        e_s = d.P_ff_skel @ d.skeleton(u_fc, u_cf, None, choice)
        return e_s, self.ring_values(e_s, np.zeros(d.P_ff_holes.shape[0]))


def asdsm_skeleton_only(disc: orc.Discretisation2D, b, *, tol=1e-10, max_sweeps=200, accel_m=1, seed=0,
                        stagnation_window=10, stagnation_factor=1e-3):
    """Algorithm 4 (R13-R15 as in asdsm2d) on the skeleton and ring values.

    Returns (u, info): u on the whole fine interior (the holes filled once at
    the end), info with the residual history, the steps, the stored-value
    count and the stop reason."""
    b_ff, b_fc, b_cf, b_cc = b
    so = SkeletonOnly(disc)
    b_s, b_h = disc.P_ff_skel @ b_ff, disc.P_ff_holes @ b_ff
    u0 = disc.initial_guess(b_ff, b_fc, b_cf, b_cc)
    u_s = disc.P_ff_skel @ u0
    u_R = so.ring_values(u_s, b_h)
    nb = np.linalg.norm(b_ff)
    hist, steps = [], []
    Z, Q = [], []
    status, k = "max_sweeps", 0
    while True:
        r_s = so.residual(b_s, u_s, u_R)
        rel = np.linalg.norm(r_s) / nb if nb > 0 else np.linalg.norm(r_s)
        hist.append(rel)
        if rel <= tol:
            status = "converged"
            break
        if k >= max_sweeps:
            break
        if orc.stagnated(hist, stagnation_window, stagnation_factor):
            status = "stagnated"
            break
        e_s, e_R = so.correction(r_s, orc.choice_bit(seed, k))
        q = so.A_ss @ e_s + so.A_sR @ e_R
        if accel_m == 1:
            qq = q @ q
            s_hat = max(0.0, (r_s @ q) / qq) if qq > 0 else 0.0
            u_s, u_R = u_s + s_hat * e_s, u_R + s_hat * e_R
            steps.append(s_hat)
        else:
            e = np.concatenate([e_s, e_R])
            for zj, qj in zip(Z, Q):
                beta_j = q @ qj
                q = q - beta_j * qj
                e = e - beta_j * zj
            nq = np.linalg.norm(q)
            if nq > 0:
                q, e = q / nq, e / nq
                a = r_s @ q
                u_s, u_R = u_s + a * e[:len(e_s)], u_R + a * e[len(e_s):]
                Z.append(e)
                Q.append(q)
                steps.append(a)
            else:
                steps.append(0.0)
            if len(Z) >= accel_m:
                Z, Q = [], []
        k += 1
    u = disc.P_ff_skel.T @ u_s + disc.P_ff_holes.T @ so.hole_values(u_s, b_h)
    info = {"hist": hist, "steps": steps, "status": status, "sweeps": k,
            "stored": len(u_s) + len(u_R), "full": disc.P_ff_skel.shape[1]}
    return u, info
