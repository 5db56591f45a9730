"""Training the learned correction on pairs that ASDSM itself generates.

A pair is (features, target) for an iterate u_k of a solve: features are the
network's six input channels [r, e (each scaled to unit RMS over the
interior), alpha_x, alpha_y, beta_x h, beta_y h], with r = s - A u_k and e the
ASDSM correction of that sweep (asdsm_correction); the target is the error
u* - u_k of the iterate, scaled to unit RMS, where u* is the converged
solution.  Crops of the full grids make the training batches; training runs
the library's forward, backward and Adam kernels (asdsm_cnn_*).
"""
from __future__ import annotations

import numpy as np

from . import asdsm


def make_pairs(problems, mc_of, sweeps=(0, 2, 4, 8, 12, 16, 24), crop=64, crops_per_iterate=8, seed=0):
    """Returns device tensors X (P, 6, crop, crop), T (P, 1, crop, crop) and the
    loss weights W (P, 1, crop, crop): the solver uses only the network's
    skeleton values, so the loss counts the skeleton points (weights scaled to
    mean 1 over each crop)."""
    import torch
    rng = np.random.default_rng(seed)
    Xs, Ts, Ws = [], [], []
    for p in problems:
        N, mc = p.N, mc_of(p.N)
        s = torch.tensor(p.s, dtype=torch.float64, device="cuda")
        g = torch.tensor(p.g, dtype=torch.float64, device="cuda")
        ref = asdsm.Solver(N, mc, p.alpha, p.beta, precision=asdsm.FP64, tol=1e-13, max_sweeps=2000)
        ustar = g.clone()
        ref.solve(s, ustar)
        ref.close()
        sv = asdsm.Solver(N, mc, p.alpha, p.beta, precision=asdsm.MIXED, tol=1e-30, max_sweeps=1, stagnation_window=0)
        n_hole = (N - 1) // mc
        jj, ii = np.meshgrid(np.arange(N), np.arange(N), indexing="ij")
        interior = (ii > 0) & (ii < N - 1) & (jj > 0) & (jj < N - 1)
        skel = torch.tensor((interior & ((ii % n_hole == 0) | (jj % n_hole == 0))).astype(np.float32), device="cuda")
        h = 1.0 / (N - 1)
        c = torch.tensor([p.alpha[0], p.alpha[1], p.beta[0] * h, p.beta[1] * h], dtype=torch.float32, device="cuda")
        for k in sweeps:
            sv.set_opts(max_sweeps=k)
            uk = g.clone()
            sv.solve(s, uk)
            r, e = sv.correction(s, uk, k)
            err = (ustar - uk).to(torch.float32)
            n = float((N - 2) ** 2)

            def unit(a):
                nrm = float(torch.linalg.vector_norm(a))
                return a * (np.sqrt(n) / nrm) if nrm > 0 else a

            feats = torch.stack([unit(r), unit(e)] + [c[q].expand(N, N) for q in range(4)])
            tgt = unit(err)[None]
            for _ in range(crops_per_iterate):
                i0 = int(rng.integers(0, N - crop + 1))
                j0 = int(rng.integers(0, N - crop + 1))
                Xs.append(feats[:, i0:i0 + crop, j0:j0 + crop])
                Ts.append(tgt[:, i0:i0 + crop, j0:j0 + crop])
                wc = skel[i0:i0 + crop, j0:j0 + crop]
                Ws.append((wc * (wc.numel() / max(float(wc.sum()), 1.0)))[None])
        sv.close()
    return torch.stack(Xs).contiguous(), torch.stack(Ts).contiguous(), torch.stack(Ws).contiguous()


def train(X, T, params, steps=1500, batch=32, lr=1e-3, seed=0, bf16=True, W=None):
    """Adam on random mini-batches (per-pixel loss weights W if given); returns (net, losses)."""
    import torch
    net = asdsm.Cnn(params, bf16=bf16)
    rng = np.random.default_rng(seed)
    losses = []
    P = X.shape[0]
    for it in range(steps):
        idx = torch.as_tensor(rng.choice(P, size=min(batch, P), replace=False), device=X.device)
        xb = X.index_select(0, idx).contiguous()
        tb = T.index_select(0, idx).contiguous()
        wb = W.index_select(0, idx).contiguous() if W is not None else None
        loss, _ = net.backward(xb, tb, weights=wb)
        net.adam(lr)
        want = it % 50 == 0 or it == steps - 1
        if want:
            losses.append(loss)
    return net, losses
