"""Learned warm start: training targets from cold solves, the training loop
and the warm solve.  Host-side orchestration only; the features, the network's
forward and backward and the solves all run in the library's CUDA kernels.

Rows, features and the output encoding are those of ``include/hcran.h``
(``hcran_warm_rows``): one row per slot of the cold initial selection.
Targets of a row (slot of user k on RRH m, subcarrier n) from a cold solve:
  y0 = log(p* / mask_m), p* = the final power of (m, k, n) when that link is
       still selected at the end, else the floor 1e-9 mask_m;
  y1 = log(xi*_m ln2 mask_m + 1e-3), the inverse of the xi' decoding;
  y2 = log zeta*_k for a streaming user (no target for an elastic one).
"""
from __future__ import annotations

import math

import numpy as np

XI_EPS = 1e-3
P_FLOOR = 1e-9
TRAIN_SEED_BASE = 10_000_000  # training instances: seeds disjoint from every evaluated workload


def _al4(x: int) -> int:
    return (x + 3) // 4 * 4


def row_offsets(insts):
    """First warm-start row of every instance (the library's order)."""
    offs, o = [], 0
    for inst in insts:
        offs.append(o)
        o += inst.N * _al4(inst.M * inst.l)
    return np.asarray(offs, np.int64), o


def cold_point_outputs(insts):
    """Network outputs that encode the cold initial point (p = mask / l,
    xi' = 0, zeta' = 1): a warm solve from them is the cold solve."""
    offs, rows = row_offsets(insts)
    y = np.zeros((rows, 16), np.float32)
    for inst, o in zip(insts, offs):
        n = inst.N * _al4(inst.M * inst.l)
        y[o:o + n, 0] = math.log(1.0 / inst.l)
        y[o:o + n, 1] = -30.0
        y[o:o + n, 2] = 0.0
    return y


def targets(insts, initial, final):
    """Training targets and masks ([rows][16] float32) from the initial
    selection (``Solver.get`` after ``warm_features``) and the cold solution."""
    offs, rows = row_offsets(insts)
    y = np.zeros((rows, 16), np.float32)
    mk = np.zeros((rows, 16), np.float32)
    for inst, o, s0, fin in zip(insts, offs, initial, final):
        M, N, l, Ke = inst.M, inst.N, inst.l, inst.K - inst.Ks
        Up = _al4(M * l)
        mask = np.asarray(inst.pmax, np.float64) / N
        S0, S1, p1 = s0["S"], fin["S"], fin["p"]
        xi, zeta = np.asarray(fin["xi"], np.float64), np.asarray(fin["zeta"], np.float64)
        n_idx, m_idx, s_idx = np.nonzero(S0 >= 0)
        k = S0[n_idx, m_idx, s_idx]
        # final power of the same (m, k, n), floor when the link was dropped
        hit = S1[n_idx, m_idx, :] == k[:, None]
        p = np.where(hit.any(axis=1), np.sum(np.where(hit, p1[n_idx, m_idx, :], 0.0), axis=1),
                     P_FLOOR * mask[m_idx])
        r = o + n_idx * Up + m_idx * l + s_idx
        y[r, 0] = np.log(np.maximum(p, P_FLOOR * mask[m_idx]) / mask[m_idx])
        y[r, 1] = np.log(xi[m_idx] * math.log(2.0) * mask[m_idx] + XI_EPS)
        mk[r, 0] = 1.0
        mk[r, 1] = 1.0
        st = k >= Ke
        if st.any():
            y[r[st], 2] = np.log(zeta[k[st] - Ke])
            mk[r[st], 2] = 1.0
    return y, mk


def build_dataset(solver, gains, insts, tol):
    """Features, targets and masks of the selected rows of a batch of cold solves."""
    import torch
    F = solver.warm_features(gains)
    initial = [solver.get(i) for i in range(len(insts))]
    solver.solve(gains, tol)
    final = [solver.get(i) for i in range(len(insts))]
    y, mk = targets(insts, initial, final)
    keep = np.nonzero(mk[:, 0] > 0)[0]
    idx = torch.from_numpy(keep).to(F.device)
    return F[idx].contiguous(), torch.from_numpy(y[keep]).to(F.device), torch.from_numpy(mk[keep]).to(F.device)


def train(net, X, Y, Mk, epochs: int = 4, batch: int = 8192, lr: float = 1e-3, seed: int = 0, stream=None):
    """Adam on the masked squared error; returns the mean loss of every epoch."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    R = X.shape[0]
    batch = min(batch, net.max_rows, R)
    out = torch.empty((batch, 16), dtype=torch.float32, device=X.device)
    loss = torch.zeros(1, dtype=torch.float32, device=X.device)
    hist = []
    for _ in range(epochs):
        perm = torch.randperm(R, generator=g).to(X.device)
        tot, nb = 0.0, 0
        for b0 in range(0, R - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            xb, yb, mb = X[idx].contiguous(), Y[idx].contiguous(), Mk[idx].contiguous()
            net.forward(xb, out, stream)
            net.loss_grad(out, yb, mb, loss, 3, stream)
            net.backward(xb, stream)
            net.adam(lr, stream=stream)
            tot += float(loss.item())
            nb += 1
        hist.append(tot / max(nb, 1))
    return hist


def warm_solve(solver, net, gains, tol, features=None, out=None):
    """Features of the initial selection -> network -> solve from its outputs."""
    import torch
    F = solver.warm_features(gains, features)
    if out is None:
        out = torch.empty((F.shape[0], 16), dtype=torch.float32, device=F.device)
    net.forward(F, out, solver.stream)
    solver.solve_warm(gains, tol, out)
    return out
