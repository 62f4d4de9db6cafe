"""Independent numpy evaluation of the paper's model quantities.

Test infrastructure only.  Written straight from the definitions of
Sec. II-A and problem (eq7) of arXiv 1803.07772, with no code shared with the
oracle or the CUDA solver.  Works on a dense power tensor
``p[n, m, k]`` (0 where user k is not served by RRH m on subcarrier n).
"""
from __future__ import annotations

import numpy as np


def dense_power(S: np.ndarray, p: np.ndarray, K: int) -> np.ndarray:
    """Scatter per-slot powers (S[n,m,s] user ids, -1 empty) into p[n, m, k]."""
    N, M, l = S.shape
    out = np.zeros((N, M, K))
    for n in range(N):
        for m in range(M):
            for s in range(l):
                k = S[n, m, s]
                if k >= 0:
                    out[n, m, k] = p[n, m, s]
    return out


def sinr(G: np.ndarray, P: np.ndarray, sigma: float) -> np.ndarray:
    """gamma[n, m, k] of Sec. II-A for every served link (0 elsewhere).

    User k on (m, n) hears every other served user i of the same (m, n) whose
    gain Gamma_{m,i} is larger (strict order, lower index first on ties),
    received through Gamma_{m,k}, plus every link of the other RRHs on n,
    received through Gamma_{j,k}.
    """
    G = G.astype(np.float64)
    N, M, K = G.shape
    out = np.zeros((N, M, K))
    for n in range(N):
        for m in range(M):
            for k in range(K):
                if P[n, m, k] <= 0:
                    continue
                intra = 0.0
                for i in range(K):
                    if i == k or P[n, m, i] <= 0:
                        continue
                    if G[n, m, i] > G[n, m, k] or (G[n, m, i] == G[n, m, k] and i < k):
                        intra += P[n, m, i]
                inter = 0.0
                for j in range(M):
                    if j != m:
                        inter += G[n, j, k] * P[n, j, :].sum()
                out[n, m, k] = P[n, m, k] * G[n, m, k] / (sigma + G[n, m, k] * intra + inter)
    return out


def rates(G, P, sigma, w=None):
    """Per-user rate r_k = sum_m w_{m,k} sum_n log2(1 + gamma) (bits/s/Hz)."""
    g = sinr(G, P, sigma)
    N, M, K = G.shape
    W = np.ones((M, K)) if w is None else np.asarray(w, dtype=np.float64).reshape(M, K)
    return (np.log2(1.0 + g) * W[None, :, :]).sum(axis=(0, 1))


def R_P(inst, P: np.ndarray):
    """Weighted elastic sum rate R of problem (eq7) and the consumed power P of
    the Sec. II-A power model: fronthaul and circuit power of every RRH plus
    eta_m times the transmit power of every user it serves."""
    sigma = inst.N0_w_per_hz * inst.Bn_hz
    Ke = inst.K - inst.Ks
    r = rates(inst.G, P, sigma, inst.w)
    R = r[:Ke].sum()
    Ptot = (inst.Pc + inst.Pf).sum() + (inst.eta[None, :, None] * P).sum()
    return R, Ptot


def psi(inst) -> np.ndarray:
    """Minimum rates of C9, solved here as the smaller root of (Eq6b) with numpy.roots."""
    out = []
    for T, lam in zip(inst.T_s, inst.lambda_pps):
        roots = np.roots([lam, -(2.0 + 2.0 * lam * T), 2.0 * T])
        x = min(r.real for r in roots)
        out.append(inst.zbar_bits / (x * inst.Bn_hz))
    return np.asarray(out)


def omega_bar(inst, P: np.ndarray, n: int, m: int, ka: int, kb: int) -> float:
    """C14 divided by Gamma_{m,ka} Gamma_{m,kb} for the pair (ka stronger, kb weaker)."""
    G = inst.G.astype(np.float64)
    sigma = inst.N0_w_per_hz * inst.Bn_hz
    xa = sum(G[n, j, ka] * P[n, j, :].sum() for j in range(inst.M) if j != m)
    xb = sum(G[n, j, kb] * P[n, j, :].sum() for j in range(inst.M) if j != m)
    return (sigma + xa) / G[n, m, ka] - (sigma + xb) / G[n, m, kb]
