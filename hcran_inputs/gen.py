"""Counter-based generator of synthetic H-CRAN channel realisations.

Channel model (Section II-A of arXiv 1803.07772 defines Gamma = |h|^2 per
(RRH, user, subcarrier); the numeric model below follows the workload
definitions used by this project, which replace the paper's d^-3 law):

* HPN (RRH 0) at the origin; the M-1 LPNs on a 200 m ring at angles 2*pi*j/(M-1)
  (the architectures of Sec. VI also place all M sites on the ring, or two
  sites at (-250 m, 0) and (250 m, 0); see `_sites`).
* Users uniform by area in a 500 m disk; link distance clamped to >= 10 m.
* Path loss 128.1 + 37.6 log10(d_km) dB, 8 dB log-normal shadowing i.i.d. per
  (RRH, user) and constant over subcarriers, Rayleigh power fading Exp(1)
  i.i.d. per (RRH, user, subcarrier).
* Gamma[n][m][k] = 10^(-(PL + X)/10) * chi, stored as float32 with k fastest.

Random numbers come from splitmix64 applied to a (seed, stream, index)
counter, so every value is reproducible from the seed alone and independent of
the order in which instances are drawn.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional, Sequence

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers (one independent counter sequence per quantity)
_S_SIZES, _S_RADIUS, _S_ANGLE, _S_SHADOW_A, _S_SHADOW_B, _S_FADING = range(6)


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_uniform(seed: int, stream: int, count: int) -> np.ndarray:
    """`count` doubles in (0, 1) from counter (seed, stream, 0..count-1)."""
    with np.errstate(over="ignore"):
        key = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64) * _GOLDEN
                   + np.uint64(stream))
        idx = np.arange(1, count + 1, dtype=np.uint64)
        x = _mix(key + idx * _GOLDEN)
    return ((x >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


@dataclasses.dataclass
class Instance:
    """One channel realisation plus the constants of its system model.

    Users 0..K-Ks-1 are elastic, K-Ks..K-1 streaming; RRH 0 is the HPN.
    """
    M: int
    N: int
    K: int
    Ks: int
    l: int
    pmax: np.ndarray          # [M] W
    eta: np.ndarray           # [M] power-amplifier factor
    Pc: np.ndarray            # [M] W circuit power
    Pf: np.ndarray            # [M] W fronthaul power
    Bn_hz: float              # subcarrier bandwidth
    N0_w_per_hz: float        # noise power spectral density
    T_s: np.ndarray           # [Ks] delay target
    lambda_pps: np.ndarray    # [Ks] Poisson arrival rate
    zbar_bits: float          # packet size
    G: np.ndarray             # [N, M, K] float32 channel power gains
    w: Optional[np.ndarray] = None   # [M*K] priority weights (None = 1)
    seed: int = 0

    @property
    def cost(self) -> int:
        return self.M * self.N * self.K


@dataclasses.dataclass
class Tolerances:
    tol_dinkelbach: float = 1e-6
    tol_scale: float = 1e-5
    tol_dual: float = 1e-5
    max_dinkelbach: int = 50
    max_scale: int = 50
    max_dual: int = 200


def _sites(M: int, layout: str):
    """RRH / base-station positions (m): "hcran" puts RRH 0 at the origin and
    the others on a 200 m ring; "ring" puts all M on the ring; "pair" puts two
    sites at (-250 m, 0) and (250 m, 0)."""
    bx = np.zeros(M)
    by = np.zeros(M)
    if layout == "hcran":
        for j in range(1, M):
            a = 2.0 * math.pi * (j - 1) / (M - 1)
            bx[j] = 200.0 * math.cos(a)
            by[j] = 200.0 * math.sin(a)
    elif layout == "ring":
        for j in range(M):
            a = 2.0 * math.pi * j / M
            bx[j] = 200.0 * math.cos(a)
            by[j] = 200.0 * math.sin(a)
    elif layout == "pair":
        if M != 2:
            raise ValueError("the pair layout has two sites")
        bx[:] = [-250.0, 250.0]
    else:
        raise ValueError("unknown layout " + layout)
    return bx, by


def _gains(seed: int, M: int, N: int, K: int, layout: str = "hcran") -> np.ndarray:
    u_r = splitmix64_uniform(seed, _S_RADIUS, K)
    u_t = splitmix64_uniform(seed, _S_ANGLE, K)
    r = 500.0 * np.sqrt(u_r)
    th = 2.0 * math.pi * u_t
    ux, uy = r * np.cos(th), r * np.sin(th)
    bx, by = _sites(M, layout)
    d = np.hypot(ux[None, :] - bx[:, None], uy[None, :] - by[:, None])   # [M, K] m
    d_km = np.maximum(d, 10.0) / 1000.0
    pl_db = 128.1 + 37.6 * np.log10(d_km)
    a = splitmix64_uniform(seed, _S_SHADOW_A, M * K).reshape(M, K)
    b = splitmix64_uniform(seed, _S_SHADOW_B, M * K).reshape(M, K)
    shadow_db = 8.0 * np.sqrt(-2.0 * np.log(a)) * np.cos(2.0 * math.pi * b)
    large = 10.0 ** (-(pl_db + shadow_db) / 10.0)                        # [M, K]
    chi = -np.log(splitmix64_uniform(seed, _S_FADING, N * M * K)).reshape(N, M, K)
    return (large[None, :, :] * chi).astype(np.float32)


def make_instance(seed: int, M: int, N: int, K: int, Ks: int, l: int,
                  pmax_hpn: float = 40.0, pmax_lpn: float = 1.0,
                  pc_hpn: float = 10.0, pc_lpn: float = 1.0,
                  eta_hpn: float = 4.0, eta_lpn: float = 2.0,
                  pf_hpn: float = 3.0, pf_lpn: float = 1.0,
                  Bn_hz: float = 180e3, N0_dbm_per_hz: float = -174.0,
                  T_s: float = 0.05, rate_bps: float = 64e3,
                  zbar_bits: float = 1024.0, layout: str = "hcran",
                  per_rrh: Optional[dict] = None) -> Instance:
    """per_rrh: optional [M] arrays "pmax", "eta", "Pc", "Pf" that replace the
    HPN / LPN constants (RRH 0 is the HPN, the others LPNs)."""
    if not (M >= 1 and N >= 1 and K >= 1 and 0 <= Ks <= K and l >= 1):
        raise ValueError("bad instance sizes")
    pmax = np.array([pmax_hpn] + [pmax_lpn] * (M - 1), dtype=np.float64)
    eta = np.array([eta_hpn] + [eta_lpn] * (M - 1), dtype=np.float64)
    Pc = np.array([pc_hpn] + [pc_lpn] * (M - 1), dtype=np.float64)
    Pf = np.array([pf_hpn] + [pf_lpn] * (M - 1), dtype=np.float64)
    if per_rrh:
        pmax = np.asarray(per_rrh.get("pmax", pmax), dtype=np.float64)
        eta = np.asarray(per_rrh.get("eta", eta), dtype=np.float64)
        Pc = np.asarray(per_rrh.get("Pc", Pc), dtype=np.float64)
        Pf = np.asarray(per_rrh.get("Pf", Pf), dtype=np.float64)
        if not all(a.shape == (M,) for a in (pmax, eta, Pc, Pf)):
            raise ValueError("per-RRH constants must have M entries")
    N0 = 10.0 ** (N0_dbm_per_hz / 10.0) * 1e-3
    lam = rate_bps / zbar_bits
    return Instance(M=M, N=N, K=K, Ks=Ks, l=l, pmax=pmax, eta=eta, Pc=Pc, Pf=Pf,
                    Bn_hz=Bn_hz, N0_w_per_hz=N0,
                    T_s=np.full(Ks, T_s), lambda_pps=np.full(Ks, lam),
                    zbar_bits=zbar_bits, G=_gains(seed, M, N, K, layout), seed=seed)


def _batch_sizes(seed: int):
    u = splitmix64_uniform(seed, _S_SIZES, 3)
    M = 3 + int(u[0] * 14)          # U{3..16}
    N = 16 + int(u[1] * 241)        # U{16..256}
    K = 10 + int(u[2] * 111)        # U{10..120}
    Ks = int(math.floor(0.3 * K + 0.5))
    return M, N, K, Ks


def _small(i: int) -> Instance:
    return make_instance(1000 + i, M=3, N=8, K=6, Ks=2, l=2)


def _medium(i: int) -> Instance:
    return make_instance(2000 + i, M=9, N=64, K=48, Ks=16, l=3)


def _batch(i: int) -> Instance:
    seed = 300000 + i
    M, N, K, Ks = _batch_sizes(seed)
    return make_instance(seed, M=M, N=N, K=K, Ks=Ks, l=3)


def _large(i: int) -> Instance:
    return make_instance(500000 + i, M=33, N=1024, K=512, Ks=128, l=4)


# The architectures compared in Sec. VI, each on 32 subcarriers with 12 users
# of whom 6 stream (125 packets/s of 1024 bits, delay target 0.2 s):
#   H-CRAN (NOMA and OMA)  one HPN and two LPN RRHs
#   1-tier C-RAN           three LPN RRHs
#   2-tier HCN             one macro BS and two pico BSs (static circuit power
#                          10 W and 6.8 W, amplifier factor 4 for each)
#   1-tier HPN             two macro BSs
# Base stations of the HCN and HPN scenarios have no fronthaul power; macro
# and pico BSs transmit at most the HPN's and the LPN's power.
_SCEN_TRAFFIC = dict(N=32, K=12, Ks=6, T_s=0.2, rate_bps=125 * 1024.0)


def _scen_hcran(i: int, l: int = 3) -> Instance:
    return make_instance(600000 + i, M=3, l=l, **_SCEN_TRAFFIC)


def _scen_hcran_oma(i: int) -> Instance:
    return _scen_hcran(i, l=1)


def _scen_cran(i: int) -> Instance:
    return make_instance(600000 + i, M=3, l=3, layout="ring",
                         per_rrh=dict(pmax=[1.0] * 3, eta=[2.0] * 3, Pc=[1.0] * 3, Pf=[1.0] * 3), **_SCEN_TRAFFIC)


def _scen_hcn(i: int) -> Instance:
    return make_instance(600000 + i, M=3, l=3,
                         per_rrh=dict(pmax=[40.0, 1.0, 1.0], eta=[4.0] * 3, Pc=[10.0, 6.8, 6.8], Pf=[0.0] * 3),
                         **_SCEN_TRAFFIC)


def _scen_hpn(i: int) -> Instance:
    return make_instance(600000 + i, M=2, l=3, layout="pair",
                         per_rrh=dict(pmax=[40.0] * 2, eta=[4.0] * 2, Pc=[10.0] * 2, Pf=[0.0] * 2), **_SCEN_TRAFFIC)


def _optimum(i: int) -> Instance:
    return make_instance(800000 + i, M=3, N=2, K=3, Ks=0, l=2)


WORKLOADS: Dict[str, dict] = {
    # 1 HPN + 2 LPNs, 8 subcarriers, 4 elastic + 2 streaming users, l = 2
    "small-3x8x6": dict(make=_small, count=1, tol=Tolerances()),
    # 1 HPN + 8 LPNs, 64 subcarriers, 32 elastic + 16 streaming users, l = 3
    "medium-9x64x48": dict(make=_medium, count=1,
                           tol=Tolerances(tol_dinkelbach=1e-6, tol_scale=1e-5, max_dual=200)),
    # 4096 uneven realisations: M in 3..16, N in 16..256, K in 10..120, 30 % streaming
    "batch-4096-uneven": dict(make=_batch, count=4096, tol=Tolerances()),
    # 1 HPN + 32 LPNs, 1024 subcarriers, 384 elastic + 128 streaming, l = 4
    "large-33x1024x512": dict(make=_large, count=256, tol=Tolerances()),
    # small H-CRAN instances whose optimum the brute-force comparator finds:
    # 1 HPN + 2 LPNs, 2 subcarriers, 3 elastic users, l = 2 (954 assignments)
    "optimum-3x2x3": dict(make=_optimum, count=256, tol=Tolerances()),
    # the architectures of Sec. VI (same seeds and users in each)
    "scenario-hcran-noma": dict(make=_scen_hcran, count=256, tol=Tolerances()),
    "scenario-hcran-oma": dict(make=_scen_hcran_oma, count=256, tol=Tolerances()),
    "scenario-cran-1tier": dict(make=_scen_cran, count=256, tol=Tolerances()),
    "scenario-hcn-2tier": dict(make=_scen_hcn, count=256, tol=Tolerances()),
    "scenario-hpn-1tier": dict(make=_scen_hpn, count=256, tol=Tolerances()),
}
SCENARIOS = ["scenario-hcran-noma", "scenario-hcran-oma", "scenario-cran-1tier", "scenario-hcn-2tier",
             "scenario-hpn-1tier"]


def make_workload(name: str, count: Optional[int] = None,
                  start: int = 0) -> List[Instance]:
    spec = WORKLOADS[name]
    n = spec["count"] if count is None else count
    return [spec["make"](start + i) for i in range(n)]


def pack_batch(insts: Sequence[Instance]):
    """Pack the gain tensors of several instances back to back (float32).

    Returns (gains, offsets) where instance b occupies
    gains[offsets[b] : offsets[b] + N*M*K] in [n][m][k] order.  Every offset is
    a multiple of 4 elements so that each slab starts 16-byte aligned.
    """
    offs = []
    tot = 0
    for inst in insts:
        offs.append(tot)
        tot += (inst.cost + 3) // 4 * 4
    buf = np.zeros(tot, dtype=np.float32)
    for inst, o in zip(insts, offs):
        buf[o:o + inst.cost] = inst.G.reshape(-1)
    return buf, np.asarray(offs, dtype=np.int64)
