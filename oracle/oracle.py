"""ctypes binding of the plain-C FP64 oracle (``hcran_oracle.c``).

TEST INFRASTRUCTURE: used by the tests, the smoke check and the CPU baseline
of the benchmark only.  See ``hcran_oracle.c`` for the method and readings.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hcran_oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "hcran_penalty.c")]
_OUT = os.path.join(_HERE, "_build", "liborc.so")
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_fp = C.POINTER(C.c_float)


class _Problem(C.Structure):
    _fields_ = [("M", C.c_int32), ("N", C.c_int32), ("K", C.c_int32), ("Ks", C.c_int32),
                ("l", C.c_int32), ("pmax", _dp), ("eta", _dp), ("Pc", _dp), ("Pf", _dp),
                ("Bn_hz", C.c_double), ("N0_w_per_hz", C.c_double), ("T_s", _dp),
                ("lambda_pps", _dp), ("zbar_bits", C.c_double), ("w", _dp), ("G", _fp)]


class _Params(C.Structure):
    _fields_ = [("tol_dinkelbach", C.c_double), ("tol_scale", C.c_double),
                ("tol_dual", C.c_double), ("max_dinkelbach", C.c_int32),
                ("max_scale", C.c_int32), ("max_dual", C.c_int32), ("q_init", C.c_double),
                ("tie_eps", C.c_double), ("noise_rel", C.c_double), ("noise_seed", C.c_uint64)]


class _Result(C.Structure):
    _fields_ = [("A", _ip), ("S", _ip), ("p", _dp), ("alpha", _dp), ("beta", _dp),
                ("xi", _dp), ("zeta", _dp), ("zeta_sic", _dp), ("q_trace", _dp),
                ("F_trace", _dp), ("scale_obj_trace", _dp), ("scale_sel_changed", _ip),
                ("ee", C.c_double), ("R", C.c_double), ("P", C.c_double),
                ("iters", C.c_int32 * 3), ("status", C.c_int32),
                ("slack_power_min", C.c_double), ("slack_rate_min", C.c_double),
                ("slack_sic_max", C.c_double), ("min_margin", C.c_double),
                ("n_ties", C.c_int32), ("n_scale_traced", C.c_int32)]


class _PenResult(C.Structure):
    _fields_ = [("p", _dp), ("alpha", _dp), ("xi", _dp), ("theta", _dp), ("theta2", _dp),
                ("ee", C.c_double), ("R", C.c_double), ("P", C.c_double),
                ("iters", C.c_int32 * 3), ("status", C.c_int32),
                ("slack_power_min", C.c_double), ("c10_max", C.c_double), ("c11_max", C.c_double),
                ("slack_sic_max", C.c_double), ("n_theta", C.c_int32), ("n_theta2", C.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (strict IEEE: no fast-math, no FMA contraction)."""
    newest = max(os.path.getmtime(f) for f in _SRCS + [os.path.join(_HERE, "hcran_oracle.h")])
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < newest:
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               "-o", tmp, *_SRCS, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        lib.orc_solve.argtypes = [C.POINTER(_Problem), C.POINTER(_Params), C.POINTER(_Result)]
        lib.orc_solve.restype = C.c_int
        lib.orc_psi.argtypes = [C.c_double] * 4
        lib.orc_psi.restype = C.c_double
        lib.orc_scale_coeffs.argtypes = [C.c_double, _dp, _dp]
        lib.orc_scale_coeffs.restype = None
        lib.orc_bruteforce.argtypes = [C.POINTER(_Problem), _dp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
        lib.orc_bruteforce.restype = C.c_int
        lib.orc_penalty_solve.argtypes = [C.POINTER(_Problem), C.POINTER(_Params), C.c_double,
                                          C.POINTER(_PenResult)]
        lib.orc_penalty_solve.restype = C.c_int
        _lib = lib
    return _lib


def psi(T_s: float, lambda_pps: float, zbar_bits: float, Bn_hz: float) -> float:
    """Minimum rate (bits/s/Hz) of C9 from the M/G/1 delay bound."""
    return _load().orc_psi(T_s, lambda_pps, zbar_bits, Bn_hz)


def scale_coeffs(z0: float):
    a, b = C.c_double(), C.c_double()
    _load().orc_scale_coeffs(z0, C.byref(a), C.byref(b))
    return a.value, b.value


def _problem(inst, keep):
    def d(x):
        a = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(a)
        return _ptr(a, _dp)
    G = np.ascontiguousarray(inst.G, dtype=np.float32)
    keep.append(G)
    Ks = inst.Ks
    return _Problem(inst.M, inst.N, inst.K, Ks, inst.l, d(inst.pmax), d(inst.eta), d(inst.Pc), d(inst.Pf),
                    float(inst.Bn_hz), float(inst.N0_w_per_hz),
                    d(inst.T_s if Ks else np.zeros(1)), d(inst.lambda_pps if Ks else np.ones(1)),
                    float(inst.zbar_bits), d(inst.w) if inst.w is not None else None, _ptr(G, _fp))


def bruteforce(inst):
    """(best EE, assignments searched, index of the best) of the global-optimum
    comparator (elastic users only; see hcran_oracle.h)."""
    lib = _load()
    keep = []
    pr = _problem(inst, keep)
    ee, na, bi = C.c_double(), C.c_int64(), C.c_int64()
    if lib.orc_bruteforce(C.byref(pr), C.byref(ee), C.byref(na), C.byref(bi)) != 0:
        raise ValueError("bruteforce rejected the problem")
    return ee.value, na.value, bi.value


@dataclasses.dataclass
class OracleResult:
    A: np.ndarray
    S: np.ndarray
    p: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    xi: np.ndarray
    zeta: np.ndarray
    zeta_sic: np.ndarray
    q_trace: np.ndarray
    F_trace: np.ndarray
    scale_obj_trace: np.ndarray
    scale_sel_changed: np.ndarray
    ee: float
    R: float
    P: float
    iters: tuple
    status: int
    slack_power_min: float
    slack_rate_min: float
    slack_sic_max: float
    min_margin: float
    n_ties: int


def _ptr(a, t):
    return a.ctypes.data_as(t)


def solve(inst, tol=None, q_init: float = 0.0, tie_eps: float = 1e-9,
          max_dinkelbach: Optional[int] = None, max_scale: Optional[int] = None,
          max_dual: Optional[int] = None, noise_rel: float = 0.0,
          noise_seed: int = 0) -> OracleResult:
    """Run the oracle on one ``hcran_inputs.Instance``.

    ``noise_rel > 0`` turns on the perturbation ensemble (test use only): every
    new power of a dual iteration is scaled by (1 + noise_rel * u), u uniform
    in [-1, 1) from a stream keyed by ``noise_seed``."""
    lib = _load()
    M, N, K, Ks, l = inst.M, inst.N, inst.K, inst.Ks, inst.l
    npair = l * (l - 1) // 2
    keep = []

    def d(x):
        a = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(a)
        return _ptr(a, _dp)

    G = np.ascontiguousarray(inst.G, dtype=np.float32)
    keep.append(G)
    pr = _Problem(M, N, K, Ks, l, d(inst.pmax), d(inst.eta), d(inst.Pc), d(inst.Pf),
                  float(inst.Bn_hz), float(inst.N0_w_per_hz),
                  d(inst.T_s if Ks else np.zeros(1)), d(inst.lambda_pps if Ks else np.ones(1)),
                  float(inst.zbar_bits), d(inst.w) if inst.w is not None else None,
                  _ptr(G, _fp))
    if tol is None:
        from hcran_inputs import Tolerances
        tol = Tolerances()
    Imax = max_dinkelbach if max_dinkelbach is not None else tol.max_dinkelbach
    Smax = max_scale if max_scale is not None else tol.max_scale
    Vmax = max_dual if max_dual is not None else tol.max_dual
    par = _Params(tol.tol_dinkelbach, tol.tol_scale, tol.tol_dual, Imax, Smax, Vmax,
                  q_init, tie_eps, float(noise_rel), int(noise_seed))
    L = N * M * l
    out = dict(A=np.zeros(K, np.int32), S=np.zeros(L, np.int32), p=np.zeros(L),
               alpha=np.zeros(L), beta=np.zeros(L), xi=np.zeros(M), zeta=np.zeros(max(Ks, 1)),
               zeta_sic=np.zeros(max(N * M * npair, 1)), q_trace=np.zeros(Imax + 1),
               F_trace=np.zeros(max(Imax, 1)), scale_obj_trace=np.zeros(max(Imax * Smax, 1)),
               scale_sel_changed=np.zeros(max(Imax * Smax, 1), np.int32))
    res = _Result()
    for name, arr in out.items():
        setattr(res, name, _ptr(arr, _ip if arr.dtype == np.int32 else _dp))
    rc = lib.orc_solve(C.byref(pr), C.byref(par), C.byref(res))
    if rc != 0:
        raise ValueError("oracle rejected the problem (code %d)" % rc)
    nd, nt = res.iters[0], res.n_scale_traced
    return OracleResult(
        A=out["A"], S=out["S"].reshape(N, M, l), p=out["p"].reshape(N, M, l),
        alpha=out["alpha"].reshape(N, M, l), beta=out["beta"].reshape(N, M, l),
        xi=out["xi"], zeta=out["zeta"][:Ks],
        zeta_sic=out["zeta_sic"][:N * M * npair].reshape(N, M, npair),
        q_trace=out["q_trace"][:nd + 1], F_trace=out["F_trace"][:nd],
        scale_obj_trace=out["scale_obj_trace"][:nt],
        scale_sel_changed=out["scale_sel_changed"][:nt],
        ee=res.ee, R=res.R, P=res.P, iters=tuple(res.iters), status=res.status,
        slack_power_min=res.slack_power_min, slack_rate_min=res.slack_rate_min,
        slack_sic_max=res.slack_sic_max, min_margin=res.min_margin, n_ties=res.n_ties)


@dataclasses.dataclass
class PenaltyResult:
    p: np.ndarray          # [N][M][K]
    alpha: np.ndarray      # [N][M][K]
    xi: np.ndarray
    theta: np.ndarray      # C10 multipliers (hcran_penalty.c gives the order)
    theta2: np.ndarray     # C11 multipliers
    ee: float
    R: float
    P: float
    iters: tuple
    status: int
    slack_power_min: float
    c10_max: float
    c11_max: float
    slack_sic_max: float


def penalty_solve(inst, tol=None, rho_rel: float = 1e-3, q_init: float = 0.0,
                  max_dinkelbach: Optional[int] = None, max_scale: Optional[int] = None,
                  max_dual: Optional[int] = None) -> PenaltyResult:
    """The paper-literal penalty form of C10/C11 (``hcran_penalty.c``) on one
    elastic-only ``hcran_inputs.Instance``."""
    from math import comb
    lib = _load()
    keep = []
    pr = _problem(inst, keep)
    if tol is None:
        from hcran_inputs import Tolerances
        tol = Tolerances()
    Imax = max_dinkelbach if max_dinkelbach is not None else tol.max_dinkelbach
    Smax = max_scale if max_scale is not None else tol.max_scale
    Vmax = max_dual if max_dual is not None else tol.max_dual
    par = _Params(tol.tol_dinkelbach, tol.tol_scale, tol.tol_dual, Imax, Smax, Vmax, q_init, 0.0, 0.0, 0)
    M, N, K, l = inst.M, inst.N, inst.K, inst.l
    L = N * M * K
    n10 = K * (M * (M - 1) // 2) * N * N
    n11 = N * M * comb(K, l + 1)
    out = dict(p=np.zeros(L), alpha=np.zeros(L), xi=np.zeros(M), theta=np.zeros(max(n10, 1)),
               theta2=np.zeros(max(n11, 1)))
    res = _PenResult()
    for name, arr in out.items():
        setattr(res, name, _ptr(arr, _dp))
    rc = lib.orc_penalty_solve(C.byref(pr), C.byref(par), float(rho_rel), C.byref(res))
    if rc != 0:
        raise ValueError("penalty oracle rejected the problem (code %d)" % rc)
    assert res.n_theta == n10 and res.n_theta2 == n11
    return PenaltyResult(p=out["p"].reshape(N, M, K), alpha=out["alpha"].reshape(N, M, K), xi=out["xi"],
                         theta=out["theta"][:n10], theta2=out["theta2"][:n11], ee=res.ee, R=res.R, P=res.P,
                         iters=tuple(res.iters), status=res.status, slack_power_min=res.slack_power_min,
                         c10_max=res.c10_max, c11_max=res.c11_max, slack_sic_max=res.slack_sic_max)
