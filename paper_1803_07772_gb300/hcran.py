"""Thin Python binding of the C ABI in ``include/hcran.h`` (ctypes).

Argument marshalling only: every step of the solve runs in the CUDA library
``_build/libhcran.so``.  PyTorch provides the device workspace and the
stream.  There is no CPU fallback: without the built library or a GPU the
calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_lib = None

_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)

STATUS_NAMES = {0: "HCRAN_OK", 1: "HCRAN_EINVAL", 2: "HCRAN_ENOMEM", 3: "HCRAN_ECUDA",
                4: "HCRAN_ETIMEDOUT", 5: "HCRAN_ENUMERIC", 6: "HCRAN_E2BIG"}
ST_NOT_CONVERGED, ST_STREAMING_UNMET, ST_EE_DECREASED, ST_NUMERIC = 1, 2, 4, 8


class HcranError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__("%s failed: %s" % (fn, STATUS_NAMES.get(code, str(code))))
        self.code = code


class Config(C.Structure):
    _fields_ = [("M", C.c_int32), ("N", C.c_int32), ("K", C.c_int32), ("Ks", C.c_int32),
                ("l", C.c_int32), ("pmax", _dp), ("eta", _dp), ("Pc", _dp), ("Pf", _dp),
                ("Bn_hz", C.c_double), ("N0_w_per_hz", C.c_double), ("T_s", _dp),
                ("lambda_pps", _dp), ("zbar_bits", C.c_double), ("w", _dp)]


class Tol(C.Structure):
    _fields_ = [("tol_dinkelbach", C.c_double), ("tol_scale", C.c_double),
                ("tol_dual", C.c_double), ("max_dinkelbach", C.c_int32),
                ("max_scale", C.c_int32), ("max_dual", C.c_int32), ("tie_eps", C.c_double),
                ("q_init", C.c_double)]


class Result(C.Structure):
    _fields_ = [("A", _ip), ("S", _ip), ("p", _fp), ("alpha", _fp), ("beta", _fp),
                ("xi", _dp), ("zeta", _dp), ("zeta_sic", _dp), ("ee", C.c_double),
                ("R", C.c_double), ("P", C.c_double), ("iters", C.c_int32 * 3),
                ("status", C.c_int32), ("slack_power_min", C.c_double),
                ("slack_rate_min", C.c_double), ("slack_sic_max", C.c_double),
                ("min_margin", C.c_double), ("n_ties", C.c_int32)]


EXPORTS = ["hcran_create", "hcran_workspace_size", "hcran_gain_elems", "hcran_prepare",
           "hcran_solve", "hcran_solve_host", "hcran_get", "hcran_get_summary",
           "hcran_get_phase_cycles", "hcran_last_launch_count", "hcran_destroy",
           "hcran_solve_noalloc", "hcran_get_schedule", "hcran_set_schedule", "hcran_autotune",
           "hcran_solve_graph", "hcran_warm_rows", "hcran_warm_features", "hcran_solve_warm",
           "hcran_set_state", "hcran_set_wait_limit", "hcran_bf_workspace_size", "hcran_bruteforce",
           "hcran_penalty_workspace_size", "hcran_penalty_solve", "hcran_get_stream_teams"]
# include/hcran_mlp.h: tensor-core kernels of the warm-start network
MLP_EXPORTS = ["hcran_mlp_dense", "hcran_mlp_tc_status", "hcran_mlp_create", "hcran_mlp_destroy",
               "hcran_mlp_param_count", "hcran_mlp_get_params", "hcran_mlp_set_params", "hcran_mlp_get_grads",
               "hcran_mlp_forward", "hcran_mlp_loss_grad", "hcran_mlp_backward", "hcran_mlp_adam"]


def load(build_if_missing: bool = True):
    """Load the solver library (building it first if asked); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and _build._stale():
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError("CUDA solver library not built: %s (run paper_1803_07772_gb300.build)" % path)
    lib = C.CDLL(path)
    vp = C.c_void_p
    sig = {
        "hcran_create": ([C.POINTER(vp), C.POINTER(Config), C.c_int32, _i64p], C.c_int),
        "hcran_workspace_size": ([vp, C.POINTER(C.c_uint64)], C.c_int),
        "hcran_gain_elems": ([vp, C.POINTER(C.c_int64)], C.c_int),
        "hcran_prepare": ([vp, vp, vp], C.c_int),
        "hcran_solve": ([vp, vp, C.POINTER(Tol), vp, vp], C.c_int),
        "hcran_solve_host": ([vp, vp, C.POINTER(Tol), vp, vp, _dp, _ip], C.c_int),
        "hcran_get": ([vp, C.c_int32, C.POINTER(Result)], C.c_int),
        "hcran_get_summary": ([vp, _dp, _dp, _dp, _ip, _ip, _dp, _ip], C.c_int),
        "hcran_get_phase_cycles": ([vp, _i64p], C.c_int),
        "hcran_last_launch_count": ([vp, _ip], C.c_int),
        "hcran_destroy": ([vp], None),
        "hcran_solve_noalloc": ([C.POINTER(Config), vp, C.POINTER(Tol), vp, C.POINTER(Result)], C.c_int),
        "hcran_get_schedule": ([vp, _ip], C.c_int),
        "hcran_set_schedule": ([vp, _ip], C.c_int),
        "hcran_autotune": ([vp, vp, C.POINTER(Tol), vp, vp, C.c_int32], C.c_int),
        "hcran_solve_graph": ([vp, vp, C.POINTER(Tol), vp, vp], C.c_int),
        "hcran_warm_rows": ([vp, _i64p], C.c_int),
        "hcran_warm_features": ([vp, vp, vp, vp, vp], C.c_int),
        "hcran_solve_warm": ([vp, vp, C.POINTER(Tol), vp, vp, vp], C.c_int),
        "hcran_set_state": ([vp, vp, C.c_int32, C.POINTER(Result), vp], C.c_int),
        "hcran_set_wait_limit": ([vp, C.c_int64, C.c_int32], C.c_int),
        "hcran_bf_workspace_size": ([C.POINTER(Config), C.c_int32, C.POINTER(C.c_uint64), _i64p], C.c_int),
        "hcran_bruteforce": ([C.POINTER(Config), C.c_int32, vp, vp, vp, _dp, _i64p], C.c_int),
        "hcran_penalty_workspace_size": ([C.POINTER(Config), C.c_int32, C.POINTER(C.c_uint64)], C.c_int),
        "hcran_get_stream_teams": ([vp, _ip], C.c_int),
        "hcran_penalty_solve": ([C.POINTER(Config), C.c_int32, vp, C.POINTER(Tol), C.c_double, vp, vp, _dp, _dp,
                                 _ip, _dp, _dp], C.c_int),
        "hcran_mlp_dense": ([vp, vp, vp, vp, C.c_int64, C.c_int32, C.c_int32, C.c_int32, vp, vp], C.c_int),
        "hcran_mlp_tc_status": ([_ip], C.c_int),
        "hcran_mlp_create": ([C.POINTER(vp), C.c_uint64, C.c_int64], C.c_int),
        "hcran_mlp_destroy": ([vp], None),
        "hcran_mlp_param_count": ([vp, _i64p], C.c_int),
        "hcran_mlp_get_params": ([vp, _fp], C.c_int),
        "hcran_mlp_set_params": ([vp, _fp], C.c_int),
        "hcran_mlp_get_grads": ([vp, _fp], C.c_int),
        "hcran_mlp_forward": ([vp, vp, C.c_int64, vp, vp], C.c_int),
        "hcran_mlp_loss_grad": ([vp, vp, vp, vp, C.c_int64, C.c_int32, vp, vp], C.c_int),
        "hcran_mlp_backward": ([vp, vp, C.c_int64, vp], C.c_int),
        "hcran_mlp_adam": ([vp, C.c_float, C.c_float, C.c_float, C.c_float, vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _check(fn: str, rc: int):
    if rc != 0:
        raise HcranError(fn, rc)


def make_tol(tol=None, tie_eps: float = 1e-4, q_init: float = 0.0, **over) -> Tol:
    """hcran_tol from a ``hcran_inputs.Tolerances`` (or defaults) plus overrides."""
    base = dict(tol_dinkelbach=1e-6, tol_scale=1e-5, tol_dual=1e-5, max_dinkelbach=50,
                max_scale=50, max_dual=200)
    if tol is not None:
        for k in base:
            base[k] = getattr(tol, k)
    base.update({k: v for k, v in over.items() if v is not None})
    return Tol(base["tol_dinkelbach"], base["tol_scale"], base["tol_dual"],
               int(base["max_dinkelbach"]), int(base["max_scale"]), int(base["max_dual"]),
               float(tie_eps), float(q_init))


class Solver:
    """A planned batch of instances bound to one device workspace."""

    def __init__(self, instances: Sequence, gain_offsets: Optional[np.ndarray] = None,
                 device: str = "cuda", stream=None):
        import torch
        self._torch = torch
        lib = load()
        self.lib = lib
        self.instances = list(instances)
        n = len(self.instances)
        cfgs = (Config * n)()
        self._keep = []

        def d(x):
            a = np.ascontiguousarray(x, dtype=np.float64)
            self._keep.append(a)
            return a.ctypes.data_as(_dp)

        for i, inst in enumerate(self.instances):
            cfgs[i] = Config(inst.M, inst.N, inst.K, inst.Ks, inst.l, d(inst.pmax), d(inst.eta),
                             d(inst.Pc), d(inst.Pf), float(inst.Bn_hz), float(inst.N0_w_per_hz),
                             d(inst.T_s) if inst.Ks else None,
                             d(inst.lambda_pps) if inst.Ks else None, float(inst.zbar_bits),
                             d(inst.w) if inst.w is not None else None)
        offs = None
        if gain_offsets is not None:
            self._offs = np.ascontiguousarray(gain_offsets, dtype=np.int64)
            offs = self._offs.ctypes.data_as(_i64p)
        h = C.c_void_p()
        _check("hcran_create", lib.hcran_create(C.byref(h), cfgs, n, offs))
        self.h = h
        nb = C.c_uint64()
        _check("hcran_workspace_size", lib.hcran_workspace_size(h, C.byref(nb)))
        ge = C.c_int64()
        _check("hcran_gain_elems", lib.hcran_gain_elems(h, C.byref(ge)))
        self.gain_elems = ge.value
        self.workspace_bytes = nb.value
        self.device = torch.device(device)
        self.workspace = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        _check("hcran_prepare", lib.hcran_prepare(h, C.c_void_p(self.workspace.data_ptr()),
                                                  C.c_void_p(self.stream.cuda_stream)))

    def solve(self, gains, tol: Tol):
        """Enqueue the solve of every instance on the bound stream (device gains)."""
        _check("hcran_solve", self.lib.hcran_solve(
            self.h, C.c_void_p(gains.data_ptr()), C.byref(tol),
            C.c_void_p(self.workspace.data_ptr()), C.c_void_p(self.stream.cuda_stream)))

    def solve_graph(self, gains, tol: Tol):
        """Same as solve, through a CUDA graph captured on first use for these
        arguments (the bound stream must be a created stream)."""
        _check("hcran_solve_graph", self.lib.hcran_solve_graph(
            self.h, C.c_void_p(gains.data_ptr()), C.byref(tol),
            C.c_void_p(self.workspace.data_ptr()), C.c_void_p(self.stream.cuda_stream)))

    def set_schedule(self, cluster_size):
        """Cluster size per instance (1 .. 8; 0: one CTA streaming from global memory;
        -T: streamed with T teams of warps, T in 1 .. 4)."""
        a = np.ascontiguousarray(cluster_size, dtype=np.int32)
        _check("hcran_set_schedule", self.lib.hcran_set_schedule(self.h, a.ctypes.data_as(_ip)))

    def autotune(self, gains, tol: Tol, max_dual_probe: int = 60) -> np.ndarray:
        """Time each cluster-size class C < 8 against clusters of min(2 C, 8); keep the faster. Returns the schedule."""
        _check("hcran_autotune", self.lib.hcran_autotune(
            self.h, C.c_void_p(gains.data_ptr()), C.byref(tol), C.c_void_p(self.workspace.data_ptr()),
            C.c_void_p(self.stream.cuda_stream), int(max_dual_probe)))
        return self.schedule()

    def stream_teams(self) -> int:
        """Teams of warps the streamed class's sweeps run (0: none)."""
        v = C.c_int32()
        _check("hcran_get_stream_teams", self.lib.hcran_get_stream_teams(self.h, C.byref(v)))
        return v.value

    def warm_rows(self) -> int:
        n = C.c_int64()
        _check("hcran_warm_rows", self.lib.hcran_warm_rows(self.h, C.byref(n)))
        return n.value

    def warm_features(self, gains, features=None):
        """Features of every slot of the initial selection ([rows][16] bfloat16 CUDA tensor)."""
        if features is None:
            features = self._torch.zeros((self.warm_rows(), 16), dtype=self._torch.bfloat16, device=self.device)
        _check("hcran_warm_features", self.lib.hcran_warm_features(
            self.h, C.c_void_p(gains.data_ptr()), C.c_void_p(self.workspace.data_ptr()),
            C.c_void_p(self.stream.cuda_stream), C.c_void_p(features.data_ptr())))
        return features

    def solve_warm(self, gains, tol: Tol, net_out):
        """Solve from the network's outputs ([rows][16] float32 CUDA tensor)."""
        _check("hcran_solve_warm", self.lib.hcran_solve_warm(
            self.h, C.c_void_p(gains.data_ptr()), C.byref(tol), C.c_void_p(self.workspace.data_ptr()),
            C.c_void_p(self.stream.cuda_stream), C.c_void_p(net_out.data_ptr())))

    def set_state(self, i: int, state: dict):
        """Start instance i of the next solve from `state` (a dict as get()
        returns; A, S, p required, the multipliers optional)."""
        inst = self.instances[i]
        N, M, K, Ks, l = inst.N, inst.M, inst.K, inst.Ks, inst.l
        keep = []

        def arr(name, dtype, size):
            if state.get(name) is None:
                return None
            a = np.ascontiguousarray(np.asarray(state[name], dtype=dtype).reshape(-1)[:size])
            keep.append(a)
            return a.ctypes.data_as(_ip if dtype == np.int32 else (_fp if dtype == np.float32 else _dp))
        L, npair = N * M * l, l * (l - 1) // 2
        r = Result()
        r.A, r.S, r.p = arr("A", np.int32, K), arr("S", np.int32, L), arr("p", np.float32, L)
        r.alpha, r.beta = arr("alpha", np.float32, L), arr("beta", np.float32, L)
        r.xi, r.zeta = arr("xi", np.float64, M), arr("zeta", np.float64, Ks) if Ks else None
        r.zeta_sic = arr("zeta_sic", np.float64, N * M * npair) if npair else None
        _check("hcran_set_state", self.lib.hcran_set_state(
            self.h, C.c_void_p(self.workspace.data_ptr()), int(i), C.byref(r), C.c_void_p(self.stream.cuda_stream)))

    def solve_host(self, gains_host, tol: Tol):
        """End-to-end solve from host gains; returns (ee, status) host arrays."""
        n = len(self.instances)
        ee = np.zeros(n)
        st = np.zeros(n, np.int32)
        ptr = gains_host.data_ptr() if hasattr(gains_host, "data_ptr") else gains_host.ctypes.data
        rc = self.lib.hcran_solve_host(
            self.h, C.c_void_p(ptr), C.byref(tol), C.c_void_p(self.workspace.data_ptr()),
            C.c_void_p(self.stream.cuda_stream), ee.ctypes.data_as(_dp), st.ctypes.data_as(_ip))
        if rc not in (0, 4, 5):  # ETIMEDOUT / ENUMERIC: per-instance status bits in st
            _check("hcran_solve_host", rc)
        return ee, st

    def launches(self) -> int:
        v = C.c_int32()
        _check("hcran_last_launch_count", self.lib.hcran_last_launch_count(self.h, C.byref(v)))
        return v.value

    def schedule(self) -> np.ndarray:
        """Cluster size per instance (0: one CTA streaming from global memory)."""
        out = np.zeros(len(self.instances), np.int32)
        _check("hcran_get_schedule", self.lib.hcran_get_schedule(self.h, out.ctypes.data_as(_ip)))
        return out

    def get(self, i: int) -> dict:
        inst = self.instances[i]
        N, M, K, Ks, l = inst.N, inst.M, inst.K, inst.Ks, inst.l
        L, npair = N * M * l, l * (l - 1) // 2
        arr = dict(A=np.zeros(K, np.int32), S=np.zeros(L, np.int32), p=np.zeros(L, np.float32),
                   alpha=np.zeros(L, np.float32), beta=np.zeros(L, np.float32),
                   xi=np.zeros(M), zeta=np.zeros(max(Ks, 1)),
                   zeta_sic=np.zeros(max(N * M * npair, 1)))
        r = Result()
        for k, a in arr.items():
            t = _ip if a.dtype == np.int32 else (_fp if a.dtype == np.float32 else _dp)
            setattr(r, k, a.ctypes.data_as(t))
        rc = self.lib.hcran_get(self.h, i, C.byref(r))
        if rc not in (0, 4, 5):  # ETIMEDOUT / ENUMERIC: the status bits say which; outputs are filled
            _check("hcran_get", rc)
        return dict(A=arr["A"], S=arr["S"].reshape(N, M, l), p=arr["p"].reshape(N, M, l),
                    alpha=arr["alpha"].reshape(N, M, l), beta=arr["beta"].reshape(N, M, l),
                    xi=arr["xi"], zeta=arr["zeta"][:Ks],
                    zeta_sic=arr["zeta_sic"][:N * M * npair].reshape(N, M, npair),
                    ee=r.ee, R=r.R, P=r.P, iters=tuple(r.iters), status=r.status,
                    slack_power_min=r.slack_power_min, slack_rate_min=r.slack_rate_min,
                    slack_sic_max=r.slack_sic_max, min_margin=r.min_margin, n_ties=r.n_ties, rc=rc)

    def set_wait_limit(self, max_tries: int = 0, stall_instance: int = -1):
        """Bound of the device waits; stall_instance >= 0 tests the timeout path on that instance."""
        _check("hcran_set_wait_limit", self.lib.hcran_set_wait_limit(self.h, int(max_tries), int(stall_instance)))

    def phase_cycles(self) -> np.ndarray:
        """[n, 8] SM cycles per phase of the last solve (see include/hcran.h)."""
        out = np.zeros((len(self.instances), 8), np.int64)
        _check("hcran_get_phase_cycles", self.lib.hcran_get_phase_cycles(
            self.h, out.ctypes.data_as(_i64p)))
        return out

    def summary(self) -> dict:
        n = len(self.instances)
        out = dict(ee=np.zeros(n), R=np.zeros(n), P=np.zeros(n), status=np.zeros(n, np.int32),
                   iters=np.zeros((n, 3), np.int32), min_margin=np.zeros(n),
                   n_ties=np.zeros(n, np.int32))
        _check("hcran_get_summary", self.lib.hcran_get_summary(
            self.h, out["ee"].ctypes.data_as(_dp), out["R"].ctypes.data_as(_dp),
            out["P"].ctypes.data_as(_dp), out["status"].ctypes.data_as(_ip),
            out["iters"].ctypes.data_as(_ip), out["min_margin"].ctypes.data_as(_dp),
            out["n_ties"].ctypes.data_as(_ip)))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.lib.hcran_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def bruteforce(instances, gains, stream=None):
    """Global-optimum comparator on the GPU (include/hcran.h): instances of one
    shape, elastic users only; gains a CUDA float32 tensor packed as
    hcran_inputs.pack_batch packs them.  Returns (best_ee, best_index,
    assignments per instance) as host arrays."""
    import torch
    lib = load()
    n = len(instances)
    cfgs = (Config * n)()
    keep = []

    def d(x):
        a = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(_dp)
    for i, inst in enumerate(instances):
        cfgs[i] = Config(inst.M, inst.N, inst.K, inst.Ks, inst.l, d(inst.pmax), d(inst.eta), d(inst.Pc),
                         d(inst.Pf), float(inst.Bn_hz), float(inst.N0_w_per_hz), None, None,
                         float(inst.zbar_bits), d(inst.w) if inst.w is not None else None)
    nb, na = C.c_uint64(), C.c_int64()
    _check("hcran_bf_workspace_size", lib.hcran_bf_workspace_size(cfgs, n, C.byref(nb), C.byref(na)))
    ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=gains.device)
    st = stream if stream is not None else torch.cuda.current_stream(gains.device)
    ee = np.zeros(n)
    idx = np.zeros(n, np.int64)
    _check("hcran_bruteforce", lib.hcran_bruteforce(cfgs, n, C.c_void_p(gains.data_ptr()),
                                                    C.c_void_p(ws.data_ptr()), C.c_void_p(st.cuda_stream),
                                                    ee.ctypes.data_as(_dp), idx.ctypes.data_as(_i64p)))
    return ee, idx, na.value


def penalty_solve(instances, gains, tol: Tol, rho_rel: float = 1e-3, stream=None) -> dict:
    """Penalty form of C10 / C11 on the GPU (include/hcran.h): instances of
    one shape, elastic users only; gains a CUDA float32 tensor packed as
    hcran_inputs.pack_batch packs them.  Returns host arrays ee [n],
    p [n][N][M][K], iters [n][3], c10_max [n], c11_max [n]."""
    import torch
    lib = load()
    n = len(instances)
    cfgs = (Config * n)()
    keep = []

    def d(x):
        a = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(_dp)
    for i, inst in enumerate(instances):
        cfgs[i] = Config(inst.M, inst.N, inst.K, inst.Ks, inst.l, d(inst.pmax), d(inst.eta), d(inst.Pc),
                         d(inst.Pf), float(inst.Bn_hz), float(inst.N0_w_per_hz), None, None,
                         float(inst.zbar_bits), d(inst.w) if inst.w is not None else None)
    nb = C.c_uint64()
    _check("hcran_penalty_workspace_size", lib.hcran_penalty_workspace_size(cfgs, n, C.byref(nb)))
    ws = torch.empty(max(nb.value, 256), dtype=torch.uint8, device=gains.device)
    st = stream if stream is not None else torch.cuda.current_stream(gains.device)
    i0 = instances[0]
    out = dict(ee=np.zeros(n), p=np.zeros((n, i0.N, i0.M, i0.K)), iters=np.zeros((n, 3), np.int32),
               c10_max=np.zeros(n), c11_max=np.zeros(n))
    _check("hcran_penalty_solve", lib.hcran_penalty_solve(
        cfgs, n, C.c_void_p(gains.data_ptr()), C.byref(tol), float(rho_rel), C.c_void_p(ws.data_ptr()),
        C.c_void_p(st.cuda_stream), out["ee"].ctypes.data_as(_dp), out["p"].ctypes.data_as(_dp),
        out["iters"].ctypes.data_as(_ip), out["c10_max"].ctypes.data_as(_dp), out["c11_max"].ctypes.data_as(_dp)))
    return out


def solve_noalloc(inst, gains, tol: Tol, stream=None) -> dict:
    """One instance through hcran_solve_noalloc (marshalling only).

    For callers that cannot allocate device memory: the library solves in its
    own fixed device array; `gains` is the caller's device tensor of
    Gamma[n][m][k] (float32) and the results come back in host arrays.
    """
    lib = load()
    keep = []

    def d(x):
        a = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(_dp)

    cfg = Config(inst.M, inst.N, inst.K, inst.Ks, inst.l, d(inst.pmax), d(inst.eta), d(inst.Pc),
                 d(inst.Pf), float(inst.Bn_hz), float(inst.N0_w_per_hz),
                 d(inst.T_s) if inst.Ks else None, d(inst.lambda_pps) if inst.Ks else None,
                 float(inst.zbar_bits), d(inst.w) if inst.w is not None else None)
    N, M, K, Ks, l = inst.N, inst.M, inst.K, inst.Ks, inst.l
    L, npair = N * M * l, l * (l - 1) // 2
    arr = dict(A=np.zeros(K, np.int32), S=np.zeros(L, np.int32), p=np.zeros(L, np.float32),
               alpha=np.zeros(L, np.float32), beta=np.zeros(L, np.float32), xi=np.zeros(M),
               zeta=np.zeros(max(Ks, 1)), zeta_sic=np.zeros(max(N * M * npair, 1)))
    r = Result()
    for k, a in arr.items():
        t = _ip if a.dtype == np.int32 else (_fp if a.dtype == np.float32 else _dp)
        setattr(r, k, a.ctypes.data_as(t))
    sptr = None
    if stream is not None:
        sptr = C.c_void_p(stream.cuda_stream)
    ptr = gains.data_ptr() if hasattr(gains, "data_ptr") else int(gains)
    _check("hcran_solve_noalloc", lib.hcran_solve_noalloc(C.byref(cfg), C.c_void_p(ptr), C.byref(tol),
                                                          sptr, C.byref(r)))
    return dict(A=arr["A"], S=arr["S"].reshape(N, M, l), p=arr["p"].reshape(N, M, l),
                alpha=arr["alpha"].reshape(N, M, l), beta=arr["beta"].reshape(N, M, l),
                xi=arr["xi"], zeta=arr["zeta"][:Ks],
                zeta_sic=arr["zeta_sic"][:N * M * npair].reshape(N, M, npair),
                ee=r.ee, R=r.R, P=r.P, iters=tuple(r.iters), status=r.status,
                min_margin=r.min_margin, n_ties=r.n_ties)
