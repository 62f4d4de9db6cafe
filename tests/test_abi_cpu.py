"""The C-ABI library loads, exports every symbol include/hcran.h declares,
and rejects bad arguments on the host (no GPU needed for these calls)."""
import ctypes as C
import math
import os
import re

import numpy as np
import pytest

from hcran_inputs import make_workload
from paper_1803_07772_gb300 import hcran

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions(header="hcran.h"):
    src = open(os.path.join(ROOT, "include", header)).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void)\s+(hcran_\w+)\s*\(", src, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = hcran.load()
    names = declared_functions()
    assert len(names) >= 10
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(hcran.EXPORTS) == names
    mlp = declared_functions("hcran_mlp.h")
    for n in mlp:
        assert hasattr(lib, n), n
    assert sorted(hcran.MLP_EXPORTS) == mlp


def _cfg(inst, **over):
    keep = []

    def d(x):
        a = np.ascontiguousarray(x, dtype=np.float64)
        keep.append(a)
        return a.ctypes.data_as(hcran._dp)

    c = hcran.Config(inst.M, inst.N, inst.K, inst.Ks, inst.l, d(inst.pmax), d(inst.eta), d(inst.Pc),
                     d(inst.Pf), inst.Bn_hz, inst.N0_w_per_hz, d(inst.T_s), d(inst.lambda_pps),
                     inst.zbar_bits, None)
    for k, v in over.items():
        if k in ("pmax", "eta", "Pc", "Pf", "T_s", "lambda_pps"):
            v = d(v)
        setattr(c, k, v)
    return c, keep


def _create(cfgs, offs=None):
    lib = hcran.load()
    arr = (hcran.Config * len(cfgs))(*cfgs)
    h = C.c_void_p()
    o = None
    if offs is not None:
        offs = np.asarray(offs, dtype=np.int64)
        o = offs.ctypes.data_as(hcran._i64p)
    rc = lib.hcran_create(C.byref(h), arr, len(cfgs), o)
    if rc == 0:
        lib.hcran_destroy(h)
    return rc


def test_create_accepts_valid_batch_and_sizes_workspace():
    insts = make_workload("batch-4096-uneven", count=3)
    cfgs = [_cfg(i) for i in insts]
    lib = hcran.load()
    arr = (hcran.Config * 3)(*[c for c, _ in cfgs])
    h = C.c_void_p()
    assert lib.hcran_create(C.byref(h), arr, 3, None) == 0
    nb, ge = C.c_uint64(), C.c_int64()
    assert lib.hcran_workspace_size(h, C.byref(nb)) == 0
    assert lib.hcran_gain_elems(h, C.byref(ge)) == 0
    assert ge.value == sum((i.cost + 3) // 4 * 4 for i in insts)
    assert nb.value % 256 == 0 and nb.value > 4 * ge.value
    lib.hcran_destroy(h)


@pytest.mark.parametrize("over", [dict(M=0), dict(N=0), dict(K=0), dict(Ks=-1), dict(l=0), dict(l=9),
                                  dict(M=65), dict(M=40, l=8), dict(Bn_hz=0.0), dict(N0_w_per_hz=-1.0),
                                  dict(Bn_hz=math.nan), dict(zbar_bits=0.0)])
def test_create_rejects_bad_scalars(over):
    inst = make_workload("small-3x8x6")[0]
    c, keep = _cfg(inst, **over)
    assert _create([c]) == 1


@pytest.mark.parametrize("field,val", [("pmax", [40.0, -1.0, 1.0]), ("eta", [4.0, 0.0, 2.0]),
                                       ("Pc", [math.nan, 1.0, 1.0]), ("T_s", [0.05, -0.05]),
                                       ("lambda_pps", [math.inf, 62.5])])
def test_create_rejects_bad_arrays(field, val):
    inst = make_workload("small-3x8x6")[0]
    c, keep = _cfg(inst, **{field: val})
    assert _create([c]) == 1


def test_create_rejects_ks_above_k_and_misaligned_offsets():
    inst = make_workload("small-3x8x6")[0]
    c, keep = _cfg(inst, Ks=7)
    assert _create([c]) == 1
    c, keep = _cfg(inst)
    assert _create([c], offs=[2]) == 1
    assert _create([c], offs=[-4]) == 1
    assert _create([c], offs=[8]) == 0


def test_null_arguments_rejected():
    lib = hcran.load()
    assert lib.hcran_create(None, None, 1, None) == 1
    assert lib.hcran_workspace_size(None, None) == 1
    assert lib.hcran_solve(None, None, None, None, None) == 1
    assert lib.hcran_get(None, 0, None) == 1


def _res_bytes(M, l, Ks, Nc):
    """Resident dual-loop footprint of Nc subcarriers, restated from the
    layout the schedule documents (slab rows padded to an odd number of
    float4, ten slot arrays, four per-RRH arrays, four SIC arrays, the
    nonzero masks and two streaming arrays)."""
    al4 = lambda x: (x + 3) & ~3
    Up = al4(M * l)
    Rs = Up if (Up // 4) % 2 == 1 else Up + 4
    Mi = M * (l * (l - 1) // 2)
    return 4 * (Nc * M * Rs + 10 * Nc * Up + 4 * al4(Nc * M) + 4 * al4(Nc * Mi)
                + al4(Nc * ((Mi + 31) // 32)) + 2 * al4(Nc * Ks))


def _iter_cycles(g):
    """Per-iteration cost of a CTA holding g (n, m) groups, restated from the
    planner's model: flat up to one group per thread (512), then about 3400
    cycles per further group per thread."""
    per = -(-g // 512)
    return 7000 + 6 * min(g, 512) + 3400 * max(per - 1, 0)


def test_schedule_picks_cheapest_cluster_that_holds_the_state():
    lib = hcran.load()
    insts = make_workload("batch-4096-uneven", count=64) + make_workload("large-33x1024x512", count=1)
    made = [_cfg(i) for i in insts]
    arr = (hcran.Config * len(made))(*[m[0] for m in made])
    h = C.c_void_p()
    assert lib.hcran_create(C.byref(h), arr, len(made), None) == 0
    cs = np.zeros(len(insts), np.int32)
    assert lib.hcran_get_schedule(h, cs.ctypes.data_as(hcran._ip)) == 0
    assert lib.hcran_get_schedule(h, None) == 1
    lib.hcran_destroy(h)
    assert set(cs.tolist()) <= set(range(9))
    assert cs[-1] == 0  # 33 x 1024 x 512: streamed from global memory
    assert len(set(cs[:-1].tolist()) - {1, 2, 4, 8}) > 0  # sizes between the powers of two are used
    budget = 216 * 1024
    cost = lambda inst, c: c * _iter_cycles(-(-inst.N // c) * inst.M)
    for inst, c in zip(insts[:-1], cs[:-1]):
        assert 0 < c <= min(8, inst.N)
        need = _res_bytes(inst.M, inst.l, inst.Ks, -(-inst.N // c))
        assert need < budget, (inst.M, inst.N, c, need)
        for c2 in range(1, min(8, inst.N) + 1):  # no cluster size that clearly fits is cheaper
            if _res_bytes(inst.M, inst.l, inst.Ks, -(-inst.N // c2)) <= budget - 8 * 1024:
                assert cost(inst, c) <= cost(inst, c2), (inst.M, inst.N, c, c2)


def test_set_schedule_validates_and_applies():
    lib = hcran.load()
    insts = make_workload("batch-4096-uneven", count=6) + make_workload("large-33x1024x512", count=1)
    made = [_cfg(i) for i in insts]
    arr = (hcran.Config * len(made))(*[m[0] for m in made])
    h = C.c_void_p()
    assert lib.hcran_create(C.byref(h), arr, len(made), None) == 0
    n = len(insts)
    get = lambda: (lambda a: (lib.hcran_get_schedule(h, a.ctypes.data_as(hcran._ip)), a)[1])(np.zeros(n, np.int32))
    base = get()
    bad = [np.where(np.arange(n) == 0, 9, base),                                   # not a cluster size
           np.where(np.arange(n) == n - 1, 1, base),                               # 33x1024 state fits no CTA
           np.array([8 if i.N >= 8 else 1 for i in insts[:-1]] + [0]) * 0 + 16]    # too large a cluster
    for b in bad:
        b = np.ascontiguousarray(b, dtype=np.int32)
        assert lib.hcran_set_schedule(h, b.ctypes.data_as(hcran._ip)) == 1
        assert np.array_equal(get(), base)
    assert lib.hcran_set_schedule(h, None) == 1
    want = np.array([8 if i.N >= 8 else c for i, c in zip(insts[:-1], base[:-1])] + [0], dtype=np.int32)
    assert lib.hcran_set_schedule(h, want.ctypes.data_as(hcran._ip)) == 0
    assert np.array_equal(get(), want)
    everything_streamed = np.zeros(n, np.int32)
    assert lib.hcran_set_schedule(h, everything_streamed.ctypes.data_as(hcran._ip)) == 0
    assert np.array_equal(get(), everything_streamed)
    lib.hcran_destroy(h)


def test_streamed_team_count_is_planned_and_set_on_the_host():
    """The 33 x 1024 x 512 shape stages its subcarriers in teams: the planner
    takes the most teams whose double buffers fit shared memory (3 of 5
    warps); hcran_set_schedule's -T forces T teams, all negative entries must
    agree, and T outside 1 .. 4 is rejected with the plan unchanged."""
    lib = hcran.load()
    insts = make_workload("batch-4096-uneven", count=2) + make_workload("large-33x1024x512", count=1)
    made = [_cfg(i) for i in insts]
    arr = (hcran.Config * len(made))(*[m[0] for m in made])
    h = C.c_void_p()
    assert lib.hcran_create(C.byref(h), arr, len(made), None) == 0
    teams = C.c_int32()

    def get_teams():
        assert lib.hcran_get_stream_teams(h, C.byref(teams)) == 0
        return teams.value
    assert get_teams() == 3
    sched = np.zeros(3, np.int32)
    assert lib.hcran_get_schedule(h, sched.ctypes.data_as(hcran._ip)) == 0
    for want in (1, 2, 3):
        s = np.ascontiguousarray(np.where(np.arange(3) == 2, -want, sched), dtype=np.int32)
        assert lib.hcran_set_schedule(h, s.ctypes.data_as(hcran._ip)) == 0
        assert get_teams() == want
    for bad in ([sched[0], sched[1], -5], [-1, sched[1], -2], [sched[0], sched[1], -4]):
        b = np.ascontiguousarray(bad, dtype=np.int32)  # -4: four teams' buffers exceed shared memory
        assert lib.hcran_set_schedule(h, b.ctypes.data_as(hcran._ip)) == 1
        assert get_teams() == 3
    assert lib.hcran_get_stream_teams(h, None) == 1
    lib.hcran_destroy(h)


def test_penalty_form_validates_shapes_on_the_host():
    """hcran_penalty_workspace_size / hcran_penalty_solve take one shape of at
    most 4 RRHs, 4 subcarriers, 8 users, l <= 3 and 128 links, elastic users
    only, and reject the rest before any device work."""
    from hcran_inputs import make_instance
    lib = hcran.load()
    nb = C.c_uint64()

    def size(insts):
        made = [_cfg(i) for i in insts]
        arr = (hcran.Config * len(made))(*[m[0] for m in made])
        return lib.hcran_penalty_workspace_size(arr, len(made), C.byref(nb))
    ok = [make_instance(1 + i, M=3, N=2, K=3, Ks=0, l=2) for i in range(2)]
    assert size(ok) == 0 and nb.value > 0
    assert size([make_instance(5, M=4, N=4, K=8, Ks=0, l=3)]) == 0   # 128 links
    for bad in ([make_instance(5, M=5, N=2, K=3, Ks=0, l=2)],       # too many RRHs
                [make_instance(5, M=3, N=2, K=9, Ks=0, l=2)],       # too many users
                [make_instance(5, M=3, N=2, K=4, Ks=1, l=2)],       # a streaming user
                [make_instance(5, M=3, N=2, K=3, Ks=0, l=4)],       # l above 3
                [ok[0], make_instance(7, M=3, N=3, K=3, Ks=0, l=2)]):  # mixed shapes
        assert size(bad) == 1
    made = [_cfg(i) for i in ok]
    arr = (hcran.Config * 2)(*[m[0] for m in made])
    tol = hcran.make_tol()
    ee = np.zeros(2)
    fake = C.c_void_p(1 << 20)  # aligned, never dereferenced: the call fails before device work
    args = lambda rho, g=fake, w=fake: lib.hcran_penalty_solve(arr, 2, g, C.byref(tol), rho, w, None,
                                                                ee.ctypes.data_as(hcran._dp), None, None,
                                                                None, None)
    assert args(0.0) == 1 and args(1.0) == 1                # rho_rel outside (0, 1)
    assert args(1e-3, g=C.c_void_p((1 << 20) + 4)) == 1     # gains not 16-byte aligned
    assert args(1e-3, w=C.c_void_p((1 << 20) + 16)) == 1    # workspace not 256-byte aligned


def test_kernel_hash_ignores_comments_but_not_code():
    """The hash that ties the stored DRAM-traffic ratio to the device code:
    comment and whitespace edits keep it, a code edit changes it."""
    import bench
    files = {f: open(os.path.join(os.path.dirname(hcran.__file__), "csrc", f), "rb").read()
             for f in bench.KERNEL_FILES}
    base = bench.kernel_hash(read=lambda f: files[f])
    assert base == bench.kernel_hash()
    commented = dict(files)
    commented["hcran_layout.h"] = b"// a new comment\n/* and a block\n comment */\n" + files["hcran_layout.h"] + b"\n\n"
    assert bench.kernel_hash(read=lambda f: commented[f]) == base
    changed = dict(files)
    changed["hcran_layout.h"] = files["hcran_layout.h"].replace(b"kClassMargin = 4096", b"kClassMargin = 4097")
    assert changed["hcran_layout.h"] != files["hcran_layout.h"]
    assert bench.kernel_hash(read=lambda f: changed[f]) != base
    assert bench._code_only(b'x = "a//b"; // c\ny = \'/\'; /* d */ z;') == b'x = "a//b"; y = \'/\'; z;'


def test_set_schedule_accepts_every_cluster_size_that_fits():
    """Every cluster size 1..8 is a valid schedule for an instance whose state
    fits and that has a subcarrier for each CTA; the schedule reads back as set."""
    lib = hcran.load()
    insts = make_workload("scenario-hcran-noma", count=2) + make_workload("small-3x8x6", count=1)
    made = [_cfg(i) for i in insts]
    arr = (hcran.Config * len(made))(*[m[0] for m in made])
    h = C.c_void_p()
    assert lib.hcran_create(C.byref(h), arr, len(made), None) == 0
    n = len(insts)
    for c in range(1, 9):
        want = np.array([c, c, min(c, 8)], np.int32)  # 32, 32 and 8 subcarriers: every size fits
        assert lib.hcran_set_schedule(h, want.ctypes.data_as(hcran._ip)) == 0, c
        got = np.zeros(n, np.int32)
        assert lib.hcran_get_schedule(h, got.ctypes.data_as(hcran._ip)) == 0
        assert np.array_equal(got, want), (c, got)
    too_many = np.array([1, 1, 9], np.int32)  # more CTAs than the portable cluster limit
    assert lib.hcran_set_schedule(h, too_many.ctypes.data_as(hcran._ip)) == 1
    lib.hcran_destroy(h)


def test_set_state_rejects_invalid_states_on_the_host():
    """hcran_set_state checks the state before any copy: NULL handle, workspace
    or arrays, an index out of range, a user on an RRH other than A_k (C5), a
    hole before a user (packing), a repeated user, a power above the mask or
    negative, a negative multiplier, zeta' out of range.  Each returns
    HCRAN_EINVAL without touching a device (none is needed here)."""
    lib = hcran.load()
    inst = make_workload("small-3x8x6")[0]
    c, keep = _cfg(inst)
    arr = (hcran.Config * 1)(c)
    h = C.c_void_p()
    assert lib.hcran_create(C.byref(h), arr, 1, None) == 0
    N, M, K, Ks, l = inst.N, inst.M, inst.K, inst.Ks, inst.l
    mask = inst.pmax / N

    def state(**over):
        A = np.array([0, 0, 1, 2, 0, 1], np.int32)
        S = -np.ones((N, M, l), np.int32)
        p = np.zeros((N, M, l), np.float32)
        for n in range(N):
            S[n, 0, :2] = [0, 1]
            S[n, 1, 0] = 2
            p[n, 0, :2] = mask[0] / 4
            p[n, 1, 0] = mask[1] / 2
        d = dict(A=A, S=S, p=p, xi=np.zeros(M), zeta=np.ones(Ks), zeta_sic=np.zeros(N * M))
        d.update(over)
        return d

    def call(st, ws=256, index=0):
        ks = []

        def a(x, t, tp):
            if x is None:
                return None
            y = np.ascontiguousarray(x, dtype=t).reshape(-1)
            ks.append(y)
            return y.ctypes.data_as(tp)
        r = hcran.Result()
        r.A, r.S, r.p = a(st["A"], np.int32, hcran._ip), a(st["S"], np.int32, hcran._ip), a(st["p"], np.float32, hcran._fp)
        r.xi, r.zeta = a(st.get("xi"), np.float64, hcran._dp), a(st.get("zeta"), np.float64, hcran._dp)
        r.zeta_sic = a(st.get("zeta_sic"), np.float64, hcran._dp)
        return lib.hcran_set_state(h, C.c_void_p(ws), index, C.byref(r), None)

    assert lib.hcran_set_state(None, C.c_void_p(256), 0, None, None) == 1
    assert call(state(), ws=0) == 1              # no workspace
    assert call(state(), ws=300) == 1            # misaligned workspace
    assert call(state(), index=1) == 1           # index out of range
    assert call(state(A=None)) == 1              # A required
    bad = []
    s = state(); s["S"][0, 1, 0] = 0; bad.append(s)            # user 0 on RRH 1 but A_0 = 0 (C5)
    s = state(); s["S"][0, 0, 0] = -1; bad.append(s)           # a hole before a user
    s = state(); s["S"][0, 0, 1] = 0; bad.append(s)            # user 0 twice on (0, 0)
    s = state(); s["S"][0, 0, 0] = 7; bad.append(s)            # no such user
    s = state(); s["A"][3] = 3; bad.append(s)                  # no such RRH
    s = state(); s["p"][0, 0, 0] = mask[0] * 1.01; bad.append(s)   # above the mask (C4)
    s = state(); s["p"][0, 0, 0] = -1e-6; bad.append(s)        # negative power
    s = state(); s["xi"] = -np.ones(M); bad.append(s)          # negative multiplier
    s = state(); s["zeta"] = np.full(Ks, 1e7); bad.append(s)   # zeta' above 1e6
    s = state(); s["zeta_sic"] = np.full(N * M, np.nan); bad.append(s)
    for i, s in enumerate(bad):
        assert call(s) == 1, i
    lib.hcran_destroy(h)


def test_set_wait_limit_validates_its_arguments():
    lib = hcran.load()
    inst = make_workload("small-3x8x6")[0]
    c, keep = _cfg(inst)
    arr = (hcran.Config * 1)(c)
    h = C.c_void_p()
    assert lib.hcran_create(C.byref(h), arr, 1, None) == 0
    assert lib.hcran_set_wait_limit(h, 0, -1) == 0
    assert lib.hcran_set_wait_limit(h, 1000, 0) == 0
    assert lib.hcran_set_wait_limit(h, -1, -1) == 1      # negative bound
    assert lib.hcran_set_wait_limit(h, 0, 1) == 1        # no instance 1
    assert lib.hcran_set_wait_limit(h, 0, -2) == 1
    assert lib.hcran_set_wait_limit(None, 0, -1) == 1
    lib.hcran_destroy(h)
