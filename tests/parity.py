"""The parity bar between a CUDA result and the FP64 oracle, and the validity
checks that every result must pass on its own.

Test infrastructure only.  An instance meets the bar in one of four ways:

``plain``
    Against the plain oracle: the RRH choice A_k equal for every served user;
    on every (n, m) the same users, apart from vanishing links (present on one
    side only and carrying less than ``VANISH`` of the RRH's mask, so they
    move neither R nor P beyond rounding); the same status bits; EE within ``EE_RTOL``; every power
    of a link both sides select within ``P_RTOL`` relative, plus an absolute
    allowance for powers far below the mask: 1e-6 of the mask when both
    sides run the same iteration counts, else the dual loop's own stopping
    tolerance varpi_1 (the method fixes a power only to max |dp| / mask <
    varpi_1, so two runs that stop one iteration apart differ by that much).

``tie``
    A selection decision on either side had a relative margin below
    ``TIE_BAND`` (1e-9, the band of the target precision): the two sides may
    break the tie differently.  The result must pass ``validity`` and its EE
    error is reported.

``stop``
    A tolerance-driven stop test (the dual loop's varpi_1, the SCALE loop's
    varpi_2, the Dinkelbach test) fired at a different iteration on the two
    sides, so the iteration counts differ: the two end points then differ by
    the tolerance in the directions the method resolves slowly (powers far
    below the mask), which later selections can turn into a different link
    of small power.  The EE must still be within ``EE_RTOL`` of the plain
    oracle, and the result must pass ``validity``.

``sensitive``
    The oracle's own end point moves under FP32-level rounding: its
    perturbation ensemble (every new dual-iteration power scaled by
    1 + 2^-24 u) spreads the EE by more than ``EE_RTOL``.  This is a property
    of the instance, not of the CUDA path; the result must pass ``validity``
    and its EE error is reported.

Anything else fails.  Every report carries the EE error against the plain
oracle, so the suites print the error for every result.
"""
from __future__ import annotations

import numpy as np

from tests import exact_model as em

TIE_BAND = 1e-9
EE_RTOL = 1e-4
P_RTOL = 1e-3
VANISH = 1e-4


def _links(S, p, n, m):
    return {int(k): float(p[n, m, s]) for s, k in enumerate(S[n, m]) if k >= 0}


def selection_diff(inst, g, o):
    """(equal, report): selection equality up to vanishing links, A on served users."""
    mask = inst.pmax / inst.N
    served = set(int(k) for k in g["S"][g["S"] >= 0]) | set(int(k) for k in o.S[o.S >= 0])
    a_diff = [k for k in sorted(served) if g["A"][k] != o.A[k]]
    vanishing, differ = 0, []
    for n in range(inst.N):
        for m in range(inst.M):
            lg, lo = _links(g["S"], g["p"], n, m), _links(o.S, o.p, n, m)
            if lg.keys() == lo.keys():
                continue
            for k in lg.keys() ^ lo.keys():
                pw = lg.get(k, lo.get(k))
                if pw < VANISH * mask[m]:
                    vanishing += 1
                else:
                    differ.append((n, m, k, pw / mask[m]))
    return (not a_diff and not differ), dict(a_diff=a_diff[:8], link_diff=differ[:8], vanishing=vanishing)


def power_error(inst, g, o, p_abs=1e-6):
    """Max relative error of the powers of links both sides select, and the
    worst link's excess over the bar (<= 1 passes); p_abs is the absolute
    allowance in units of the mask."""
    mask = inst.pmax / inst.N
    worst, excess = 0.0, 0.0
    for n in range(inst.N):
        for m in range(inst.M):
            lg, lo = _links(g["S"], g["p"], n, m), _links(o.S, o.p, n, m)
            for k in lg.keys() & lo.keys():
                a, b = lg[k], lo[k]
                lim = P_RTOL * max(a, b) + p_abs * mask[m]
                worst = max(worst, abs(a - b) / max(b, 1e-300))
                excess = max(excess, abs(a - b) / lim)
    return worst, excess


def validity(inst, r, label="", ref=None):
    """The result on its own: C1 (at most l distinct users per (n, m), packed,
    in SIC order), C5 (a user only on its RRH), C4 (0 < p <= mask), C12
    after the projection, C14 in divided form (max Omega_bar / mask: the
    multiplier method enforces it in the limit, so it is held to 1e-2, or to
    the oracle result `ref`'s own value plus 1e-2), the streaming status bit
    against the reported slack, and the reported EE against R / P recomputed
    from S and p by the independent model."""
    S, p, A = np.asarray(r["S"]), np.asarray(r["p"], dtype=np.float64), np.asarray(r["A"])
    N, M, l = S.shape
    mask = inst.pmax / inst.N
    for n in range(N):
        for m in range(M):
            ids = [int(k) for k in S[n, m] if k >= 0]
            assert all(k >= 0 for k in S[n, m, :len(ids)]), (label, "C1 packing", n, m)
            assert len(set(ids)) == len(ids) <= l, (label, "C1", n, m)
            g = [float(inst.G[n, m, k]) for k in ids]
            assert all(g[i] > g[i + 1] or (g[i] == g[i + 1] and ids[i] < ids[i + 1]) for i in range(len(ids) - 1)), \
                (label, "SIC order", n, m)
            for s, k in enumerate(ids):
                assert A[k] == m, (label, "C5", n, m, k)
                assert 0.0 < p[n, m, s] <= mask[m] * (1 + 1e-6), (label, "C4", n, m, s)
    P = em.dense_power(S, p, inst.K)
    assert np.all(P.sum(axis=(0, 2)) <= inst.pmax * (1 + 1e-5)), (label, "C12")
    sic_bar = 1e-2 + (max(ref.slack_sic_max, 0.0) if ref is not None else 0.0)
    assert r["slack_sic_max"] < sic_bar, (label, "C14", r["slack_sic_max"], sic_bar)
    if inst.Ks:
        assert bool(r["status"] & 2) == (r["slack_rate_min"] < -1e-3), (label, "status vs C13 slack")
    R, Pt = em.R_P(inst, P)
    assert np.isfinite(r["ee"]) and r["ee"] >= 0.0, label
    assert abs(r["ee"] - R / Pt) <= 1e-5 * max(R / Pt, 1e-12), (label, "EE vs model", r["ee"], R / Pt)


def check(inst, g, o, label="", p_abs=1e-6):
    """Plain-bar report of one result against one oracle result."""
    same, sel = selection_diff(inst, g, o)
    ee_err = abs(g["ee"] - o.ee) / max(abs(o.ee), 1e-300)
    p_err, p_excess = power_error(inst, g, o, p_abs)
    rep = dict(label=label, ee_gpu=g["ee"], ee_orc=o.ee, ee_rel=ee_err, p_maxrel=p_err, p_excess=p_excess,
               same_selection=same, sel=sel, margin_gpu=g["min_margin"], margin_orc=o.min_margin,
               status=(g["status"], o.status), iters_gpu=tuple(g["iters"]), iters_orc=tuple(o.iters))
    # the status bits (Dinkelbach cap, streaming rate unmet, EE below an
    # earlier iterate) are part of the result
    rep["ok"] = bool(same and ee_err <= EE_RTOL and p_excess <= 1.0 and (g["status"] & 7) == (o.status & 7))
    return rep


def classify(inst, g, o, tol, label="", ensemble_fn=None, **solve_kw):
    """Tier of one result: 'plain', 'tie', 'stop', 'sensitive' or 'fail', with the report."""
    rep = check(inst, g, o, label, p_abs=max(1e-6, tol.tol_dual))
    if rep["ok"]:
        validity(inst, g, label, ref=o)
        return "plain", rep
    validity(inst, g, label, ref=o)
    if min(g["min_margin"], o.min_margin) < TIE_BAND:
        return "tie", rep
    if tuple(g["iters"]) != tuple(o.iters) and rep["ee_rel"] <= EE_RTOL:
        return "stop", rep
    if ensemble_fn is not None:
        ees = np.array([x.ee for x in ensemble_fn(inst, tol, **solve_kw)])
        spread = float((ees.max() - ees.min()) / max(abs(ees[0]), 1e-300))
        rep["ensemble_ee_spread"] = spread
        if spread > EE_RTOL:
            return "sensitive", rep
    return "fail", rep
