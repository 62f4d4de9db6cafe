"""Pins of the penalty-form oracle (C10 / C11 kept with their multipliers,
``oracle/hcran_penalty.c``) against what the mathematics fixes:

- one link: the EE-optimal power of the Lambert-W closed form;
- no active penalty (one RRH, at most l users): the penalty form is the
  selection form's iteration with every user selected, so both oracles must
  agree to rounding;
- KKT stationarity of the Lagrangian of the penalty form, with C10 and C11
  multipliers active, by finite differences of an independent numpy model
  built from the documented constraint order;
- planted mistakes in a copy of the source fail these pins.
"""
import itertools
import math

import numpy as np
import pytest

import oracle.oracle as oo
from hcran_inputs import Tolerances
from tests import test_oracle_mutants as mut
from tests.test_oracle_pins import SIGMA, TIGHT, lambert_ee_opt, micro

LN2 = math.log(2.0)


@pytest.mark.parametrize("gain,pmax", [(2e-14, 10.0), (5e-15, 0.5)])
def test_penalty_single_link_is_lambert_w(gain, pmax):
    inst = micro([[[gain]]], pmax=[pmax], eta=[3.0], Pc=[2.0], Pf=[1.0])
    r = oo.penalty_solve(inst, TIGHT)
    g = float(np.float32(gain)) / SIGMA
    p_star = lambert_ee_opt(g, 3.0, 3.0, pmax)
    assert r.p[0, 0, 0] == pytest.approx(p_star, rel=1e-6)
    assert r.ee == pytest.approx(math.log2(1 + g * p_star) / (3.0 + 3.0 * p_star), rel=1e-9)
    assert r.c10_max == 0.0 and r.c11_max == 0.0


@pytest.mark.parametrize("seed", [3, 11, 7])
def test_penalty_without_active_penalty_equals_selection_form(seed):
    """One RRH and K = l users: no C10 pair, no C11 set, no inter-cell term
    (so C14 never binds), the same initial point mask / l on every link.  The
    selection form admits every user and then takes the same steps."""
    rng = np.random.default_rng(seed)
    G = (10.0 ** rng.uniform(-13.0, -12.0, size=(3, 1, 2))).astype(np.float32)
    inst = micro(G, l=2, pmax=[0.1], eta=[3.0])
    tol = Tolerances(tol_dinkelbach=0.0, tol_scale=0.0, tol_dual=0.0,
                     max_dinkelbach=3, max_scale=4, max_dual=60)
    pen = oo.penalty_solve(inst, tol)
    sel = oo.solve(inst, tol)
    assert np.all(sel.S >= 0)  # every user selected on every subcarrier
    dense = np.zeros((3, 1, 2))
    for n in range(3):
        for s in range(2):
            dense[n, 0, sel.S[n, 0, s]] = sel.p[n, 0, s]
    assert pen.iters == sel.iters
    assert np.allclose(pen.p, dense, rtol=1e-10, atol=0)
    assert pen.ee == pytest.approx(sel.ee, rel=1e-12)


def _lagrangian(inst, ph, q, xi, theta, theta2, rho_rel):
    """L(log p) of the penalty form at alpha = 1, beta = 0 (the first SCALE
    pass): sum log2 gamma - q sum eta p - xi'(C12) - theta (C10) - theta' (C11),
    written from Sec. II-A and the constraint order of hcran_penalty.c."""
    p = np.exp(ph)
    G = inst.G.astype(np.float64)
    N, M, K = G.shape
    l = inst.l
    mask = np.asarray(inst.pmax) / N
    val = 0.0
    for n in range(N):
        P = p[n].sum(axis=1)
        for m in range(M):
            for k in range(K):
                intra = sum(p[n, m, i] for i in range(K)
                            if i != k and (G[n, m, i] > G[n, m, k] or (G[n, m, i] == G[n, m, k] and i < k)))
                inter = sum(G[n, j, k] * P[j] for j in range(M) if j != m)
                val += math.log2(p[n, m, k] * G[n, m, k] / (SIGMA + G[n, m, k] * intra + inter))
    val -= q * float(np.sum(np.asarray(inst.eta)[None, :, None] * p))
    val -= float(np.sum(xi * (p.sum(axis=(0, 2)) - np.asarray(inst.pmax))))
    t = 0
    for k in range(K):
        for m in range(M):
            for m2 in range(m + 1, M):
                for n in range(N):
                    for n2 in range(N):
                        rho = rho_rel ** 2 * mask[m] * mask[m2]
                        val -= theta[t] * (p[n, m, k] * p[n2, m2, k] - rho)
                        t += 1
    assert t == len(theta)
    t = 0
    for n in range(N):
        for m in range(M):
            for S in itertools.combinations(range(K), l + 1):
                val -= theta2[t] * (np.prod([p[n, m, u] for u in S]) - (rho_rel * mask[m]) ** (l + 1))
                t += 1
    assert t == len(theta2)
    return val


@pytest.mark.parametrize("seed,l", [(5, 1), (8, 2)])
def test_penalty_kkt_stationarity_with_active_c10_c11(seed, l):
    """Fixed E, one SCALE pass (alpha = 1): at the converged point of the dual
    loop every interior link is a stationary point of the Lagrangian with the
    returned multipliers, which include active C10 and C11 terms."""
    rng = np.random.default_rng(seed)
    N, M, K = 2, 2, l + 2
    G = (10.0 ** rng.uniform(-13.5, -12.5, size=(N, M, K))).astype(np.float32)
    inst = micro(G, l=l, pmax=[1.0, 1.0], eta=[2.0, 2.0])
    rho_rel = 1e-2
    tol = Tolerances(tol_dinkelbach=0.0, tol_scale=0.0, tol_dual=1e-7,
                     max_dinkelbach=1, max_scale=1, max_dual=400000)
    q = 0.2  # low enough that the inner solve ends above its start (no keep rule, no projection)
    r = oo.penalty_solve(inst, tol, rho_rel=rho_rel, q_init=q)
    assert r.iters[2] < 400000, "dual loop did not converge"
    assert r.slack_power_min > 0.0
    assert np.max(r.theta) > 0 and np.max(r.theta2) > 0
    mask = np.asarray(inst.pmax) / N
    ph = np.log(r.p)
    h = 1e-6
    checked = 0
    for idx in np.ndindex(N, M, K):
        pe, mk = r.p[idx], mask[idx[1]]
        if not (2e-9 * mk < pe < mk * (1 - 1e-6)):
            continue
        up, dn = ph.copy(), ph.copy()
        up[idx] += h
        dn[idx] -= h
        grad = (_lagrangian(inst, up, q, r.xi, r.theta, r.theta2, rho_rel) -
                _lagrangian(inst, dn, q, r.xi, r.theta, r.theta2, rho_rel)) / (2 * h)
        assert abs(grad) < 1e-4 / LN2, (idx, grad)  # measured <= 3.3e-6
        checked += 1
    assert checked >= 3


PEN_MUTANTS = {
    "c11_term_dropped": ("if (in) den += s->th11[((size_t)n * M + m) * I->nsub + c] * prod;",
                         "(void)in;"),
    "c10_partner_transposed": ("den += s->th10[t] * s->p[((size_t)n2 * M + m2) * K + k];",
                               "den += s->th10[t] * s->p[((size_t)n * M + m) * K + k];"),
    "victims_other_rrh_gain_transposed": (
        "for (int i = 0; i < K; i++) den += s->pi[((size_t)n * M + j) * K + i] * gain(I, n, m, i);",
        "for (int i = 0; i < K; i++) den += s->pi[((size_t)n * M + j) * K + i] * gain(I, n, j, i);"),
}


@pytest.mark.parametrize("name", sorted(PEN_MUTANTS))
def test_penalty_pins_catch_mutant(tmp_path, monkeypatch, name):
    find, repl = PEN_MUTANTS[name]
    so = mut.build_mutant(tmp_path, name, find, repl, target=mut.SRC_PEN)
    monkeypatch.setattr(oo, "_lib", None)
    monkeypatch.setattr(oo, "build", lambda force=False: so)
    failed = []
    for pin in (lambda: test_penalty_kkt_stationarity_with_active_c10_c11(5, 1),
                lambda: test_penalty_kkt_stationarity_with_active_c10_c11(8, 2)):
        try:
            pin()
        except Exception as exc:
            failed.append(repr(exc)[:80])
    assert failed, "no pin caught mutant %s" % name
