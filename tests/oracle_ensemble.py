"""Perturbation ensemble of the FP64 oracle, for the parity tests.

The end point of the method can depend on rounding.  When an Algorithm 1 pass
ends on an iteration cap, the primal iterate of the dual subgradient loop is
clipped at the mask or at the floor on many links, and a rounding-level
difference can pick a different clip pattern; the last Dinkelbach pass of
most instances is such a pass (it is the one that lowers the EE while it
serves the streaming users).  There no FP32 implementation, and no re-ordered
FP64 one, can be held to the plain oracle's end point.  What the method does
fix is the set of end points the oracle itself reaches when its arithmetic
carries rounding-level perturbations.

``ensemble`` returns the plain oracle result first, then ``n`` results in
which every new power of a dual iteration is scaled by (1 + NOISE_REL * u),
u uniform in [-1, 1), NOISE_REL = 2^-24 (the FP32 unit roundoff), one stream
per seed 1..n.  For an instance whose end point is stable all members agree
to ~1e-8 and the ensemble bar is the plain one.
"""
import multiprocessing as mp
import os

import oracle

NOISE_REL = 2.0 ** -24


def _one(args):
    inst, tol, kw, seed, noise = args
    if seed == 0:
        return oracle.solve(inst, tol, **kw)
    return oracle.solve(inst, tol, noise_rel=noise, noise_seed=seed, **kw)


def ensemble(inst, tol, n=7, noise_rel=NOISE_REL, **kw):
    """Plain oracle result, then n perturbed ones (seeds 1..n) with relative
    noise noise_rel on every new dual-iteration power."""
    oracle.build()  # compile once before the workers start
    jobs = [(inst, tol, kw, s, noise_rel) for s in range(n + 1)]
    procs = max(1, min(len(jobs), os.cpu_count() or 1))
    with mp.get_context("spawn").Pool(procs) as pool:  # spawn: the parent may hold a CUDA context
        return pool.map(_one, jobs, chunksize=1)
