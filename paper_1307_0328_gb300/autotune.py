"""Domain-shape tuning and the synthetic replica sets of the batched workloads.

The tuner picks, per instance, the domain edge and the Step-5 sub-block edge.
A CTA's time is set mostly by per-site chains (the legs of one site are
handled in order), which do not depend on the domain's size, so a batch's
throughput follows the number of sites resident per SM: CTAs per SM (shared
memory of the plan, pmwa_tile_smem; up to 128 registers a thread; the 32-CTA
limit) times the sites of a domain.  Among the square domains that divide L,
at most 16 and at least 4 sites wide when the lattice allows it, the tuner
takes the most sites per SM, then the most warps per SM, then the larger
domain (fewer bonds between domains), with 2x2 shifted sub-blocks.  A
measured leg count (legs_hint) shrinks the plan.  Results are cached per
(L, beta, t, V, mu, eta, c_off, legs_hint) class.  N_cycle follows the rule
that every vertex leg is reached about once per sweep on average,
N_cycle = ceil(2 <n_v> / <n_w>), from a short pilot of the instance itself,
capped at 512.
"""
import math

import numpy as np

from . import _lib

SM_SMEM = 228 * 1024
_cache = {}


def _divisors(L):
    return [s for s in range(L, 1, -1) if L % s == 0]


def _threads(sites, smem=None):
    """Threads of the sweep kernel's CTA for a domain plan, as the library
    picks them: 64, 128 or 256 by the domain's sites, 512 for a large domain
    whose plan leaves room for one CTA per SM."""
    if sites <= 32:
        return 64
    if sites <= 96:
        return 128
    return 512 if smem is not None and SM_SMEM // (smem + 2048) <= 1 else 256


def per_sm(smem, sites):
    """CTAs of a domain plan per SM: shared memory (1 KB the hardware
    reserves a CTA, up to 1 KB of the kernels' static shared memory),
    registers (up to 128 a thread) and the 32-CTA limit."""
    by_regs = 65536 // (128 * _threads(sites, smem))
    return min(SM_SMEM // (smem + 2048), by_regs, 32)


def legs_wanted(p, sites):
    """Vertex legs the library plans a domain's leg table for: the measured
    mean (legs_hint per site) plus 8 standard deviations, else 1.1 times the
    bound 4 beta (D + t) per site (D the largest diagonal vertex density)."""
    hint = int(p.get("legs_hint", 0) or 0)
    if hint > 0:
        m = float(hint) * sites
        return m + 8.0 * math.sqrt(m) + 128.0
    D = _lib.pmwa_tables(**{k: v for k, v in p.items() if k in _lib.DEFAULTS})["D"]
    return 1.1 * 4.0 * float(p["beta"]) * (D + float(p.get("t", 1.0))) * sites + 256.0


def tune(p):
    """dom_x, dom_y, sub_block for one parameter dict (square lattices)."""
    key = tuple(round(float(p.get(k, d)), 9) for k, d in
                [("Lx", 8), ("Ly", 8), ("beta", 2.0), ("t", 1.0), ("V", 0.0), ("mu", 0.0), ("eta", 0.2),
                 ("c_off", -1.0), ("legs_hint", 0)])
    if key in _cache:
        return dict(_cache[key])
    Lx, Ly = int(p["Lx"]), int(p["Ly"])
    best, best_score = None, None
    for sx in _divisors(Lx):
        if sx > 16 or (sx < Lx and sx < 2):
            continue
        sy = sx if Ly % sx == 0 else Lx if Lx == Ly else None
        if sy is None or (sy < Ly and sy < 2):
            continue
        if min(sx, sy) < 4 and any(d >= 4 and d <= 16 for d in _divisors(Lx)):
            continue
        B = 2 if (sx % 2 == 0 and sy % 2 == 0 and min(sx, sy) >= 4) else 0
        trial = dict(p, dom_x=sx, dom_y=sy, sub_block=B)
        try:
            plan = _lib.pmwa_tile_plan(**{k: v for k, v in trial.items() if k in _lib.DEFAULTS})
        except _lib.PmwaError:
            continue  # no plan fits shared memory
        sm = plan["smem"]
        sites = sx * sy
        # the plan must hold the legs it is made for (else the sweep stops
        # with PMWA_ECAPACITY)
        if not sm or plan["legcap"] < min(int(legs_wanted(trial, sites)), 65000):
            continue
        k = per_sm(sm, sites)
        score = (k * sites, k * _threads(sites, sm), sites)
        if best_score is None or score > best_score:
            best, best_score = dict(dom_x=sx, dom_y=sy, sub_block=B), score
    if best is None:
        raise ValueError("no domain shape fits shared memory for %r" % (p,))
    _cache[key] = best
    return dict(best)


def n_cycle_rule(p, rows):
    """N_cycle of instance p from measured rows (pmwa_n_cycle: ceil(2 <n_v> /
    <n_w>), capped at 512 passes for instances with almost no worms, which
    lie far outside the O(10)-O(100) worms per domain the method is made
    for)."""
    return _lib.n_cycle(_lib.make_params(**{k: v for k, v in p.items() if k in _lib.DEFAULTS}), rows)


def replica_set(n=512, seed=3):
    """The batched workload: n independent hard-core Bose-Hubbard instances,
    L from {16, 24, 32, 48, 64}, beta t from {1, 2, 4, 8, 16}, mu uniform in
    [-2, 2], V from {0, 1}, eta from {0.05, 0.1, 0.2}, drawn with numpy's
    Philox generator keyed by `seed`; each instance gets its own Monte Carlo
    seed and replica id and a half-filled random start."""
    rng = np.random.Generator(np.random.Philox(seed))
    L = rng.choice([16, 24, 32, 48, 64], n)
    beta = rng.choice([1.0, 2.0, 4.0, 8.0, 16.0], n)
    mu = rng.uniform(-2.0, 2.0, n)
    V = rng.choice([0.0, 1.0], n)
    eta = rng.choice([0.05, 0.1, 0.2], n)
    out = []
    for i in range(n):
        p = dict(Lx=int(L[i]), Ly=int(L[i]), beta=float(beta[i]), t=1.0, V=float(V[i]), mu=float(mu[i]),
                 eta=float(eta[i]), seed=100000 + i, replica=i, init=1, init_seed=200000 + i,
                 exchange_every=2, n_cycle=16)
        p.update(tune(p))
        out.append(p)
    return out
