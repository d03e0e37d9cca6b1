"""The domain tuner (host only: it reads the library's shared-memory plans).

  * CTAs per SM count 2 KB per CTA beyond the plan (1 KB the hardware
    reserves, up to 1 KB of the kernels' static shared memory): a plan of
    115,648 bytes runs one CTA per SM, one of 113,000 bytes two.
  * Every tuned shape divides L, is 4 to 16 sites wide where L allows it,
    and its plan holds the legs the library wants (the sweep would stop with
    PMWA_ECAPACITY otherwise).
  * The choice has the most sites resident per SM among the admissible
    shapes (brute force over the divisors), ties to more warps per SM.
"""
import pytest

import paper_1307_0328_gb300 as P
from paper_1307_0328_gb300 import autotune as A


def test_residency_counts_static_shared_memory():
    assert A.per_sm(115648, 64) == 1
    assert A.per_sm(113000, 64) == 2
    assert A.per_sm(1000, 16) == 65536 // (128 * 64)
    assert A.per_sm(1000, 256) == 65536 // (128 * 256)


def _admissible(p):
    out = []
    L = int(p["Lx"])
    for s in range(2, 17):
        if L % s:
            continue
        if s < 4 and any(L % d == 0 for d in range(4, 17)):
            continue
        B = 2 if (s % 2 == 0 and s >= 4) else 0
        trial = dict(p, dom_x=s, dom_y=s, sub_block=B)
        try:
            plan = P.pmwa_tile_plan(**{k: v for k, v in trial.items() if k in P._lib.DEFAULTS})
        except P.PmwaError:
            continue
        if not plan["smem"] or plan["legcap"] < min(int(A.legs_wanted(trial, s * s)), 65000):
            continue
        k = A.per_sm(plan["smem"], s * s)
        out.append(((k * s * s, k * A._threads(s * s), s * s), s, plan))
    return out


CASES = [
    dict(Lx=48, Ly=48, beta=16.0, t=1.0, V=1.0, mu=-1.89, eta=0.1, legs_hint=171),
    dict(Lx=48, Ly=48, beta=16.0, t=1.0, V=1.0, mu=-1.89, eta=0.1, legs_hint=0),
    dict(Lx=64, Ly=64, beta=1.0, t=1.0, V=0.0, mu=0.3, eta=0.1),
    dict(Lx=24, Ly=24, beta=8.0, t=1.0, V=0.0, mu=0.5, eta=0.05, legs_hint=60),
    dict(Lx=16, Ly=16, beta=16.0, t=1.0, V=0.0, mu=0.15, eta=0.05),
]


@pytest.mark.parametrize("p", CASES)
def test_choice_is_the_best_admissible_shape(p):
    A._cache.clear()
    got = A.tune(p)
    adm = _admissible(p)
    assert adm, p
    best = max(adm, key=lambda a: a[0])
    assert got["dom_x"] == got["dom_y"] == best[1], (got, [(a[0], a[1]) for a in adm])


def test_replica_set_shapes_hold_their_legs():
    reps = A.replica_set(64)
    for p in reps:
        s = p["dom_x"]
        assert p["Lx"] % s == 0 and p["dom_y"] == s
        assert 4 <= s <= 16
        plan = P.pmwa_tile_plan(**{k: v for k, v in p.items() if k in P._lib.DEFAULTS})
        assert plan["legcap"] >= min(int(A.legs_wanted(p, s * s)), 65000), (p, plan)
    assert len({(p["Lx"], p["beta"]) for p in reps}) > 10
