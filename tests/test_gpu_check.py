"""The device invariant check (pmwa_check).

The invariants are those of a worldline configuration with worms: every key a
bond leg or a worm, strictly increasing times per site, a state continuous
around every circle with the base state equal to the state above the last
event, each leg's partner at the same time on the other site of its bond,
particle conservation at every vertex.  Steps 2-5 keep them all.

  * On the CPU: the planted faults below are real faults, i.e. the oracle's
    own check (which runs on import) rejects them, while the host-side check
    of pmwa_import's format (tags, order, continuity, base) passes them, so
    they reach the device check.
  * On the GPU: the check holds after Step 2 and after Steps 3, 4, 5 and 6
    of every sweep on the parity geometries, after sweeps of the 256x256
    workload and on every replica of a batch; on a planted fault it names
    the lowest failing site and the failing invariant.
"""
import numpy as np
import pytest

from oracle import oracle as O

import paper_1307_0328_gb300 as P

PARTNER, CONSERVATION = 7, 8


def _sites(buf):
    """Canonical configuration -> [base, [keys]] per site."""
    N, k, out = int(buf[0]), 1, []
    for _ in range(N):
        hd = int(buf[k])
        n = hd & 0x7fffffff
        out.append([hd >> 63, [int(x) for x in buf[k + 1:k + 1 + n]]])
        k += 1 + n
    return out


def _pack(sites):
    words = [len(sites)]
    for base, keys in sites:
        words.append(len(keys) | (base << 63))
        words.extend(keys)
    return np.array(words, dtype=np.uint64)


def _is_leg(key):
    return ((key >> 2) & 7) <= 5


def _partner_site(sites, s, key):
    """The one other site holding a key at the same time and tag."""
    pk = key >> 2
    found = [o for o, (_, keys) in enumerate(sites) if o != s and any((x >> 2) == pk for x in keys)]
    assert len(found) == 1, found
    return found[0]


def plant_partner_fault(buf):
    """Move one vertex leg to the next time grid point (order and states
    kept): its vertex loses the partner leg on both sites.  Returns the
    edited buffer and the lowest site that fails."""
    sites = _sites(buf)
    for s, (_, keys) in enumerate(sites):
        for k, key in enumerate(keys):
            if not _is_leg(key):
                continue
            m = key >> 5
            moved = ((m + 1) << 5) | (key & 31)
            if m + 1 >= 1 << 59 or (k + 1 < len(keys) and (moved >> 2) >= (keys[k + 1] >> 2)):
                continue
            o = _partner_site(sites, s, key)
            keys[k] = moved
            return _pack(sites), min(s, o)
    raise AssertionError("no vertex leg to move")


def plant_conservation_fault(buf):
    """Flip the occupation of the interval between two consecutive vertex
    legs of one site (state above the first, state below the second):
    continuity and the base state still hold, but both vertices stop
    conserving particles.  Returns the edited buffer and the lowest site
    that fails."""
    sites = _sites(buf)
    for s, (_, keys) in enumerate(sites):
        for k in range(len(keys) - 1):
            a, b = keys[k], keys[k + 1]
            if not (_is_leg(a) and _is_leg(b)):
                continue
            o1, o2 = _partner_site(sites, s, a), _partner_site(sites, s, b)
            keys[k], keys[k + 1] = a ^ 1, b ^ 2
            return _pack(sites), min(s, o1, o2)
    raise AssertionError("no two consecutive vertex legs")


def _host_format_ok(buf):
    """The checks pmwa_import makes on the host, restated: tags, strictly
    increasing times, continuity, base state."""
    for base, keys in _sites(buf):
        n = len(keys)
        for k, key in enumerate(keys):
            if (key >> 2) & 7 == 6:
                return False
            if k and (keys[k - 1] >> 2) >= (key >> 2):
                return False
            nx = keys[(k + 1) % n]
            below_next = (1 - (nx & 1)) if (nx >> 2) & 7 == 7 else (nx >> 1) & 1
            if (key & 1) != below_next:
                return False
        if n and base != (keys[-1] & 1):
            return False
    return True


PLANT_KW = dict(Lx=8, Ly=8, beta=2.0, eta=0.3, V=1.0, mu=0.7, dom_x=4, dom_y=4, sub_block=2, n_cycle=5,
                exchange_every=1, seed=5)


@pytest.mark.parametrize("plant", [plant_partner_fault, plant_conservation_fault])
def test_planted_faults_are_faults(plant):
    o = O.Oracle(**PLANT_KW)
    o.sweep(6)
    good = o.export()
    bad, _ = plant(good)
    assert _host_format_ok(good) and _host_format_ok(bad)
    fresh = O.Oracle(**PLANT_KW)
    fresh.import_(good)
    with pytest.raises(RuntimeError, match="status 5"):
        fresh.import_(bad)


CHECK_GEOMS = [
    dict(Lx=2, Ly=2, beta=1.5, eta=0.5, n_cycle=4, seed=3, init=0),
    dict(Lx=8, Ly=8, beta=2.0, eta=0.3, V=1.0, mu=0.7, dom_x=4, dom_y=4, sub_block=2, n_cycle=5,
         exchange_every=1, seed=5),
    dict(Lx=16, Ly=16, beta=4.0, eta=0.1, dom_x=8, dom_y=8, sub_block=4, n_cycle=8, exchange_every=2, seed=7,
         init=1, init_seed=7),
    dict(Lx=8, Ly=8, beta=2.0, eta=0.2, V=3.0, mu=4.2, dom_x=4, dom_y=4, sub_block=2, n_cycle=4, seed=9, init=2),
    dict(Lx=6, Ly=9, beta=4.0, eta=0.15, t=0.0, c_off=0.3, mu=0.8, dom_x=3, dom_y=3, n_cycle=3, seed=11),
    dict(Lx=12, Ly=4, beta=3.0, eta=0.25, V=3.0, mu=-1.5, t=0.7, dom_x=6, dom_y=2, sub_block=2, n_cycle=4, seed=13),
    dict(Lx=32, Ly=32, beta=4.0, eta=0.25, dom_x=16, dom_y=16, sub_block=2, n_cycle=8, exchange_every=2, seed=19,
         init=1, init_seed=9),
]


@pytest.mark.gpu
@pytest.mark.parametrize("kw", CHECK_GEOMS)
def test_check_holds_after_every_step(kw):
    g = P.Sim(**kw)
    nd = (kw["Lx"] // kw.get("dom_x", kw["Lx"])) * (kw["Ly"] // kw.get("dom_y", kw["Ly"]))
    K = kw.get("exchange_every", 2)
    try:
        assert g.check() is None
        for s in range(24):
            g.sweep_index = s
            if nd > 1 and s % K == 0:
                g.boundary()
                assert g.check() is None, (s, "boundary")
            snap = g.export()
            for stop in (3, 4, 5, 6):
                g.import_(snap)
                g.sweep_index = s
                g.tile(stop)
                assert g.check() is None, (s, stop)
    finally:
        g.close()


@pytest.mark.gpu
def test_check_holds_on_the_256x256_workload_and_a_batch():
    g = P.Sim(Lx=256, Ly=256, beta=4.0, eta=0.1, dom_x=16, dom_y=16, sub_block=2, exchange_every=2,
              n_cycle=31, init=1, init_seed=7, seed=7)
    try:
        for _ in range(3):
            g.sweep(10)
            assert g.check() is None
    finally:
        g.close()
    reps = [dict(Lx=L, Ly=L, beta=b, eta=0.1, V=float(i % 2), mu=0.3 * (i % 3), dom_x=8, dom_y=8, sub_block=2,
                 n_cycle=8, seed=40 + i, replica=i, init=1, init_seed=i)
            for i, (L, b) in enumerate([(16, 1.0), (24, 2.0), (32, 4.0), (48, 2.0), (64, 1.0), (16, 8.0)])]
    b = P.Batch(reps)
    try:
        b.sweep(20)
        for i in range(len(reps)):
            assert b.check(i) is None, i
    finally:
        b.close()


@pytest.mark.gpu
@pytest.mark.parametrize("plant,code", [(plant_partner_fault, PARTNER), (plant_conservation_fault, CONSERVATION)])
def test_check_names_a_planted_fault(plant, code):
    """The edited configuration passes pmwa_import's host-side format check;
    the device check names the lowest failing site and the invariant.  No
    sweep runs on it."""
    g = P.Sim(**PLANT_KW)
    try:
        g.sweep(6)
        good = g.export()
        bad, site = plant(good)
        g.import_(bad)
        assert g.check() == (site, code)
        assert P.CHECK_NAMES[code] in ("partner", "conservation")
        g.import_(good)
        assert g.check() is None
    finally:
        g.close()
