"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs, bit for bit in configuration and integer counters, FP64
estimators within 1e-12 relative (summation order differs).

Each step of the paper's pseudo code is checked on its own from the same
imported configuration (Step 2 + boundary Step 3; Steps 3, 3-4, 3-5, 3-6),
and whole sweeps are checked sweep by sweep.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402

import paper_1307_0328_gb300 as P  # noqa: E402

REL = 1e-12
# integer fields of a measurement row, compared exactly
ROW_FIELDS = ("sweep", "n_v", "n_k", "n_w", "occ_lo", "occ_hi", "w_dom_min", "dom_empty")

GEOMS = [
    # the 8x8, beta t = 2, eta = 0.2 workload, one domain
    dict(Lx=8, Ly=8, beta=2.0, eta=0.2, n_cycle=6, seed=1, init=1, init_seed=1),
    # 2x2 lattice (every pair carries two bonds), empty start
    dict(Lx=2, Ly=2, beta=1.5, eta=0.5, n_cycle=4, seed=3, init=0),
    # domains + sub-blocks, non-zero V and mu
    dict(Lx=8, Ly=8, beta=2.0, eta=0.3, V=1.0, mu=0.7, dom_x=4, dom_y=4, sub_block=2,
         n_cycle=5, exchange_every=1, seed=5),
    # 16x16 in 8x8 domains (the 256x256 workload in small), K = 2
    dict(Lx=16, Ly=16, beta=4.0, eta=0.1, dom_x=8, dom_y=8, sub_block=4, n_cycle=8,
         exchange_every=2, seed=7, init=1, init_seed=7),
    # checkerboard start, large V and mu (the checkerboard-solid regime), domains
    dict(Lx=8, Ly=8, beta=2.0, eta=0.2, V=3.0, mu=4.2, dom_x=4, dom_y=4, sub_block=2, n_cycle=4,
         seed=29, init=2),
    # odd sizes, non-square domains, t = 0 and a long circle
    dict(Lx=6, Ly=9, beta=4.0, eta=0.15, t=0.0, c_off=0.3, mu=0.8, dom_x=3, dom_y=3,
         n_cycle=3, seed=11),
    # large V, negative mu, bounce-rich directed loops
    dict(Lx=12, Ly=4, beta=3.0, eta=0.25, V=3.0, mu=-1.5, t=0.7, dom_x=6, dom_y=2,
         sub_block=2, n_cycle=4, seed=13),
    # many worms and a tight leg-count hint: the domain's configuration
    # (legs + worms) overflows the shared-memory staging area after the first
    # sweep, so Steps 3 read it from HBM instead
    dict(Lx=8, Ly=8, beta=2.0, t=0.5, eta=4.0, n_cycle=4, seed=23, init=1, init_seed=3, legs_hint=5),
    # beta t = 16 on one 16x16 domain: the leg table fills shared memory, so
    # the plan leaves out the partner table and Step 5 searches for partners
    dict(Lx=16, Ly=16, beta=16.0, eta=0.1, sub_block=2, n_cycle=8, seed=47, init=1, init_seed=4),
    # one 32x32 domain (four sites a thread) at high density: many sites are
    # occupied all the time, so a thread's occupied time exceeds 2^64 grid
    # units and needs its 128-bit sum
    dict(Lx=32, Ly=32, beta=0.25, eta=0.1, mu=8.0, n_cycle=3, seed=41, init=1, init_seed=2),
    # more than 32 worms per domain: the block-wide Step-5 passes (the cases
    # above hold fewer and take the one-warp passes)
    dict(Lx=16, Ly=16, beta=4.0, eta=0.3, sub_block=2, n_cycle=6, seed=17, init=1, init_seed=5),
    dict(Lx=32, Ly=32, beta=4.0, eta=0.25, dom_x=16, dom_y=16, sub_block=2, n_cycle=8,
         exchange_every=2, seed=19, init=1, init_seed=9),
    # more than 255 passes of the block-wide grouping: its per-chunk counts
    # carry a pass stamp that starts over every 255 passes
    dict(Lx=16, Ly=16, beta=2.0, eta=0.5, sub_block=2, n_cycle=300, seed=53, init=1, init_seed=6),
    # one Step-5 group of 64 to 128 worms (sub_block 0: the whole domain): a
    # move may wait for a predecessor 64 or more ranks before it
    dict(Lx=8, Ly=8, beta=4.0, eta=0.45, sub_block=0, n_cycle=6, seed=59, init=1, init_seed=8),
]
MANY_WORMS = GEOMS[-4:]


def _pair(kw):
    return P.Sim(**kw), O.Oracle(**kw)


def _same(a, b, what):
    if not np.array_equal(a, b):
        n = min(len(a), len(b))
        diff = np.nonzero(a[:n] != b[:n])[0]
        first = int(diff[0]) if len(diff) else n
        raise AssertionError("%s: %d vs %d words, first difference at word %d" % (what, len(a), len(b), first))


@pytest.mark.parametrize("kw", GEOMS)
def test_steps_bit_exact(kw):
    """From the same configuration, every step on its own."""
    g, o = _pair(kw)
    nd = (kw["Lx"] // (kw.get("dom_x") or kw["Lx"])) * (kw["Ly"] // (kw.get("dom_y") or kw["Ly"]))
    for s in range(6):
        snap = o.export()
        if nd > 1:
            g.import_(snap); g.sweep_index = s
            o.boundary(); g.boundary()
            _same(g.export(), o.export(), "Step 2 at sweep %d" % s)
            snap = o.export()
        for stop in (3, 4, 5, 6):
            o.import_(snap); o.sweep_index = s
            g.import_(snap); g.sweep_index = s
            o.tile(stop); g.tile(stop)
            _same(g.export(), o.export(), "Steps 3..%d at sweep %d" % (stop, s))
        ro, rg = o.rows(), g.rows()
        assert len(ro) == 1 and len(rg) == 1
        for f in ROW_FIELDS:
            assert ro[f][0] == rg[f][0], f
        assert rg["q_impr"][0] == pytest.approx(ro["q_impr"][0], rel=REL)
        o.sweep_index = s + 1


@pytest.mark.parametrize("kw", GEOMS)
def test_sweeps_bit_exact(kw):
    """Whole sweeps from the initial state, compared after every sweep."""
    g, o = _pair(kw)
    for s in range(12):
        o.sweep(1)
        g.sweep(1)
        _same(g.export(), o.export(), "after sweep %d" % s)
    ro, rg = o.rows(), g.rows()
    for f in ROW_FIELDS:
        assert np.array_equal(ro[f], rg[f]), f
    assert np.allclose(rg["q_impr"], ro["q_impr"], rtol=REL, atol=0)


def test_rho_slices_match():
    kw = GEOMS[2]
    g, o = _pair(kw)
    o.sweep(5)
    g.sweep(5)
    assert np.allclose(g.rho_slices(8), o.rho_slices(8), rtol=REL, atol=0)


def test_green_functions_match_oracle_densities():
    """pmwa_green against the same correlators taken in numpy from the CPU
    oracle's worm densities of the same configuration (within 1e-12)."""
    kw = dict(Lx=12, Ly=8, beta=3.0, eta=0.3, V=0.5, mu=0.2, dom_x=6, dom_y=4, sub_block=2, n_cycle=4, seed=31)
    g, o = _pair(kw)
    o.sweep(4)
    g.sweep(4)
    K, rmax = 5, 4
    gx, gy, pl = P.pmwa_green(g.h, K, rmax)
    r = o.rho_slices(K)
    Lx, Ly = kw["Lx"], kw["Ly"]
    idx = np.arange(Lx * Ly)
    x, y = idx % Lx, idx // Lx
    eta = kw["eta"]
    for d in range(1, rmax + 1):
        ex = (r * r[(x + d) % Lx + Lx * y]).mean() / eta ** 2
        ey = (r * r[x + Lx * ((y + d) % Ly)]).mean() / eta ** 2
        assert gx[d - 1] == pytest.approx(ex, rel=1e-12)
        assert gy[d - 1] == pytest.approx(ey, rel=1e-12)
    p4 = (r * r[(x + 1) % Lx + Lx * y] * r[x + Lx * ((y + 1) % Ly)] * r[(x + 1) % Lx + Lx * ((y + 1) % Ly)]).mean()
    assert pl == pytest.approx(p4 / eta ** 4, rel=1e-12)


def test_many_sweeps_8x8_one_domain():
    """Config-1 shape over 200 sweeps: configuration identical at the end."""
    kw = dict(Lx=8, Ly=8, beta=2.0, eta=0.2, n_cycle=8, seed=1, init=1, init_seed=1)
    g, o = _pair(kw)
    o.sweep(200)
    g.sweep(200)
    _same(g.export(), o.export(), "after 200 sweeps")
    ro, rg = o.rows(), g.rows()
    assert np.array_equal(ro["n_v"], rg["n_v"]) and np.array_equal(ro["n_w"], rg["n_w"])


def test_capacity_overflow_is_reported():
    """A per-site slot far too small makes pmwa_sweep return PMWA_ECAPACITY
    (no device fault); the handle stays usable for queries."""
    g = P.Sim(Lx=8, Ly=8, beta=8.0, eta=0.2, n_cycle=2, cap_site=8)
    with pytest.raises(P.PmwaError) as e:
        g.sweep(3)
    assert e.value.status == P.PMWA_ECAPACITY
    assert g.sweep_index >= 0


def test_rows_buffer_full_is_reported():
    g = P.Sim(Lx=4, Ly=4, rows_cap=4, n_cycle=1)
    g.sweep(4)
    with pytest.raises(P.PmwaError) as e:
        g.sweep(1)
    assert e.value.status == P.PMWA_EROWS
    assert len(g.rows()) == 4
    g.sweep(1)


@pytest.mark.parametrize("kw", MANY_WORMS)
def test_many_worm_cases_exceed_one_warp(kw):
    """The last four geometries really hold more than 32 worms per domain
    (so the block-wide passes are the ones compared above)."""
    g = P.Sim(**kw)
    g.sweep(4)
    r = g.rows()
    nd = (kw["Lx"] // (kw.get("dom_x") or kw["Lx"])) * (kw["Ly"] // (kw.get("dom_y") or kw["Ly"]))
    assert r["n_w"][1:].min() / nd > 32, r["n_w"]


def test_too_small_leg_hint_is_a_capacity_error():
    """A leg-count hint far below the real count makes the sweep return
    PMWA_ECAPACITY (checked in the kernel, no device fault); the sweeps
    queued behind the failed one leave at once, the handle refuses further
    sweeps until a configuration is imported, and the device stays
    usable."""
    kw = dict(Lx=16, Ly=16, beta=4.0, eta=0.1, dom_x=16, dom_y=16, sub_block=2, n_cycle=4, seed=3, legs_hint=1)
    g = P.Sim(**kw)
    with pytest.raises(P.PmwaError) as e:
        g.sweep(6)
    assert e.value.status == P.PMWA_ECAPACITY
    # the configuration is now undefined: the handle refuses to go on ...
    with pytest.raises(P.PmwaError) as e:
        g.sweep(1)
    assert e.value.status == P.PMWA_EINVARIANT
    assert g.check() == (-1, 0)
    # ... until a configuration is imported
    ok = P.Sim(**dict(kw, legs_hint=0))
    ok.sweep(2)
    g.import_(ok.export())
    assert np.array_equal(g.export(), ok.export())
    assert g.check() is None


@pytest.mark.parametrize("legs_hint", [0, 18])
def test_full_size_256x256_bit_exact(legs_hint):
    """The 256x256, beta t = 4, eta = 0.1 workload at full size in the launch
    configuration the benchmark times (16x16-site domains, 2x2 sub-blocks,
    boundary step every 2 sweeps, N_cycle 31; with the a-priori leg table
    and with a leg-count hint): 12 sweeps from the seeded half-filled start
    on both sides, configuration and counters equal bit for bit after every
    third sweep."""
    kw = dict(Lx=256, Ly=256, beta=4.0, t=1.0, V=0.0, mu=0.0, eta=0.1, dom_x=16, dom_y=16, sub_block=2,
              exchange_every=2, n_cycle=31, init=1, init_seed=7, seed=7, legs_hint=legs_hint)
    g, o = _pair(kw)
    for _ in range(4):
        g.sweep(3)
        o.sweep(3)
        _same(g.export(), o.export(), "configuration")
        a, b = g.rows(), o.rows()
        for f in ("sweep", "n_v", "n_k", "n_w", "occ_lo", "occ_hi"):
            assert np.array_equal(a[f], b[f]), f
        assert np.allclose(a["q_impr"], b["q_impr"], rtol=REL, atol=0)


# Known-answer vectors of Philox4x32-10 published with Random123 (Salmon et
# al., SC'11): counter words, key words, output words.
PHILOX_KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff,) * 4, (0xffffffff,) * 2, (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


def test_device_philox_known_answers():
    """The device generator that every kernel draws from reproduces the
    published known-answer vectors, and agrees with the oracle's on a sweep
    of counters and keys."""
    g = P.Sim(Lx=32, Ly=32, beta=1.0, eta=0.2)  # its idle slots hold the blocks
    got = P.pmwa_philox_blocks(g.h, [list(c) + list(k) for c, k, _ in PHILOX_KAT])
    for row, (_, _, want) in zip(got, PHILOX_KAT):
        assert [int(x) for x in row] == list(want)
    rng = np.random.default_rng(5)
    ck = rng.integers(0, 2 ** 32, size=(512, 6), dtype=np.uint64).astype(np.uint32)
    dev = P.pmwa_philox_blocks(g.h, ck)
    for j in range(len(ck)):
        assert np.array_equal(dev[j], O.philox(ck[j, :4], ck[j, 4:])), j


def test_config4_shape_in_small_bit_exact():
    """The 2048x2048, beta t = 16 workload in small: 32x32 sites in 2x2
    domains of 16x16 sites, Step 2 every 2 sweeps, 2x2 sub-blocks, eta = 0.1.
    After the chain warms up, every domain holds more worms than the CTA has
    threads (about 400 per domain), so Step 5 groups the worms with warp 0's
    walk instead of the block-wide passes.  Bit-exact after each of 36
    sweeps."""
    kw = dict(Lx=32, Ly=32, beta=16.0, eta=0.1, dom_x=16, dom_y=16, sub_block=2, n_cycle=20,
              exchange_every=2, seed=13, init=1, init_seed=11)
    g, o = _pair(kw)
    for s in range(36):
        o.sweep(1)
        g.sweep(1)
        _same(g.export(), o.export(), "after sweep %d" % s)
    ro, rg = o.rows(), g.rows()
    for f in ROW_FIELDS:
        assert np.array_equal(ro[f], rg[f]), f
    assert np.allclose(rg["q_impr"], ro["q_impr"], rtol=REL, atol=0)
    assert ro["w_dom_min"][-10:].min() > 256  # the many-worm grouping did run


def test_full_size_thermalised_bit_exact():
    """The 256x256, beta t = 4 workload in the launch configuration of the
    benchmark (16x16-site domains, K = 2, 2x2 sub-blocks, N_cycle = 43, a leg
    hint of 18 per site) from a thermalised configuration: the oracle
    thermalises the same parameters on 64x64 for 120 sweeps (about 17 vertex
    legs per site, the benchmark's density), the configuration is repeated
    4 x 4 times, and two sweeps from it must be bit-exact."""
    small = dict(Lx=64, Ly=64, beta=4.0, eta=0.1, dom_x=16, dom_y=16, sub_block=2, n_cycle=43,
                 exchange_every=2, seed=7, init=1, init_seed=7)
    o = O.Oracle(**small)
    o.sweep(120)
    r = o.rows()
    assert 2.0 * r["n_v"][-20:].mean() / (64 * 64) > 15.0  # thermalised leg density
    big = O.tile_config(o.export(), 64, 4)
    kw = dict(small, Lx=256, Ly=256, seed=9)
    ob = O.Oracle(**kw)
    ob.import_(big)
    ob.sweep_index = 120
    assert ob.check() == 0
    g = P.Sim(legs_hint=18, **kw)
    g.import_(big)
    g.sweep_index = 120
    for s in range(2):
        ob.sweep(1)
        g.sweep(1)
        _same(g.export(), ob.export(), "after sweep %d" % s)
    ro, rg = ob.rows(), g.rows()
    for f in ROW_FIELDS:
        assert np.array_equal(ro[f], rg[f]), f
    assert np.allclose(rg["q_impr"], ro["q_impr"], rtol=REL, atol=0)
    assert 2.0 * ro["n_v"].mean() / (256 * 256) > 15.0
