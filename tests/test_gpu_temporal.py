"""GPU parity of the temporal domains (Supplement S-II; Step 1 and Eq. 3):
the CUDA path through the C ABI against the CPU oracle on the same inputs,
bit for bit in configuration and integer counters, FP64 estimators within
1e-12 relative.

Each step is checked on its own from the same configuration (Step 1; Step 2
+ boundary Step 3; Steps 3, 3-4, 3-5, 3-6), then whole sweeps.  The cases
cover one spatial domain and several, sub-blocks, N_beta from 2 to 5,
t = 0, an empty 2x2 start, and beta t = 16 with several hundred worms per
domain (both Step-5 groupings).  At full size the t = V = 0 closed form must
hold with N_beta = 4 on 256x256.  Replica batches run Step 1 too.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import ed  # noqa: E402
from oracle import oracle as O  # noqa: E402

import paper_1307_0328_gb300 as P  # noqa: E402

REL = 1e-12
ROW_FIELDS = ("sweep", "n_v", "n_k", "n_w", "occ_lo", "occ_hi", "w_dom_min", "dom_empty")

GEOMS = [
    dict(Lx=8, Ly=8, beta=2.0, eta=0.2, n_cycle=6, seed=1, init=1, init_seed=1, dom_tau=2),
    dict(Lx=8, Ly=8, beta=2.0, eta=0.3, V=1.0, mu=0.7, dom_x=4, dom_y=4, sub_block=2, n_cycle=5,
         exchange_every=1, seed=5, dom_tau=3),
    dict(Lx=16, Ly=16, beta=4.0, eta=0.1, dom_x=8, dom_y=8, sub_block=4, n_cycle=8, exchange_every=2,
         seed=7, init=1, init_seed=7, dom_tau=4),
    dict(Lx=2, Ly=2, beta=1.5, eta=0.5, n_cycle=4, seed=3, init=0, dom_tau=5),
    dict(Lx=6, Ly=9, beta=4.0, eta=0.15, t=0.0, c_off=0.3, mu=0.8, dom_x=3, dom_y=3, n_cycle=3, seed=11,
         dom_tau=3),
    dict(Lx=16, Ly=16, beta=4.0, eta=0.3, sub_block=2, n_cycle=6, seed=17, init=1, init_seed=5, dom_tau=2),
    dict(Lx=32, Ly=32, beta=16.0, eta=0.1, dom_x=16, dom_y=16, sub_block=2, n_cycle=8, exchange_every=2,
         seed=19, init=1, init_seed=9, dom_tau=2),
]


def _pair(kw):
    return P.Sim(**kw), O.Oracle(**kw)


def _same(a, b, what):
    if not np.array_equal(a, b):
        n = min(len(a), len(b))
        diff = np.nonzero(a[:n] != b[:n])[0]
        first = int(diff[0]) if len(diff) else n
        raise AssertionError("%s: %d vs %d words, first difference at word %d" % (what, len(a), len(b), first))


def _rows_same(rg, ro):
    for f in ROW_FIELDS:
        assert np.array_equal(ro[f], rg[f]), f
    assert np.allclose(rg["q_impr"], ro["q_impr"], rtol=REL, atol=0)


@pytest.mark.parametrize("kw", GEOMS)
def test_temporal_steps_bit_exact(kw):
    g, o = _pair(kw)
    nd = (kw["Lx"] // (kw.get("dom_x") or kw["Lx"])) * (kw["Ly"] // (kw.get("dom_y") or kw["Ly"]))
    for s in range(6):
        snap = o.export()
        g.import_(snap)
        g.sweep_index = s
        o.sweep_index = s
        o.temporal()
        g.temporal()
        _same(g.export(), o.export(), "Step 1 at sweep %d" % s)
        if nd > 1:
            o.boundary()
            g.boundary()
            _same(g.export(), o.export(), "Step 2 at sweep %d" % s)
        snap = o.export()
        for stop in (3, 4, 5, 6):
            o.import_(snap)
            o.sweep_index = s
            g.import_(snap)
            g.sweep_index = s
            o.tile(stop)
            g.tile(stop)
            _same(g.export(), o.export(), "Steps 3..%d at sweep %d" % (stop, s))
        _rows_same(g.rows(), o.rows())
        assert g.check() is None


@pytest.mark.parametrize("kw", GEOMS)
def test_temporal_sweeps_bit_exact(kw):
    g, o = _pair(kw)
    for s in range(12):
        o.sweep(1)
        g.sweep(1)
        _same(g.export(), o.export(), "after sweep %d" % s)
    _rows_same(g.rows(), o.rows())


def test_temporal_many_worms_take_the_warp_walk():
    """beta t = 16 in 16x16 domains with N_beta = 2: after warming up the
    domains hold more worms than the CTA has threads; still bit-exact."""
    kw = dict(GEOMS[-1])
    g, o = _pair(kw)
    for s in range(30):
        o.sweep(1)
        g.sweep(1)
    _same(g.export(), o.export(), "after 30 sweeps")
    ro, rg = o.rows(), g.rows()
    _rows_same(rg, ro)
    assert ro["n_w"][-5:].min() / 4 > 256  # per spatial domain, both slabs


def test_temporal_decoupled_sites_full_size():
    """t = V = 0, N_beta = 4, 256x256 in 16x16-site domains: every site is
    the two-level problem -mu n - eta (b + b+); density and <Q>/N follow the
    closed form within 4 standard errors over 400 sweeps."""
    beta, mu, eta = 4.0, 1.0, 0.3
    g = P.Sim(Lx=256, Ly=256, beta=beta, t=0.0, V=0.0, mu=mu, eta=eta, c_off=0.5, dom_x=16, dom_y=16,
              sub_block=2, n_cycle=4, seed=3, dom_tau=4)
    g.sweep(100)
    g.rows()
    g.sweep(400)
    s = P.summary(g.rows(), g.params, bins=20)
    cf = ed.single_site(beta, mu, eta)
    for k, want in (("n", cf["n"]), ("Q_impr", cf["Q"]), ("Q_raw", cf["Q"])):
        assert abs(s[k] - want) < 4.0 * s[k + "_err"] + 1e-12, (k, s[k], s[k + "_err"], want)
    assert g.check() is None


@pytest.mark.parametrize("graph", [0, 2])
def test_temporal_batch_equals_alone_and_oracle(graph):
    """A replica batch mixing instances with and without temporal domains
    (Step 1 runs batched, one warp per site, only where it is due) gives each
    instance exactly its bytes swept alone, and the oracle's."""
    kws = [GEOMS[0], GEOMS[1], GEOMS[3], dict(Lx=8, Ly=8, beta=2.0, eta=0.2, n_cycle=5, seed=77, replica=9),
           dict(GEOMS[2], exchange_every=3, replica=4)]
    batch = P.Batch(kws)
    if graph:
        batch.graph(graph)
    batch.sweep(6)
    for i, kw in enumerate(kws):
        alone = P.Sim(**kw)
        alone.sweep(6)
        assert np.array_equal(batch.export(i), alone.export()), i
        _rows_same(batch.rows(i), alone.rows())
        o = O.Oracle(**kw)
        o.sweep(6)
        assert np.array_equal(batch.export(i), o.export()), i
