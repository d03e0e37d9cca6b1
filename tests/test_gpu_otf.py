"""GPU parity of the on-the-fly vertex generation (the paper's closing
discussion of extensions; the oracle's form is pinned against exact
diagonalisation): with vertex_window = w the vertex phase of a bond erases
and places diagonal vertices only within w beta of a worm of the current
configuration on either of its sites, in the tile kernel and in the
boundary kernel's Step 3.  Bit for bit against the oracle after every step
and every sweep, with one domain and several, with temporal domains, and a
window so small that the vertex phase leaves the configuration unchanged."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402

import paper_1307_0328_gb300 as P  # noqa: E402

ROW_FIELDS = ("sweep", "n_v", "n_k", "n_w", "occ_lo", "occ_hi", "w_dom_min", "dom_empty")

GEOMS = [
    dict(Lx=8, Ly=8, beta=2.0, eta=0.2, n_cycle=6, seed=1, init=1, init_seed=1, vertex_window=0.1),
    dict(Lx=8, Ly=8, beta=2.0, eta=0.3, V=1.0, mu=0.7, dom_x=4, dom_y=4, sub_block=2, n_cycle=5,
         exchange_every=1, seed=5, vertex_window=0.05),
    dict(Lx=16, Ly=16, beta=4.0, eta=0.1, dom_x=8, dom_y=8, sub_block=4, n_cycle=8, exchange_every=2,
         seed=7, init=1, init_seed=7, vertex_window=0.2, dom_tau=2),
    dict(Lx=32, Ly=32, beta=4.0, eta=0.25, dom_x=16, dom_y=16, sub_block=2, n_cycle=8, exchange_every=2,
         seed=19, init=1, init_seed=9, vertex_window=0.02),
    dict(Lx=6, Ly=6, beta=4.0, eta=0.1, n_cycle=6, seed=13, vertex_window=0.6),
]


def _same(a, b, what):
    if not np.array_equal(a, b):
        n = min(len(a), len(b))
        diff = np.nonzero(a[:n] != b[:n])[0]
        first = int(diff[0]) if len(diff) else n
        raise AssertionError("%s: %d vs %d words, first difference at word %d" % (what, len(a), len(b), first))


@pytest.mark.parametrize("kw", GEOMS)
def test_vertex_window_steps_and_sweeps_bit_exact(kw):
    g, o = P.Sim(**kw), O.Oracle(**kw)
    multi = "dom_x" in kw
    for s in range(4):
        snap = o.export()
        g.import_(snap)
        g.sweep_index = s
        o.sweep_index = s
        if kw.get("dom_tau", 1) > 1:
            o.temporal()
            g.temporal()
        if multi:
            o.boundary()
            g.boundary()
            _same(g.export(), o.export(), "Step 2 at sweep %d" % s)
        snap = o.export()
        for stop in (3, 6):
            o.import_(snap)
            o.sweep_index = s
            g.import_(snap)
            g.sweep_index = s
            o.tile(stop)
            g.tile(stop)
            _same(g.export(), o.export(), "Steps 3..%d at sweep %d" % (stop, s))
        g.rows()
        o.rows()
    g2, o2 = P.Sim(**kw), O.Oracle(**kw)
    for s in range(10):
        o2.sweep(1)
        g2.sweep(1)
        _same(g2.export(), o2.export(), "after sweep %d" % s)
    ro, rg = o2.rows(), g2.rows()
    for f in ROW_FIELDS:
        assert np.array_equal(ro[f], rg[f]), f
    assert np.allclose(rg["q_impr"], ro["q_impr"], rtol=1e-12, atol=0)


def test_a_vanishing_window_leaves_the_vertex_phase_idle():
    kw = dict(Lx=8, Ly=8, beta=4.0, eta=0.1, n_cycle=6, seed=13)
    base = P.Sim(**kw)
    base.sweep(20)
    snap, s0 = base.export(), base.sweep_index
    g = P.Sim(vertex_window=1e-12, **kw)
    g.import_(snap)
    g.sweep_index = s0
    g.tile(3)
    assert np.array_equal(g.export(), snap)
