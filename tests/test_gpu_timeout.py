"""The PMWA_ETIMEOUT path of the bounded device loops, exercised without a
fault: the handle's loop caps (pmwa_set_loop_caps) are lowered so that the
ziggurat or the Eq. 1 worm-number sampler runs out of words or proposals in
an ordinary sweep.  The sweep must return PMWA_ETIMEOUT, every later call
that reads the configuration must return PMWA_EINVARIANT (the configuration
is undefined), and pmwa_import must restore the handle, after which the
chain continues bit for bit like the oracle's."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_1307_0328_gb300 as P  # noqa: E402
from oracle import oracle as O  # noqa: E402

KW = dict(Lx=8, Ly=8, beta=2.0, eta=0.3, V=0.5, mu=0.4, dom_x=4, dom_y=4, sub_block=2, n_cycle=5,
          exchange_every=1, seed=31, init=1, init_seed=2)


@pytest.mark.parametrize("caps", [(1, 128), (64, 1)], ids=["ziggurat_words", "sampler_proposals"])
def test_loop_cap_timeout_then_import_recovers(caps):
    g = P.Sim(**KW)
    g.sweep(3)
    g.rows()
    snap, s0 = g.export(), g.sweep_index
    P.pmwa_set_loop_caps(g.h, *caps)
    with pytest.raises(P.PmwaError) as e:
        g.sweep(4)
    assert e.value.status == P.PMWA_ETIMEOUT
    P.pmwa_set_loop_caps(g.h)  # the specification's caps again
    for call in (lambda: g.sweep(1), g.export, lambda: g.rho_slices(4)):
        with pytest.raises(P.PmwaError) as e:
            call()
        assert e.value.status == P.PMWA_EINVARIANT
    assert g.check()[0] == -1
    # out-of-range caps are refused
    for bad in [(0, 128), (65, 128), (64, 0), (64, 129)]:
        with pytest.raises(P.PmwaError) as e:
            P.pmwa_set_loop_caps(g.h, *bad)
        assert e.value.status == P.PMWA_EINVAL
    g.import_(snap)
    g.sweep_index = s0
    g.rows()
    o = O.Oracle(**KW)
    o.import_(snap)
    o.sweep_index = s0
    g.sweep(3)
    o.sweep(3)
    assert np.array_equal(g.export(), o.export())
    assert g.check() is None
