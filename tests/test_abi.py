"""CPU checks of the C ABI: libpmwa.so builds for sm_103a, loads, exports
every function include/pmwa.h declares, validates parameters, and derives
its host tables (directed-loop thresholds of Eq. 2, vertex thinning, the
ziggurat) bit for bit like the independently written oracle."""
import os
import re

import numpy as np
import pytest

import paper_1307_0328_gb300 as P
from oracle import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "pmwa.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmwa_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = P.load()
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_and_param_validation():
    assert P.pmwa_strerror(0) == "ok"
    assert "capacity" in P.pmwa_strerror(P.PMWA_ECAPACITY)
    good = P.make_params(Lx=8, Ly=8)
    assert P.pmwa_footprint(good) > 0
    for bad in [dict(Lx=1), dict(beta=0.0), dict(eta=-1.0), dict(dom_x=3), dict(sub_block=3),
                dict(Lx=8, dom_x=1), dict(n_cycle=5000), dict(exchange_every=0)]:
        assert P.pmwa_footprint(P.make_params(**bad)) == 0, bad


@pytest.mark.parametrize("kw", [dict(), dict(V=1.0, mu=0.5), dict(V=3.0, mu=4.2),
                                dict(V=0.0, mu=-2.0, t=0.5, beta=16.0, eta=0.05),
                                dict(t=0.0, mu=1.0, c_off=0.3)])
def test_host_tables_equal_oracle_tables(kw):
    a = P.pmwa_tables(**kw)
    b = O.tables(**kw)
    assert np.array_equal(a["d"], b["d"])
    assert a["D"] == b["D"]
    assert np.array_equal(a["TV"], b["TV"])
    assert np.array_equal(a["TH"], b["TH"])
    assert a["SV"] == b["SV"] and a["SW"] == b["SW"]
    z = O.zig_tables()
    for k in "XFWK":
        assert np.array_equal(a[k], z[k]), k


def test_tile_plan_sizes_from_the_hint_and_keeps_occupancy():
    """A measured leg count (legs_hint) sizes the leg table of the 256x256,
    beta t = 4 domains (16x16 sites) below the a-priori bound 4 beta (D + t)
    and keeps two CTAs per SM; small domains with room to spare also stage
    their configuration in shared memory; a negative hint is rejected."""
    kw = dict(Lx=256, Ly=256, beta=4.0, eta=0.1, dom_x=16, dom_y=16, sub_block=2, n_cycle=31)
    hinted = P.pmwa_tile_plan(**kw, legs_hint=15)
    bound = P.pmwa_tile_plan(**kw)
    assert 15 * 256 < hinted["legcap"] < bound["legcap"]
    assert (228 * 1024) // (hinted["smem"] + 1024) >= 2
    small = P.pmwa_tile_plan(Lx=8, Ly=8, beta=2.0, eta=0.2, n_cycle=6, legs_hint=12)
    assert small["oldcap"] >= small["legcap"] > 12 * 64
    with pytest.raises(P.PmwaError):
        P.pmwa_tile_plan(**kw, legs_hint=-1)
