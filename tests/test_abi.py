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


def _oracle_rows(**kw):
    o = O.Oracle(**kw)
    o.sweep(96)
    return o.rows()


@pytest.mark.parametrize("kw", [dict(Lx=4, Ly=4, beta=2.0, eta=0.2, n_cycle=6, seed=3),
                                dict(Lx=8, Ly=4, beta=1.0, eta=0.3, V=1.0, mu=0.6, t=0.7, dom_x=4,
                                     dom_y=2, n_cycle=4, seed=5),
                                dict(Lx=4, Ly=4, beta=1.0, eta=0.4, t=0.0, mu=0.5, n_cycle=3, seed=8),
                                dict(Lx=8, Ly=8, beta=2.0, eta=0.2, V=1.0, mu=0.4, dom_x=4, dom_y=4,
                                     dom_tau=3, n_cycle=5, seed=11)])
def test_step6_observables_follow_their_definitions(kw):
    """pmwa_row_observables / pmwa_observables (host code of the library)
    against the Step-6 definitions restated here from the model (Eq. 5 per
    bond, C = max E + c_off) and a plain binning, on rows of the oracle."""
    rows = _oracle_rows(**kw)
    p = P.make_params(**kw)
    N = kw["Lx"] * kw["Ly"]
    t, V, mu, beta, eta = kw.get("t", 1.0), kw.get("V", 0.0), kw.get("mu", 0.0), kw["beta"], kw["eta"]
    Es = [V * (s & 1) * (s >> 1) - mu / 4.0 * ((s & 1) + (s >> 1)) for s in range(4)]
    C = max(Es) + t / 2.0
    nv = rows["n_v"].astype(float)
    occ = rows["occ_lo"].astype(float) + rows["occ_hi"].astype(float) * 2.0 ** 64
    Q = rows["q_impr"] / (beta * eta * N)
    want = dict(E=(2 * N * C - nv / beta) / N, n=occ / 2.0 ** 62 / N,
                Q_raw=rows["n_w"].astype(float) / (beta * eta * N), Q_impr=Q)
    want["E_eta"] = want["E"] - eta * Q
    if t > 0:
        want["kin"] = rows["n_k"].astype(float) / (beta * t * 2 * N)
    got = P.observables(rows, p)
    assert set(got) == set(want)
    for k in want:
        assert np.allclose(got[k], want[k], rtol=1e-13, atol=1e-13), k
    s = P.summary(rows, p, bins=8)
    m = len(rows) // 8
    for k in want:
        b = want[k][: 8 * m].reshape(8, m).mean(axis=1)
        assert s[k] == pytest.approx(b.mean(), rel=1e-12, abs=1e-13), k
        assert s[k + "_err"] == pytest.approx(b.std(ddof=1) / np.sqrt(8), rel=1e-9, abs=1e-15), k
    nd = (kw["Lx"] // kw.get("dom_x", kw["Lx"])) * (kw["Ly"] // kw.get("dom_y", kw["Ly"])) * kw.get("dom_tau", 1)
    used = rows[: 8 * m]
    assert s["w_dom_mean"] == pytest.approx(used["n_w"].mean() / nd, rel=1e-12)
    assert s["w_dom_min"] == used["w_dom_min"].min()
    assert s["dom_empty_frac"] == pytest.approx(used["dom_empty"].sum() / (len(used) * nd), rel=1e-12, abs=0)
    if nd == 1:  # one domain: its worms are all worms
        assert np.array_equal(rows["w_dom_min"], rows["n_w"])
        assert np.array_equal(rows["dom_empty"], (rows["n_w"] == 0).astype(np.uint32))
    with pytest.raises(P.PmwaError):
        P.summary(rows[:1], p, bins=2)


def test_n_cycle_rule():
    """N_cycle = ceil(2 <n_v> / <n_w>) over the given rows, at least 1 and at
    most 512; the a-priori form from <n_v> = N_b beta (d_mean + t/2) and
    <n_w> = beta eta N / 2."""
    kw = dict(Lx=8, Ly=8, beta=2.0, eta=0.2, n_cycle=6, seed=1)
    rows = _oracle_rows(**kw)
    p = P.make_params(**kw)
    half = rows[len(rows) // 2:]
    want = int(np.ceil(2.0 * half["n_v"].mean() / max(half["n_w"].mean(), 1.0)))
    assert P.n_cycle(p, half) == max(1, min(512, want))
    # a priori at V = mu = 0, t = 1: d(s) = t/2 for every s, so
    # N_cycle = ceil(2 * 2N beta (1/2 + 1/2) / (beta eta N / 2)) = ceil(8 / eta)
    assert P.n_cycle(p) == int(np.ceil(8.0 / 0.2))
    assert P.n_cycle(P.make_params(**dict(kw, eta=0.001))) == 512


def test_vertex_window_parameter():
    """vertex_window in [0, 1] (the on-the-fly vertex phase); replica batches
    refuse it (their kernels run the plain vertex phase)."""
    kw = dict(Lx=8, Ly=8, beta=2.0, eta=0.2)
    assert P.pmwa_footprint(P.make_params(vertex_window=0.1, **kw)) > 0
    for bad in (-0.1, 1.5, float("nan")):
        assert P.pmwa_footprint(P.make_params(vertex_window=bad, **kw)) == 0
    import ctypes as C
    from paper_1307_0328_gb300._lib import Params
    arr = (Params * 1)(P.make_params(vertex_window=0.1, **kw))
    assert P.load().pmwa_batch_footprint(arr, 1) == 0
    arr = (Params * 1)(P.make_params(**kw))
    assert P.load().pmwa_batch_footprint(arr, 1) > 0
