"""Pins of the oracle's temporal domains (Supplement S-II: the space-time cut
into N_beta slabs along imaginary time; Step 1 of the pseudo code and Eq. 3).

- Step 1's law against the paper's hard-core closed form
  P(s') = (1 + tanh^S(s1')(I1 eta) tanh^S(s2')(I2 eta))^-1 and against the
  semigroup identity sum_s' f_qs'(I1) f_s'p(I2) = f_qp(I1 + I2) of
  f_ab(I) = <a| e^{I eta Q} |b>, both evaluated here with numpy's cosh, sinh
  and tanh (not the oracle's arithmetic).
- The structure the method relies on: the worldline state at a temporal
  boundary changes only in Step 1 (Steps 2-5 stop at the boundaries), every
  invariant holds after every step, and with N_beta = 1 nothing changes.
- The whole chain with N_beta = 2, 3 and 4 against exact diagonalisation
  within 4 standard errors, alone and with spatial domains and sub-blocks,
  and the decoupled-site closed form at t = V = 0 on 8x8.
"""
import numpy as np
import pytest

from oracle import ed
from oracle import oracle as O

TWO59 = 2.0 ** 59


def f_ab(a, b, x):
    return np.cosh(x) if a == b else np.sinh(x)


@pytest.mark.parametrize("p,q", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_step1_law_closed_form_and_semigroup(p, q):
    rng = np.random.default_rng(17 + 2 * p + q)
    XW = 2.0 * 0.3 / TWO59  # beta eta = 0.6
    cases = [(int(m1), int(m2)) for m1, m2 in rng.integers(1, 2 ** 59, size=(60, 2))]
    cases += [(1, 2 ** 58), (2 ** 58, 1), (3, 5), (2 ** 59 - 7, 2 ** 40)]
    for M1, M2 in cases:
        P = O.pdom(p, q, M1, M2, XW)
        x1, x2 = M1 * XW, M2 * XW
        assert P.sum() == pytest.approx(1.0, rel=1e-14)
        for sn in (0, 1):
            s1, s2 = q ^ sn, sn ^ p
            S = lambda s: 1.0 if s == 0 else -1.0  # noqa: E731
            closed = 1.0 / (1.0 + np.tanh(x1) ** S(s1) * np.tanh(x2) ** S(s2))
            assert P[sn] == pytest.approx(closed, rel=1e-9, abs=1e-15), (M1, M2, sn)
            # normalised by f_qp(I1 + I2): the semigroup identity of e^{I eta Q}
            want = f_ab(q, sn, x1) * f_ab(sn, p, x2) / f_ab(q, p, x1 + x2)
            assert P[sn] == pytest.approx(want, rel=1e-9, abs=1e-15), (M1, M2, sn)


def test_step1_law_empty_piece():
    """A piece of zero length admits no worm: its end states must agree."""
    XW = 1.0 / TWO59
    assert np.array_equal(O.pdom(0, 1, 0, 1000, XW), [0.0, 1.0])   # I1 = 0: s' = q = 1
    assert np.array_equal(O.pdom(0, 1, 1000, 0, XW), [1.0, 0.0])   # I2 = 0: s' = p = 0
    assert np.array_equal(O.pdom(1, 0, 1000, 0, XW), [0.0, 1.0])   # I2 = 0: s' = p = 1


def _boundary_states(buf, N, NB):
    """State of the worldline just below each temporal boundary of each site
    (the boundaries at m_k = floor(k 2^59 / N_beta), tag 6), from an export."""
    bpk = [((k << 59) // NB << 3) | 6 for k in range(NB)]
    out = np.zeros((N, NB), dtype=np.int64)
    k = 1
    for s in range(N):
        hd = int(buf[k])
        n = hd & 0x7fffffff
        keys = [int(x) for x in buf[k + 1:k + 1 + n]]
        k += 1 + n
        for j, b in enumerate(bpk):
            below = [x for x in keys if (x >> 2) < b]
            if below:
                out[s, j] = below[-1] & 1
            elif keys:
                out[s, j] = keys[-1] & 1
            else:
                out[s, j] = hd >> 63
    return out


GEOS = [
    dict(Lx=4, Ly=4, beta=2.0, eta=0.3, dom_tau=2, n_cycle=6, seed=3),
    dict(Lx=4, Ly=4, beta=2.0, eta=0.3, V=1.0, mu=0.4, dom_tau=3, dom_x=2, dom_y=2, n_cycle=6, seed=4,
         exchange_every=1),
    dict(Lx=8, Ly=8, beta=4.0, eta=0.2, dom_tau=4, dom_x=4, dom_y=4, sub_block=2, n_cycle=6, seed=5),
    dict(Lx=2, Ly=2, beta=1.0, eta=0.5, dom_tau=5, n_cycle=4, seed=6, init=0),
]


@pytest.mark.parametrize("kw", GEOS)
def test_boundary_states_change_only_in_step1(kw):
    o = O.Oracle(**kw)
    N, NB = kw["Lx"] * kw["Ly"], kw["dom_tau"]
    multi = "dom_x" in kw
    changed = 0
    for s in range(25):
        o.sweep_index = s
        before = _boundary_states(o.export(), N, NB)
        o.temporal()
        assert o.check() == 0
        after = _boundary_states(o.export(), N, NB)
        changed += int((before != after).sum())
        if multi:
            o.boundary()
            assert o.check() == 0
            assert np.array_equal(_boundary_states(o.export(), N, NB), after), "Step 2 moved a boundary state"
        snap = o.export()
        for stop in (3, 4, 5, 6):
            o.import_(snap)
            o.sweep_index = s
            o.tile(stop)
            assert o.check() == 0
            assert np.array_equal(_boundary_states(o.export(), N, NB), after), "Steps 3..%d" % stop
        o.rows()
    assert changed > 0  # Step 1 does resample them


def test_one_temporal_domain_is_the_plain_chain():
    """dom_tau = 1 (or 0, as in the library's parameters) has no boundary:
    the run is the same as without the field."""
    kw = dict(Lx=6, Ly=6, beta=2.0, eta=0.2, dom_x=3, dom_y=3, sub_block=0, n_cycle=5, seed=9)
    a, b, c = O.Oracle(**kw), O.Oracle(dom_tau=1, **kw), O.Oracle(dom_tau=0, **kw)
    for o in (a, b, c):
        o.sweep(20)
    assert np.array_equal(a.export(), b.export())
    assert np.array_equal(a.export(), c.export())
    with pytest.raises(ValueError):
        O.Oracle(dom_tau=-1, **kw)
    with pytest.raises(ValueError):
        O.Oracle(dom_tau=65, **kw)


def _replicas(Lx, Ly, R, sweeps, therm, seed0, **kw):
    out = {}
    for r in range(R):
        o = O.Oracle(Lx=Lx, Ly=Ly, seed=seed0 + r, **kw)
        o.sweep(therm)
        o.rows()
        o.sweep(sweeps)
        assert o.check() == 0
        for k, v in O.observables(o.rows(), o.params).items():
            out.setdefault(k, []).append(v.mean())
    return {k: np.array(v) for k, v in out.items()}


CASES = [
    (2, 2, dict(beta=2.0, eta=0.2), dict(dom_tau=2), 100_000),
    (3, 3, dict(beta=2.0, eta=0.3, V=1.0, mu=0.6), dict(dom_tau=3), 72_000),
    (4, 2, dict(beta=2.0, eta=0.3, mu=-0.5), dict(dom_tau=2, dom_x=2, dom_y=2, sub_block=2), 72_000),
    (3, 3, dict(beta=4.0, eta=0.3, V=0.5), dict(dom_tau=4, exchange_every=2), 48_000),
]


@pytest.mark.parametrize("Lx,Ly,model,geo,sweeps", CASES)
def test_temporal_domains_chain_matches_ed(Lx, Ly, model, geo, sweeps):
    m = dict(t=1.0, V=0.0, mu=0.0)
    m.update(model)
    ex = ed.thermal(Lx, Ly, m["beta"], m["t"], m["V"], m["mu"], m["eta"], slices_r=False)
    ob = _replicas(Lx, Ly, 24, sweeps // 24, 500, 31, n_cycle=8, **m, **geo)
    want = dict(E=ex["E"], n=ex["n"], Q_raw=ex["Q"], Q_impr=ex["Q"], kin=ex["kin"])
    msgs = []
    for k, w in want.items():
        v = ob[k]
        mean, err = float(v.mean()), float(v.std(ddof=1) / np.sqrt(len(v)))
        z = (mean - w) / err
        msgs.append("%s %.5f+-%.5f ed %.5f z=%.2f" % (k, mean, err, w, z))
        assert abs(z) < 4.0, "; ".join(msgs)


def test_temporal_domains_decoupled_sites():
    """t = V = 0 with N_beta = 4 and spatial domains: each site is the
    two-level problem -mu n - eta (b + b+), exact at any L."""
    beta, mu, eta = 2.0, 1.0, 0.4
    ob = _replicas(8, 8, 16, 300, 100, 5, beta=beta, t=0.0, V=0.0, mu=mu, eta=eta, c_off=0.5, n_cycle=4,
                   dom_tau=4, dom_x=4, dom_y=4, sub_block=2)
    cf = ed.single_site(beta, mu, eta)
    for k, want in [("n", cf["n"]), ("Q_raw", cf["Q"]), ("Q_impr", cf["Q"]), ("E", cf["E"])]:
        v = ob[k]
        mean, err = float(v.mean()), float(v.std(ddof=1) / np.sqrt(len(v)))
        assert abs(mean - want) < 4.0 * err, (k, mean, err, want)


# ---- on-the-fly vertex generation (the paper's closing discussion of
# extensions): the vertex phase confined to windows around the worms

OTF = [
    (2, 2, dict(beta=2.0, eta=0.3), dict(vertex_window=0.1), 96_000),
    (3, 3, dict(beta=2.0, eta=0.3, V=1.0, mu=0.6), dict(vertex_window=0.05), 72_000),
    (4, 2, dict(beta=2.0, eta=0.3, mu=-0.5), dict(vertex_window=0.2, dom_x=2, dom_y=2, sub_block=2), 72_000),
    (3, 3, dict(beta=2.0, eta=0.3), dict(vertex_window=0.1, dom_tau=2), 72_000),
]


@pytest.mark.parametrize("Lx,Ly,model,geo,sweeps", OTF)
def test_on_the_fly_vertex_phase_matches_ed(Lx, Ly, model, geo, sweeps):
    m = dict(t=1.0, V=0.0, mu=0.0)
    m.update(model)
    ex = ed.thermal(Lx, Ly, m["beta"], m["t"], m["V"], m["mu"], m["eta"], slices_r=False)
    ob = _replicas(Lx, Ly, 24, sweeps // 24, 500, 61, n_cycle=8, **m, **geo)
    want = dict(E=ex["E"], n=ex["n"], Q_raw=ex["Q"], Q_impr=ex["Q"], kin=ex["kin"])
    msgs = []
    for k, w in want.items():
        v = ob[k]
        mean, err = float(v.mean()), float(v.std(ddof=1) / np.sqrt(len(v)))
        z = (mean - w) / err
        msgs.append("%s %.5f+-%.5f ed %.5f z=%.2f" % (k, mean, err, w, z))
        assert abs(z) < 4.0, "; ".join(msgs)


def test_on_the_fly_vertex_phase_keeps_far_vertices():
    """Outside the window nothing is redrawn: with a window of 1e-12 beta
    (a few hundred grid points of 2^59) the vertex phase leaves the
    configuration as it was, while a window of 0.02 beta changes it but not
    as much as the global vertex phase."""
    kw = dict(Lx=6, Ly=6, beta=4.0, eta=0.1, n_cycle=6, seed=13)
    base = O.Oracle(**kw)
    base.sweep(30)
    snap, s0 = base.export(), base.sweep_index
    outs = {}
    for w in (0.0, 1e-12, 0.02):
        o = O.Oracle(vertex_window=w, **kw)
        o.import_(snap)
        o.sweep_index = s0
        o.tile(3)
        assert o.check() == 0
        outs[w] = o.export()
    assert np.array_equal(outs[1e-12], snap)
    same = lambda x: np.isin(x[1:], snap[1:]).mean()  # noqa: E731
    assert same(outs[0.0]) < same(outs[0.02]) < 1.0
    with pytest.raises(ValueError):
        O.Oracle(vertex_window=-0.1, **kw)
