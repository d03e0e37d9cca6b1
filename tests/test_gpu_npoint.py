"""GPU parity of the equal-time n-point functions of listed site tuples
(pmwa_npoint) with the oracle on the same configurations, within 1e-12
(both take the product in tuple order and the sum over slices in order from
the same densities, which agree to 1e-12).

Cases: n from 1 to the maximum 16; tuple counts that are not a multiple of
the 128-thread block; K from 1 to 16; a 2x2 lattice whose scratch holds
about a hundred tuples at a time, so that 1000 tuples run in chunks; and
the argument errors (a site twice, a site out of range, n out of range).
"""
import numpy as np
import pytest

from oracle import oracle as O

import paper_1307_0328_gb300 as P

pytestmark = pytest.mark.gpu

REL = 1e-12

GEOMS = [
    dict(Lx=8, Ly=8, beta=2.0, eta=0.2, n_cycle=6, seed=1, init=1, init_seed=1),
    dict(Lx=12, Ly=8, beta=3.0, eta=0.3, V=0.5, mu=0.2, dom_x=6, dom_y=4, sub_block=2, n_cycle=4, seed=31),
    dict(Lx=19, Ly=17, beta=2.0, eta=0.3, V=0.5, mu=0.4, n_cycle=6, seed=29, init=1, init_seed=4),
    dict(Lx=4, Ly=4, beta=0.25, t=0.0, c_off=0.1, eta=0.5, n_cycle=4, seed=5),
]


def _pair(kw, sweeps=6):
    g, o = P.Sim(**kw), O.Oracle(**kw)
    g.sweep(sweeps)
    o.sweep(sweeps)
    assert np.array_equal(g.export(), o.export())
    return g, o


def _tuples(rng, N, m, n):
    return np.array([rng.choice(N, size=n, replace=False) for _ in range(m)], dtype=np.int32)


@pytest.mark.parametrize("kw", GEOMS)
def test_npoint_matches_the_oracle(kw):
    g, o = _pair(kw)
    N = kw["Lx"] * kw["Ly"]
    rng = np.random.Generator(np.random.Philox(7))
    try:
        for K, n, m in ((1, 1, 5), (4, 2, 129), (7, 3, 300), (16, 4, 257), (5, min(16, N), 33)):
            t = _tuples(rng, N, m, n)
            a, b = g.npoint(K, t), o.npoint(K, t)
            scale = max(float(np.abs(b).max()), 1e-300)
            assert np.allclose(a, b, rtol=REL, atol=REL * scale), (K, n, m, float(np.abs(a - b).max()))
        assert g.npoint(4, np.zeros((0, 2), dtype=np.int32)).shape == (0,)
    finally:
        g.close()


def test_npoint_in_chunks():
    kw = dict(Lx=2, Ly=2, beta=1.5, eta=0.5, n_cycle=4, seed=3, init=0)
    g, o = _pair(kw, sweeps=8)
    rng = np.random.Generator(np.random.Philox(11))
    try:
        t = _tuples(rng, 4, 1000, 2)
        a, b = g.npoint(8, t), o.npoint(8, t)
        assert np.allclose(a, b, rtol=REL, atol=REL * float(np.abs(b).max()))
    finally:
        g.close()


def test_npoint_arguments():
    g = P.Sim(Lx=8, Ly=8, beta=1.0, eta=0.3, n_cycle=4, seed=2)
    try:
        for K, t in ((4, [[0, 0]]), (4, [[0, 64]]), (4, [[-1, 2]]), (0, [[0, 1]]), (4, np.arange(17)[None, :])):
            with pytest.raises(P.PmwaError) as e:
                g.npoint(K, np.array(t, dtype=np.int32))
            assert e.value.status == P.PMWA_EINVAL, (K, t)
    finally:
        g.close()


# ---- resolved by the component of Q at arbitrary times (pmwa_npoint_alpha)

def _alpha_tuples(rng, N, K, m, n, same_site):
    """m tuples of n points (site, slice, component); with same_site, every
    tuple puts its points on at most two sites, so that several share an
    interval (the multi-point interval form) or a circle without legs."""
    out = np.zeros((m, n, 3), dtype=np.int32)
    for j in range(m):
        sites = rng.choice(N, size=2, replace=False) if same_site else rng.choice(N, size=n, replace=N < n)
        seen = set()
        for c in range(n):
            while True:
                s = int(sites[rng.integers(0, len(sites))]) if same_site else int(sites[c])
                k = int(rng.integers(0, K))
                if (s, k) not in seen:
                    break
            seen.add((s, k))
            out[j, c] = (s, k, int(rng.integers(0, 2)))
    return out


@pytest.mark.parametrize("kw", GEOMS + [dict(Lx=8, Ly=8, beta=4.0, eta=0.2, dom_tau=3, n_cycle=6, seed=41)])
def test_npoint_alpha_matches_oracle(kw):
    g, o = _pair(kw)
    N = kw["Lx"] * kw["Ly"]
    rng = np.random.default_rng(N)
    for K, n, m, same in [(1, 1, 37, False), (8, 2, 130, True), (8, 3, 129, True), (12, 4, 70, True),
                          (16, 4, 65, False), (6, 5, 33, True), (8, 16, 9, False)]:
        if n > K * (2 if same else N):
            continue
        pts = _alpha_tuples(rng, N, K, m, n, same)
        got = g.npoint_alpha(K, pts)
        want = o.npoint_alpha(K, pts)
        assert np.allclose(got, want, rtol=REL, atol=1e-300), (K, n, same)


def test_npoint_alpha_argument_errors():
    g = P.Sim(Lx=4, Ly=4, beta=1.0, eta=0.3, n_cycle=4, seed=3)
    g.sweep(2)
    bad = [np.array([[[0, 1, 0], [0, 1, 1]]]),   # one (site, slice) twice
           np.array([[[16, 0, 0]]]),             # site out of range
           np.array([[[0, 8, 0]]]),              # slice out of range
           np.array([[[0, 0, 2]]])]              # no such component
    for pts in bad:
        with pytest.raises(P.PmwaError) as e:
            g.npoint_alpha(8, pts)
        assert e.value.status == P.PMWA_EINVAL
