"""GPU parity of the Supplement S-I estimators resolved by the component of
Q (pmwa_rho_alpha) and of the unequal-time Green function built from them
(pmwa_green_tau), against the oracle on the same configurations.

  * The per-slice densities and interval ids are equal bit for bit (both
    sides take the same binary64 operations in the same order).
  * G_d(r, dk) agrees to 1e-12 relative (the sums run in another order).
  * Sizes: several tiles of 128 sites with a ragged tail, K from 1 to the
    maximum 64 with ragged values, rmax up to L/2, sites without vertex
    legs, and the 256x256 workload at full size.
  * Arguments out of range return PMWA_EINVAL.
  * t = V = 0 on 32x32: G matches the two-level closed form (exact
    diagonalisation of a 2x2 torus at t = 0) within 4 standard errors.
"""
import numpy as np
import pytest

from oracle import ed
from oracle import oracle as O

import paper_1307_0328_gb300 as P

pytestmark = pytest.mark.gpu

REL = 1e-12

GEOMS = [
    dict(Lx=8, Ly=8, beta=2.0, eta=0.2, n_cycle=6, seed=1, init=1, init_seed=1),
    dict(Lx=2, Ly=2, beta=1.5, eta=0.5, n_cycle=4, seed=3, init=0),
    dict(Lx=8, Ly=8, beta=2.0, eta=0.3, V=1.0, mu=0.7, dom_x=4, dom_y=4, sub_block=2, n_cycle=5,
         exchange_every=1, seed=5),
    dict(Lx=6, Ly=9, beta=4.0, eta=0.15, t=0.0, c_off=0.3, mu=0.8, dom_x=3, dom_y=3, n_cycle=3, seed=11),
    dict(Lx=12, Ly=4, beta=3.0, eta=0.25, V=3.0, mu=-1.5, t=0.7, dom_x=6, dom_y=2, sub_block=2, n_cycle=4, seed=13),
    # few vertices: most sites have no legs
    dict(Lx=4, Ly=4, beta=0.25, t=0.0, c_off=0.1, eta=0.5, n_cycle=4, seed=5),
    # 19 x 17 = 323 sites: two full tiles of 128 threads and a ragged tail
    dict(Lx=19, Ly=17, beta=2.0, eta=0.3, V=0.5, mu=0.4, n_cycle=6, seed=29, init=1, init_seed=4),
]


def _pair(kw, sweeps=6):
    g, o = P.Sim(**kw), O.Oracle(**kw)
    g.sweep(sweeps)
    o.sweep(sweeps)
    assert np.array_equal(g.export(), o.export())
    return g, o


def _close(a, b):
    scale = max(float(np.abs(b).max()), 1e-300)
    assert np.allclose(a, b, rtol=REL, atol=REL * scale), float(np.abs(a - b).max())


def _green_fits(kw, K, rmax):
    """pmwa_green_tau's room: every site's densities (rmax >= 1) and the sums
    in the idle next-configuration slots, 8 cap bytes per site."""
    N, cap = kw["Lx"] * kw["Ly"], P.pmwa_slot_capacity(**kw)
    return ((2 * N * K if rmax > 0 else 0) + 2 * (rmax + 1) * K) <= N * cap


@pytest.mark.parametrize("kw", GEOMS)
def test_rho_alpha_and_green_tau_match_the_oracle(kw):
    """K = 16 and 64 exceed the room for all sites at once on most of these
    lattices, so pmwa_rho_alpha fills it by chunks of sites."""
    g, o = _pair(kw)
    try:
        rmax = min(kw["Lx"], kw["Ly"]) // 2
        for K in (1, 7, 16, 64):
            rg, ivg = g.rho_alpha(K)
            ro, ivo = o.rho_alpha(K)
            assert np.array_equal(rg, ro), K
            assert np.array_equal(ivg, ivo), K
            for r in (0, rmax):
                if K > 16 and r > 0:
                    continue
                if _green_fits(kw, K, r):
                    _close(g.green_tau(K, r), o.green_tau(K, r))
                else:
                    with pytest.raises(P.PmwaError) as e:
                        g.green_tau(K, r)
                    assert e.value.status == P.PMWA_EINVAL
    finally:
        g.close()


def test_full_size_256x256():
    kw = dict(Lx=256, Ly=256, beta=4.0, eta=0.1, dom_x=16, dom_y=16, sub_block=2, exchange_every=2,
              n_cycle=31, init=1, init_seed=7, seed=7)
    g, o = _pair(kw, sweeps=4)
    try:
        K = 8
        rg, ivg = g.rho_alpha(K)
        ro, ivo = o.rho_alpha(K)
        assert np.array_equal(rg, ro)
        assert np.array_equal(ivg, ivo)
        _close(g.green_tau(K, 3), o.green_tau(K, 3))
    finally:
        g.close()


def test_arguments_out_of_range():
    g = P.Sim(Lx=8, Ly=8, beta=1.0, eta=0.3, n_cycle=4, seed=2)
    try:
        for K, rmax in ((0, 1), (65, 1), (8, 5), (8, -1)):
            with pytest.raises(P.PmwaError) as e:
                g.green_tau(K, rmax)
            assert e.value.status == P.PMWA_EINVAL, (K, rmax)
        with pytest.raises(P.PmwaError) as e:
            g.rho_alpha(0)
        assert e.value.status == P.PMWA_EINVAL
    finally:
        g.close()


def test_decoupled_sites_closed_form():
    """t = V = 0, mu = 1, eta = 0.4, beta = 2 on 32x32 in 16x16 domains; 16
    bins of 250 sweeps after 1000 of thermalisation."""
    K = 8
    want = ed.green_tau(2, 2, 2.0, 0.0, 0.0, 1.0, 0.4, K, 1)
    g = P.Sim(Lx=32, Ly=32, beta=2.0, t=0.0, mu=1.0, eta=0.4, c_off=0.5, dom_x=16, dom_y=16, sub_block=2,
              n_cycle=8, seed=21, init=1, init_seed=6)
    try:
        g.sweep(1000)
        g.rows()
        vals = []
        for _ in range(4000):
            g.sweep(1)
            vals.append(g.green_tau(K, 1))
        g.rows()
    finally:
        g.close()
    v = np.array(vals)
    bad = []
    for d, r in ((0, 0), (0, 1), (1, 1)):
        for dk in range(K):
            if r == 0 and dk == 0:
                assert np.all(v[:, d, r, dk] == 0.0)
                continue
            b = v[:, d, r, dk].reshape(16, -1).mean(axis=1)
            m, s = float(b.mean()), float(b.std(ddof=1) / 4.0)
            if not abs(m - want[d, r, dk]) < 4.0 * s:
                bad.append("d%d r%d dk%d %.5f+-%.5f want %.5f" % (d, r, dk, m, s, want[d, r, dk]))
    assert not bad, "; ".join(bad)
