"""Supplement S-I resolved by the component of Q (Q_b = b, Q_b+ = b+), and
the unequal-time Green function G_d(r, tau) = <b_{i + r e_d}(tau) b+_i(0)>
built from it, on the oracle.

Pins (none of them re-types the oracle's formulas):
  * rho_b + rho_b+ is the total worm density eta g_sigma(I eta) of the
    slice's interval, which does not depend on where the slice sits, on
    every site and slice; on a site without vertex legs the two components
    are equal;
  * two-point densities of one site are unchanged when the two points are
    exchanged; summed over both components they are eta^2 when the points
    share an interval (Q^2 = 1 and Q commutes with e^{x Q}) and the product
    of the two total densities otherwise;
  * t = V = 0: the sites decouple, G(r = 0, tau) is the Green function of one
    two-level site (exact diagonalisation of a 2x2 torus at t = 0, strongly
    asymmetric in tau), and G(r >= 1, tau) = <b>^2, on an 8x8 lattice;
  * 3x3 at t = 1, V = 0, mu = 1.5, eta = 0.3, against exact diagonalisation
    within 4 standard errors.  Particle-hole symmetry is broken there, so
    G(r = 0) at tau = beta/4 and 3 beta/4 differ by about 5 errors and a
    mistake that reverses time inside an interval shows.  (At V = mu = 0 an
    estimator that took two points of one interval as independent was off
    by about 10 errors.)
"""
import numpy as np
import pytest

from oracle import ed
from oracle import oracle as O

Z = 4.0

CONFIGS = [
    dict(Lx=4, Ly=4, beta=2.0, eta=0.3, n_cycle=6, seed=3),
    dict(Lx=6, Ly=4, beta=3.0, eta=0.2, V=1.0, mu=-1.0, dom_x=3, dom_y=2, exchange_every=2, n_cycle=6, seed=11),
    # few vertices: most sites have no legs
    dict(Lx=4, Ly=4, beta=0.25, t=0.0, c_off=0.1, eta=0.5, n_cycle=4, seed=5),
]


def _oracle(kw, sweeps=20):
    o = O.Oracle(**kw)
    o.sweep(sweeps)
    return o


@pytest.mark.parametrize("kw", CONFIGS)
def test_components_sum_to_the_total_density(kw):
    o = _oracle(kw)
    for K in (1, 5, 16):
        rho, iv = o.rho_alpha(K)
        tot = o.rho_slices(K)
        assert np.allclose(rho.sum(axis=2), tot, rtol=1e-13, atol=0)
        free = iv < 0
        assert np.array_equal(rho[free][:, 0], rho[free][:, 1])
        assert np.all(rho >= 0)


def test_sites_without_legs_occur():
    rho, iv = _oracle(CONFIGS[2]).rho_alpha(4)
    assert (iv < 0).any() and (iv >= 0).any()


@pytest.mark.parametrize("kw", CONFIGS)
def test_two_point_symmetry_and_sums(kw):
    o = _oracle(kw)
    K = 6
    eta = kw["eta"]
    pair = o.rho_pair(K)
    tot = o.rho_slices(K)
    _, iv = o.rho_alpha(K)
    # exchange of the two points
    assert np.array_equal(pair, pair.transpose(0, 2, 1, 4, 3))
    s = pair.sum(axis=(3, 4))
    N = pair.shape[0]
    n_same = 0
    for i in range(N):
        for k1 in range(K):
            for k2 in range(K):
                if k1 == k2:
                    assert s[i, k1, k2] == 0.0
                elif iv[i, k1] == iv[i, k2]:
                    n_same += 1
                    assert abs(s[i, k1, k2] - eta * eta) <= 1e-13 * eta * eta
                else:
                    want = tot[i, k1] * tot[i, k2]
                    assert abs(s[i, k1, k2] - want) <= 1e-13 * want
    assert n_same > 0


def test_decoupled_sites_green_function():
    """t = V = 0, mu = 1, eta = 0.4, beta = 2, c_off = 0.5 on 8x8, four
    replicas, K = 8 slices; the error of an average comes from 16 bins of
    375 sweeps (the autocorrelation time at t = 0 is about 100 sweeps)."""
    K = 8
    G = ed.green_tau(2, 2, 2.0, 0.0, 0.0, 1.0, 0.4, K, 1)
    vals = []
    for rep in range(4):
        o = O.Oracle(Lx=8, Ly=8, beta=2.0, t=0.0, mu=1.0, eta=0.4, c_off=0.5, n_cycle=8, seed=50 + rep,
                     init=1, init_seed=rep)
        o.sweep(400)
        for _ in range(1500):
            o.sweep(1)
            vals.append(o.green_tau(K, 1))
    v = np.array(vals)
    msgs, bad = [], []
    for d, r in ((0, 0), (0, 1), (1, 1)):
        for dk in range(K):
            if r == 0 and dk == 0:
                assert np.all(v[:, d, r, dk] == 0.0)
                continue
            m, s = O.binned(v[:, d, r, dk], 16)
            msgs.append("d%d r%d dk%d %.5f+-%.5f ed %.5f" % (d, r, dk, m, s, G[d, r, dk]))
            if not abs(m - G[d, r, dk]) < Z * s:
                bad.append(msgs[-1])
            assert s < 0.03 * G[d, r, dk], msgs[-1]
    assert not bad, "; ".join(bad)


def test_green_function_against_ed_without_particle_hole_symmetry():
    K = 4
    kw = dict(beta=2.0, t=1.0, V=0.0, mu=1.5, eta=0.3)
    G = ed.green_tau(3, 3, kw["beta"], kw["t"], kw["V"], kw["mu"], kw["eta"], K, 1)
    assert abs(G[0, 0, 1] - G[0, 0, 3]) > 0.1 * G[0, 0, 1]
    o = O.Oracle(Lx=3, Ly=3, n_cycle=8, seed=19, **kw)
    o.sweep(500)
    vals = []
    for _ in range(40000):
        o.sweep(1)
        vals.append(o.green_tau(K, 1))
    v = np.array(vals)
    msgs, bad = [], []
    for d, r in ((0, 0), (0, 1), (1, 1)):
        for dk in range(K):
            if r == 0 and dk == 0:
                continue
            m, s = O.binned(v[:, d, r, dk], 64)
            msgs.append("d%d r%d dk%d %.5f+-%.5f ed %.5f" % (d, r, dk, m, s, G[d, r, dk]))
            if not abs(m - G[d, r, dk]) < Z * s:
                bad.append(msgs[-1])
            assert s < 0.05 * G[d, r, dk], msgs[-1]
    assert not bad, "; ".join(bad)
