"""Supplement S-I n-point functions of distinct sites at equal time from
listed site tuples (oracle side): <Q_i1 ... Q_in> = eta^-n <rho_i1 ... rho_in>.

Pins:
  * n = 2 and n = 4 reproduce the correlators assembled independently from
    the same densities (equal-time G(r) and the plaquette function), and the
    result does not depend on the order of the sites in a tuple beyond
    rounding;
  * n = 3 (an odd function, non-zero only because eta breaks the U(1)
    symmetry) on a 3x3 torus at t = 1, eta = 0.5 against exact
    diagonalisation, averaged over the nine translations of the tuple
    (i, i + x, i + x + y), within 4 standard errors of 64 bins.
"""
import numpy as np

from oracle import ed
from oracle import oracle as O

Z = 4.0


def _sites(Lx, Ly):
    idx = np.arange(Lx * Ly)
    return idx, idx % Lx, idx // Lx


def test_two_and_four_points_match_the_assembled_correlators():
    Lx, Ly, K = 6, 4, 5
    o = O.Oracle(Lx=Lx, Ly=Ly, beta=2.0, eta=0.3, V=0.5, mu=0.2, dom_x=3, dom_y=2, n_cycle=6, seed=9)
    o.sweep(12)
    idx, x, y = _sites(Lx, Ly)
    r = o.rho_slices(K)
    eta = 0.3
    nx = (x + 1) % Lx + Lx * y
    ny = x + Lx * ((y + 1) % Ly)
    nxy = (x + 1) % Lx + Lx * ((y + 1) % Ly)
    two = o.npoint(K, np.stack([idx, nx], axis=1))
    assert np.allclose(two, (r * r[nx]).mean(axis=1) / eta ** 2, rtol=1e-13, atol=0)
    four = o.npoint(K, np.stack([idx, nx, ny, nxy], axis=1))
    assert np.allclose(four, (r * r[nx] * r[ny] * r[nxy]).mean(axis=1) / eta ** 4, rtol=1e-13, atol=0)
    back = o.npoint(K, np.stack([nxy, ny, nx, idx], axis=1))
    assert np.allclose(four, back, rtol=1e-14, atol=0)
    one = o.npoint(K, idx[:, None])
    assert np.allclose(one, r.mean(axis=1) / eta, rtol=1e-14, atol=0)


def test_three_points_against_ed():
    Lx = Ly = 3
    beta, eta = 2.0, 0.5
    H, Q = ed.hamiltonians(Lx, Ly, 1.0, 0.0, 0.0, eta)
    w, U = np.linalg.eigh(H - eta * Q)
    p = np.exp(-beta * (w - w.min()))
    Zs = p.sum()
    dim = 1 << (Lx * Ly)
    st = np.arange(dim)

    def q_op(i):
        A = np.zeros((dim, dim))
        A[st ^ (1 << i), st] = 1.0
        return A

    def avg(A):
        return float(p @ np.einsum("ik,ik->k", U, A @ U) / Zs)

    idx, x, y = _sites(Lx, Ly)
    s1 = (x + 1) % Lx + Lx * y
    s2 = (x + 1) % Lx + Lx * ((y + 1) % Ly)
    want = np.mean([avg(q_op(i) @ q_op(int(s1[i])) @ q_op(int(s2[i]))) for i in idx])
    tuples = np.stack([idx, s1, s2], axis=1)
    o = O.Oracle(Lx=Lx, Ly=Ly, beta=beta, eta=eta, n_cycle=8, seed=17)
    o.sweep(500)
    vals = []
    for _ in range(60000):
        o.sweep(1)
        vals.append(o.npoint(4, tuples).mean())
    m, s = O.binned(np.array(vals), 64)
    assert abs(m - want) < Z * s, (m, s, want)
    assert s < 0.05 * want
