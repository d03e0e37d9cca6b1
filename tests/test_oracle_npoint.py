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
import pytest

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


# ---- resolved by the component of Q, at arbitrary times, several points per
# interval (Supplement S-I with every operator inserted in the interval's
# matrix element)

def _expQ(x):
    return np.array([[np.cosh(x), np.sinh(x)], [np.sinh(x), np.cosh(x)]])


Q_A = [np.array([[0.0, 1.0], [0.0, 0.0]]),   # b: <0|b|1> = 1
       np.array([[0.0, 0.0], [1.0, 0.0]])]   # b+: <1|b+|0> = 1


def test_interval_density_is_the_matrix_element():
    """The oracle's closed product of F factors against the 2x2 matrices of
    e^{x Q} (Q = b + b+) and of b, b+ multiplied out with numpy: on an
    interval with end states p, q, and on the circle of a site without legs
    (the cyclic trace)."""
    rng = np.random.default_rng(4)
    eta = 0.4
    XW = 3.0 * eta / 2.0 ** 59  # beta eta = 1.2
    for _ in range(200):
        g = int(rng.integers(1, 6))
        a = rng.integers(0, 2, g)
        p, q = int(rng.integers(0, 2)), int(rng.integers(0, 2))
        M = int(rng.integers(g + 1, 2 ** 59))
        M1 = np.sort(rng.choice(M, size=g, replace=False)).astype(np.uint64)
        cuts = [0] + [int(v) for v in M1] + [M]
        mat = _expQ(0.0)
        mat = _expQ(cuts[1] * XW) @ mat
        for j in range(g):
            mat = _expQ((cuts[j + 2] - cuts[j + 1]) * XW) @ Q_A[a[j]] @ mat
        want = eta ** g * mat[q, p] / _expQ(M * XW)[q, p]
        got = O.interval_density(p, q, M, M1, a, eta, XW)
        assert got == pytest.approx(want, rel=1e-10, abs=1e-300), (g, a, p, q)
        # the circle of a site without legs: points at increasing time points
        pk = np.sort(rng.choice(2 ** 62 // 8, size=g, replace=False) * 8 + 3).astype(np.uint64)
        pieces = [int(pk[j + 1] >> np.uint64(3)) - int(pk[j] >> np.uint64(3)) for j in range(g - 1)]
        pieces.append(2 ** 59 - sum(pieces))
        mat = np.eye(2)
        for j in range(g):
            mat = _expQ(pieces[j] * XW) @ Q_A[a[j]] @ mat
        want = eta ** g * np.trace(mat) / np.trace(_expQ(2 ** 59 * XW))
        got = O.interval_density(-1, 0, 2 ** 59, pk, a, eta, XW)
        assert got == pytest.approx(want, rel=1e-10, abs=1e-300), (g, a, "circle")


def test_alpha_npoint_reduces_to_the_one_and_two_point_densities():
    Lx, Ly, K = 4, 4, 6
    o = O.Oracle(Lx=Lx, Ly=Ly, beta=2.0, eta=0.4, V=0.5, mu=0.3, n_cycle=6, seed=21)
    o.sweep(15)
    eta = 0.4
    rho, iv = o.rho_alpha(K)
    pair = o.rho_pair(K)
    N = Lx * Ly
    pts1 = np.array([[[s, k, a]] for s in range(N) for k in (0, 3) for a in (0, 1)], dtype=np.int32)
    got1 = o.npoint_alpha(K, pts1)
    want1 = np.array([rho[s, :, a].mean() / eta for s in range(N) for k in (0, 3) for a in (0, 1)])
    assert np.allclose(got1, want1, rtol=1e-13, atol=0)
    pts2 = np.array([[[s, 1, 1], [s, 4, 0]] for s in range(N)], dtype=np.int32)
    got2 = o.npoint_alpha(K, pts2)
    want2 = np.array([np.mean([pair[s, (1 + t) % K, (4 + t) % K, 1, 0] for t in range(K)]) / eta ** 2
                      for s in range(N)])
    assert np.allclose(got2, want2, rtol=1e-12, atol=0)
    with pytest.raises(RuntimeError):
        o.npoint_alpha(K, np.array([[[0, 1, 1], [0, 1, 0]]], dtype=np.int32))  # one point twice


@pytest.mark.parametrize("ops", [
    # three operators on one site (several on one interval), b b+ b
    [(0, 0, 0), (0, 2, 1), (0, 5, 0)],
    # three across two sites
    [(0, 1, 1), (1, 3, 0), (0, 6, 0)],
    # four on one site, b b+ b b+
    [(0, 0, 0), (0, 3, 1), (0, 5, 0), (0, 6, 1)],
    # four across two sites, two on each
    [(0, 0, 0), (1, 2, 1), (0, 4, 1), (1, 6, 0)],
])
def test_alpha_npoint_against_ed(ops):
    """n = 3 and n = 4 component-resolved correlators at unequal times on a
    2x2 torus (beta t = 2, V = 0.5, mu = 0.4, eta = 0.5: odd orders are
    non-zero because eta breaks the U(1) symmetry) against exact
    diagonalisation, averaged over the four translations of the tuple,
    within 4 standard errors from the scatter of 32 independent replicas of
    2000 sweeps (the products of densities have heavy tails, so the error of
    one chain's bins can come out too small)."""
    Lx = Ly = 2
    beta, eta, V, mu, K = 2.0, 0.5, 0.5, 0.4, 8
    N = Lx * Ly

    def shift(s, d):
        x, y = s % Lx, s // Lx
        dx, dy = d % Lx, d // Lx
        return (x + dx) % Lx + Lx * ((y + dy) % Ly)

    want = np.mean([ed.correlator(Lx, Ly, beta, 1.0, V, mu, eta,
                                  [(shift(s, d), k * beta / K, a) for s, k, a in ops]) for d in range(N)])
    tuples = np.array([[[shift(s, d), k, a] for s, k, a in ops] for d in range(N)], dtype=np.int32)
    reps = []
    for r in range(32):
        o = O.Oracle(Lx=Lx, Ly=Ly, beta=beta, eta=eta, V=V, mu=mu, n_cycle=8, seed=100 + r)
        o.sweep(200)
        acc = 0.0
        for _ in range(2000):
            o.sweep(1)
            acc += o.npoint_alpha(K, tuples).mean()
        reps.append(acc / 2000)
    reps = np.array(reps)
    m, s = float(reps.mean()), float(reps.std(ddof=1) / np.sqrt(len(reps)))
    assert abs(m - want) < Z * s, (m, s, want)
    assert s < 0.3 * abs(want), (m, s, want)  # resolved well away from zero
