"""The two cheaper pre-decisions the GPU takes before a binary64 test of the
deterministic specification, checked on the CPU against the test they stand
for.  Both must give the exact test's answer wherever they decide; the bit-
exact GPU parity tests check the kernels, these check the margin arguments.

1. The ziggurat's wedge test y < e^-x on strip i (x in [X[i+1], X[i]], y in
   [F[i], F[i+1]]) decided by the tangent of e^-x at X[i+1] (a lower bound)
   and the chord (an upper bound, e^-x being convex), each moved by
   eps = F[i+1] 2^-40 away from the curve.
2. The Eq. 4 heat bath over the 16 root states of a boundary vertex decided
   from binary32 weights when the uniform lies more than 2^-12 from every
   cumulative fraction (and from 0 and 1); the binary32 fractions lie within
   2^-16 of the binary64 ones.
"""
import numpy as np
import pytest

import paper_1307_0328_gb300 as P


def _tables():
    t = P.pmwa_tables(Lx=8, Ly=8, beta=2.0, eta=0.2)
    X, F, W = np.array(t["X"]), np.array(t["F"]), np.array(t["W"])
    K = np.array(t["K"], dtype=np.uint64)
    return X, F, W, K


def test_wedge_bounds_agree_with_the_exponential():
    """4e6 wedge draws over all strips: the bounds never contradict y < e^-x,
    every decided draw lies at least the margin from the curve, and fewer
    than 0.1 % of the draws are left to the exact exponential."""
    X, F, W, K = _tables()
    S = np.zeros(256)
    S[1:] = (F[1:256] - F[2:257]) / (X[1:256] - X[2:257])
    rng = np.random.default_rng(1)
    n = 4_000_000
    i = rng.integers(1, 256, n)
    u = np.maximum(rng.integers(0, 2 ** 53, n, dtype=np.uint64), K[i])  # the wedge: u >= K[i]
    x = u.astype(np.float64) * W[i]
    t1 = rng.integers(0, 2 ** 53, n, dtype=np.uint64).astype(np.float64) * 2.0 ** -53
    y = F[i] + t1 * (F[i + 1] - F[i])
    fa = F[i + 1]
    dl = x - X[i + 1]
    eps = fa * 2.0 ** -40
    lo = fa * (1.0 - dl) - eps
    hi = (fa + dl * S[i]) + eps
    e = np.exp(-x)
    exact = y < e
    acc, rej = y < lo, y > hi
    assert not np.any(acc & rej)
    assert not np.any(acc & ~exact)
    assert not np.any(rej & exact)
    # the decided draws keep (almost all of) the margin from the curve, far
    # beyond a few units in the last place of exp
    assert np.min((e - y)[acc] / fa[acc]) > 0.5 * 2.0 ** -40
    assert np.min((y - e)[rej] / fa[rej]) > 0.5 * 2.0 ** -40
    assert 1.0 - np.mean(acc | rej) < 1e-3


def _weights(far, single, I, S, dvw, tk, XW, dtype):
    """Eq. 4 root-state weights of one vertex in the given precision: the
    vertex weight of S times the four leg factors F(sigma, I XW) with
    F(0, x) = 2 + expm1(-2x), F(1, x) = -expm1(-2x) (the order of the
    kernels: dn a, dn b, up a, up b)."""
    f = lambda sg, e: -e if sg else dtype(2.0) + e
    e = [np.expm1(dtype(-2.0) * dtype(I[k]) * dtype(XW)) for k in range(4)]
    s0, s1, s2, s3 = S & 1, (S >> 1) & 1, (S >> 2) & 1, (S >> 3) & 1
    if s0 + s1 != s2 + s3:
        return dtype(0.0)
    w = dtype(dvw[s0 | (s1 << 1)]) if s0 == s2 else dtype(tk)
    if not single[0]:
        w = w * f(far[0] ^ s0, e[0])
    if not single[1]:
        w = w * f(far[1] ^ s1, e[1])
    w = w * (f(s2 ^ s0, e[2]) if single[0] else f(s2 ^ far[2], e[2]))
    w = w * (f(s3 ^ s1, e[3]) if single[1] else f(s3 ^ far[3], e[3]))
    return w


@pytest.mark.parametrize("V,mu,beta,eta", [(0.0, 0.0, 4.0, 0.1), (3.0, 4.2, 16.0, 0.02), (1.0, -1.5, 2.0, 0.2)])
def test_binary32_heat_bath_agrees_outside_its_margin(V, mu, beta, eta):
    """Random boundary vertices (far states, single-vertex sites, interval
    lengths from one grid point to the whole circle): the binary32 fractions
    lie within 2^-16 of the binary64 ones, and wherever the uniform clears
    every boundary by 2^-12 the two pick the same root state."""
    t = P.pmwa_tables(Lx=8, Ly=8, beta=beta, eta=eta, V=V, mu=mu)
    dvw, tk = list(t["d"]), 1.0
    XW = beta * eta * 2.0 ** -59
    rng = np.random.default_rng(7)
    worst, decided, agree = 0.0, 0, 0
    for _ in range(3000):
        far = rng.integers(0, 2, 4)
        single = rng.random(2) < 0.1
        I = [int(2 ** 59 if single[k % 2] else min(2 ** 59, int(2.0 ** rng.uniform(0, 59)))) for k in range(4)]
        w64 = np.array([_weights(far, single, I, S, dvw, tk, XW, np.float64) for S in range(16)])
        w32 = np.array([_weights(far, single, I, S, dvw, tk, XW, np.float32) for S in range(16)], dtype=np.float32)
        tot64 = 0.0
        cum64 = np.zeros(16)
        for S in range(16):  # the kernels' order S = 0..15
            if w64[S] > 0.0:
                tot64 = tot64 + w64[S]
            cum64[S] = tot64 if w64[S] > 0.0 else 0.0
        if not tot64 > 0.0:
            continue
        c32 = np.cumsum(w32, dtype=np.float32)
        tot32 = np.float32(c32[-1])
        pos = w64 > 0.0
        worst = max(worst, float(np.max(np.abs(c32[pos] / tot32 - cum64[pos] / tot64))))
        for _ in range(20):
            wu = int(rng.integers(0, 2 ** 64, dtype=np.uint64))
            r64 = float(wu >> 11) * 2.0 ** -53
            u = r64 * tot64
            hit = [S for S in range(16) if pos[S] and u < cum64[S]]
            s64 = hit[0] if hit else max(S for S in range(16) if pos[S])
            r = np.float32(float(wu >> 11)) * np.float32(2.0 ** -53)
            fr = c32 / tot32
            p32 = w32 > 0
            near = np.any(p32 & (np.abs(r - fr) <= 2.0 ** -12)) or r <= 2.0 ** -12
            if near:
                continue
            h32 = [S for S in range(16) if p32[S] and r < fr[S]]
            if not h32:
                continue
            decided += 1
            agree += int(h32[0] == s64)
    assert worst < 2.0 ** -16, worst
    assert decided > 40000
    assert agree == decided
