"""Pins of the oracle's building blocks against mathematics that does not come
from the oracle: the statistics of a uniform generator, libm's exp, the
ziggurat's published constant and geometry, the exact worm-number law of
Eq. 1, and the detailed-balance conditions of Eq. 2."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

U32 = 2 ** 32


def _philox_words(n, key=(7, 9), unit=3):
    out = np.zeros((n, 4), dtype=np.uint32)
    for i in range(n):
        out[i] = O.philox([i, unit, 5, 11], list(key))
    return out


# Known-answer vectors of Philox4x32-10 published with the Random123 library
# of Salmon, Moraes, Dror and Shaw (SC'11): (counter, key) -> output words.
PHILOX_KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("ctr,key,want", PHILOX_KAT)
def test_philox_known_answers(ctr, key, want):
    """The oracle's Philox4x32-10 reproduces the published known-answer
    vectors: a wrong multiplier, Weyl constant, round count or word order
    fails here even though it would keep the output uniform."""
    assert [int(x) for x in O.philox(list(ctr), list(key))] == list(want)


def test_philox_uniform_bytes_and_bits():
    """Output bytes are uniform (chi^2) and every output bit is fair."""
    w = _philox_words(20000)
    by = w.view(np.uint8).ravel()
    cnt = np.bincount(by, minlength=256)
    chi2 = ((cnt - by.size / 256) ** 2 / (by.size / 256)).sum()
    assert stats.chi2.sf(chi2, 255) > 1e-4
    bits = np.unpackbits(w.view(np.uint8)).reshape(-1, 128).mean(axis=0)
    assert np.abs(bits - 0.5).max() < 5 * 0.5 / np.sqrt(w.shape[0])


def test_philox_avalanche():
    """Flipping one counter or key bit changes about half the 128 output bits."""
    rng = np.random.default_rng(0)
    flips = []
    for _ in range(300):
        c = rng.integers(0, U32, 4, dtype=np.uint64).astype(np.uint32)
        k = rng.integers(0, U32, 2, dtype=np.uint64).astype(np.uint32)
        base = O.philox(c, k)
        b = rng.integers(0, 192)
        c2, k2 = c.copy(), k.copy()
        if b < 128:
            c2[b // 32] ^= np.uint32(1 << (b % 32))
        else:
            k2[(b - 128) // 32] ^= np.uint32(1 << (b % 32))
        d = O.philox(c2, k2) ^ base
        flips.append(np.unpackbits(d.view(np.uint8)).sum())
    assert abs(np.mean(flips) - 64) < 2.0


def test_exp_det_close_to_libm():
    """exp_det is within 2 ulp of libm exp on [-745, 709]; expm1_det within
    4 ulp of libm expm1 (both taken against numpy's binary64 result)."""
    xs = np.concatenate([np.linspace(-745, 709, 4001), np.linspace(-2, 2, 4001),
                         np.array([0.0, -0.0, 1e-300, -1e-300, 0.5, -0.5])])
    lib = O.lib()
    for x in xs:
        got = lib.or_exp_det(float(x))
        want = math.exp(float(x))
        if want < 2.3e-308:  # subnormal range: absolute check
            assert abs(got - want) <= 4 * 5e-324 + 2e-16 * want
            continue
        assert abs(got - want) <= 2 * math.ulp(want), x
    # every degree band of the series (|x| <= 2^-6, 2^-4, 2^-2, 1) and its
    # edges, both signs, plus the exp_det branch beyond 1
    mags = np.concatenate([np.geomspace(1e-12, 1.0, 6001), np.linspace(0.0, 3.0, 6001),
                           np.array([2.0 ** -6, 2.0 ** -4, 2.0 ** -2, 1.0])])
    mags = np.concatenate([mags, np.nextafter(mags, 0.0), np.nextafter(mags, 4.0)])
    for x in np.concatenate([mags, -mags]):
        got = lib.or_expm1_det(float(x))
        want = math.expm1(float(x))
        assert abs(got - want) <= 4 * math.ulp(want) + 1e-300, x


def test_ziggurat_geometry():
    """The strips have equal area v, R matches the value Marsaglia and Tsang
    (2000) print for the 256-strip exponential ziggurat, 7.69711747013104972,
    and the base strip's rectangle plus tail also has area v."""
    z = O.zig_tables()
    X, F, v, R = z["X"], z["F"], z["v"], z["R"]
    assert R == pytest.approx(7.69711747013104972, rel=1e-13)
    assert v == pytest.approx((R + 1) * math.exp(-R), rel=1e-15)
    areas = X[1:256] * (F[2:257] - F[1:256])
    assert np.allclose(areas, v, rtol=1e-9)
    assert X[0] * F[1] == pytest.approx(v, rel=1e-14)
    assert np.all(np.diff(X[1:257]) < 0)


def test_ziggurat_exponential_law():
    """10^6 deviates pass Kolmogorov-Smirnov against Exp(1); mean and
    variance within 5 sigma of 1."""
    x = O.exp_deviates(1_000_000, seed=12345)
    assert stats.kstest(x, "expon").pvalue > 1e-3
    n = len(x)
    assert abs(x.mean() - 1) < 5 / math.sqrt(n)
    assert abs(x.var() - 1) < 5 * math.sqrt(8 / n)
    # the tail beyond R = 7.697 is reached and correct: P(x > 8) = e^-8
    frac = (x > 8).mean()
    assert abs(frac - math.exp(-8)) < 5 * math.sqrt(math.exp(-8) / n)


def _law(x, sigma, nmax):
    f = math.cosh(x) if sigma == 0 else math.sinh(x)
    p = np.zeros(nmax + 1)
    for n in range(sigma, nmax + 1, 2):
        p[n] = x ** n / math.factorial(n) / f
    return p


@pytest.mark.parametrize("x,sigma,M", [(0.05, 0, 2 ** 40), (0.05, 1, 2 ** 40), (0.7, 1, 2 ** 40),
                                       (1.0, 1, 2 ** 40), (1.7, 1, 2 ** 40), (2.5, 0, 2 ** 40),
                                       (4.0, 1, 2 ** 40), (0.3, 0, 2 ** 40),
                                       (0.3, 0, 2 ** 59), (1.7, 1, 2 ** 59), (0.05, 1, 2 ** 59)])
def test_worm_number_law(x, sigma, M):
    """Eq. 1 for hard-core bosons: P(n) = x^n / n! / f_sigma(x) for n of
    parity sigma, f_0 = cosh, f_1 = sinh.  Chi^2 on 20000 draws, each from
    its own Philox unit; offsets are uniform on the interval (KS).  The two
    interval lengths put the mean spacing SW near 2^40 and near 2^60, the two
    ends of the fixed-point scale arithmetic of the gaps."""
    SW = M / x                      # so that x = M / SW
    draws = 20000
    counts = np.zeros(64, dtype=int)
    pos = []
    for u in range(draws):
        offs = O.sample_worms(M, sigma, SW, seed=99, unit=u)
        n = len(offs)
        assert n % 2 == sigma
        assert np.all(np.diff(offs.astype(np.int64)) > 0) if n > 1 else True
        counts[min(n, 63)] += 1
        pos.extend((offs.astype(np.float64) / M).tolist())
    p = _law(x, sigma, 62)
    exp_ = p * draws
    keep = exp_ > 5
    obs = counts[:63][keep]
    e = exp_[keep]
    rest_o = draws - obs.sum()
    rest_e = draws - e.sum()
    chi2 = ((obs - e) ** 2 / e).sum() + ((rest_o - rest_e) ** 2 / rest_e if rest_e > 5 else 0)
    dof = keep.sum() - 1 + (1 if rest_e > 5 else 0)
    assert dof >= 1
    assert stats.chi2.sf(chi2, dof) > 1e-4, (counts[:8], exp_[:8])
    if len(pos) > 50:
        assert stats.kstest(pos, "uniform").pvalue > 1e-4


@pytest.mark.parametrize("V,mu,t", [(0.0, 0.0, 1.0), (1.0, 0.5, 1.0), (3.0, 4.2, 1.0),
                                    (0.0, -2.0, 1.0), (1.0, 1.2, 0.3)])
def test_directed_loop_detailed_balance(V, mu, t):
    """Eq. 2: for every scattering family the probabilities P(i->j) read off
    the u32 threshold table satisfy w_i P(i->j) = w_j P(j->i), sum to 1, and
    never leave by a zero-weight leg.  At V = mu = 0 there is no bounce."""
    tb = O.tables(V=V, mu=mu, t=t)
    TH = tb["TH"].astype(np.float64)
    d = tb["d"]

    def w(S):
        s0, s1, s2, s3 = S & 1, (S >> 1) & 1, (S >> 2) & 1, (S >> 3) & 1
        if s0 + s1 != s2 + s3:
            return 0.0
        return d[s0 | (s1 << 1)] if s0 == s2 else t

    for S in range(16):
        if w(S) <= 0:
            continue
        for i in range(4):
            T = S ^ (1 << i)
            P = np.diff(np.concatenate([[0.0], TH[S, i]])) / U32
            assert P.sum() == pytest.approx(1.0, abs=1e-12)
            for j in range(4):
                Sj = T ^ (1 << j)
                if w(Sj) == 0:
                    assert P[j] == 0
                    continue
                Pb = np.diff(np.concatenate([[0.0], TH[Sj, j]])) / U32
                assert w(S) * P[j] == pytest.approx(w(Sj) * Pb[i], abs=4.0 / U32 * max(w(S), w(Sj)))
            if V == 0 and mu == 0:
                assert P[i] == 0


def test_vertex_weights_and_thinning():
    """Diagonal weights d(s) = C - E(s), C = max E + t/2 (Eq. 5 per bond);
    thinning thresholds are floor(d/D 2^32)."""
    V, mu, t = 1.5, 0.8, 1.0
    tb = O.tables(V=V, mu=mu, t=t)
    E = np.array([V * (s & 1) * (s >> 1) - mu / 4 * ((s & 1) + (s >> 1)) for s in range(4)])
    C = E.max() + t / 2
    assert np.allclose(tb["d"], C - E, rtol=0, atol=1e-15)
    assert tb["D"] == pytest.approx((C - E).max())
    for s in range(4):
        want = U32 if tb["d"][s] == tb["D"] else math.floor(tb["d"][s] / tb["D"] * U32)
        assert int(tb["TV"][s]) == want
