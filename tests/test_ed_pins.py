"""Pins of the exact-diagonalisation tool (oracle/ed.py) against results that
do not come from it: closed forms, a brute-force classical sum and the
one-particle band structure.  These make ED trustworthy as the reference the
Monte Carlo oracle is then compared with."""
import itertools

import numpy as np
import pytest

from oracle import ed


def test_bond_list_each_site_ends_four_bonds():
    for Lx, Ly in [(2, 2), (3, 3), (4, 2)]:
        deg = np.zeros(Lx * Ly, dtype=int)
        for a, c in ed.bonds(Lx, Ly):
            deg[a] += 1
            deg[c] += 1
        assert (deg == 4).all()
        assert len(ed.bonds(Lx, Ly)) == 2 * Lx * Ly


@pytest.mark.parametrize("mu,eta,beta", [(1.0, 0.2, 2.0), (-0.6, 0.5, 1.0), (0.0, 0.3, 4.0)])
def test_decoupled_sites_closed_form(mu, eta, beta):
    """t = V = 0: sites decouple into two-level problems with a closed form."""
    ex = ed.thermal(2, 2, beta, 0.0, 0.0, mu, eta, slices_r=False)
    cf = ed.single_site(beta, mu, eta)
    assert ex["n"] == pytest.approx(cf["n"], rel=1e-10, abs=1e-12)
    assert ex["Q"] == pytest.approx(cf["Q"], rel=1e-10, abs=1e-12)
    assert ex["E"] == pytest.approx(cf["E"], rel=1e-10, abs=1e-12)


def test_classical_limit_matches_brute_force_sum():
    """t = eta = 0: H is diagonal; compare with an explicit Boltzmann sum over
    occupation patterns (pins the V and mu terms and the bond list)."""
    Lx, Ly, beta, V, mu = 3, 2, 1.3, 0.8, 0.4
    N = Lx * Ly
    Z = 0.0
    En = 0.0
    Nn = 0.0
    for occ in itertools.product([0, 1], repeat=N):
        e = sum(V * occ[a] * occ[c] for a, c in ed.bonds(Lx, Ly)) - mu * sum(occ)
        w = np.exp(-beta * e)
        Z += w
        En += e * w
        Nn += sum(occ) * w
    ex = ed.thermal(Lx, Ly, beta, 0.0, V, mu, 0.0, slices_r=False)
    assert ex["E"] == pytest.approx(En / Z / N, rel=1e-12)
    assert ex["n"] == pytest.approx(Nn / Z / N, rel=1e-12)


@pytest.mark.parametrize("Lx,Ly", [(2, 2), (3, 3), (4, 2)])
def test_one_particle_band(Lx, Ly):
    """One boson on the lattice hops freely: energies -2t(cos kx + cos ky)."""
    t = 0.7
    H, _ = ed.hamiltonians(Lx, Ly, t, 0.0, 0.0, 0.0)
    one = [1 << i for i in range(Lx * Ly)]
    h1 = H[np.ix_(one, one)]
    got = np.sort(np.linalg.eigvalsh(h1))
    ks = [(2 * np.pi * i / Lx, 2 * np.pi * j / Ly) for i in range(Lx) for j in range(Ly)]
    want = np.sort([-2 * t * (np.cos(kx) + np.cos(ky)) for kx, ky in ks])
    assert np.allclose(got, want, atol=1e-12)


def test_thermodynamic_derivatives():
    """<Q> = (1/beta) d lnZ/d eta and <N> = (1/beta) d lnZ/d mu (finite
    differences of the partition function built from the eigenvalues)."""
    Lx, Ly, beta, t, V, mu, eta = 2, 2, 1.5, 1.0, 0.7, 0.3, 0.25

    def lnZ(**kw):
        a = dict(t=t, V=V, mu=mu, eta=eta)
        a.update(kw)
        H, Q = ed.hamiltonians(Lx, Ly, a["t"], a["V"], a["mu"], a["eta"])
        w = np.linalg.eigvalsh(H - a["eta"] * Q)
        return np.log(np.exp(-beta * w).sum())

    h = 1e-5
    ex = ed.thermal(Lx, Ly, beta, t, V, mu, eta, slices_r=False)
    N = Lx * Ly
    dq = (lnZ(eta=eta + h) - lnZ(eta=eta - h)) / (2 * h) / beta / N
    dn = (lnZ(mu=mu + h) - lnZ(mu=mu - h)) / (2 * h) / beta / N
    dt = (lnZ(t=t + h) - lnZ(t=t - h)) / (2 * h) / beta / (2 * N)
    assert ex["Q"] == pytest.approx(dq, rel=1e-6)
    assert ex["n"] == pytest.approx(dn, rel=1e-6)
    assert ex["kin"] == pytest.approx(dt, rel=1e-6)


def test_particle_hole_symmetry():
    ex = ed.thermal(3, 3, 2.0, 1.0, 0.0, 0.0, 0.2, slices_r=False)
    assert ex["n"] == pytest.approx(0.5, abs=1e-12)


def test_lowest_states_agree_with_full_diagonalisation():
    """The sparse low-state thermal averages equal the dense ones on 4x2 at
    the strong-coupling, low-temperature parameters of the paper's
    checkerboard-solid point (V/t = 3, mu/t = 4.2, beta t = 16), where the
    states left out carry no weight."""
    for eta in (0.1, 0.3):
        lo = ed.thermal_lowest(4, 2, 16.0, 1.0, 3.0, 4.2, eta, k=40)
        full = ed.thermal(4, 2, 16.0, 1.0, 3.0, 4.2, eta, slices_r=False)
        assert lo["p_last"] < 1e-30
        for k_, k2 in (("E", "E"), ("n", "n"), ("Q", "Q"), ("kin", "kin")):
            assert abs(lo[k_] - full[k2]) < 1e-10, (eta, k_, lo[k_], full[k2])


def test_printed_solid_energy_fixes_the_model_reading():
    """The paper's checkerboard-solid energy (Fig. 2 (a): -2.32222 by DLA at
    V/t = 3, mu/t = 4.2, beta t = 16, L = 128) equals the strong-coupling
    value -mu/2 - 2 t^2/(3 V) of H = -t sum (b+b + h.c.) + V sum n n - mu
    sum n to 1e-4: half filling, and each particle's four virtual hops cost
    3V.  That fixes the reading of the garbled model equation (mu per site,
    V per nearest-neighbour pair)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_energies.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    cs = {r[0]: r for r in rows}["CS"]
    mu, e_dla = float(cs[1]), float(cs[4])
    t, V = 1.0, 3.0
    assert abs(e_dla - (-mu / 2.0 - 2.0 * t * t / (3.0 * V))) < 1e-4
