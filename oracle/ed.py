"""Exact diagonalisation of H_eta = H - eta Q for the hard-core Bose-Hubbard
model on a small periodic Lx x Ly lattice (TEST INFRASTRUCTURE ONLY).

H is Eq. 5 of the paper read per bond over the same bond list the Monte Carlo
uses (bond b = 2a + d joins a to a + x^ or a + y^, so a 2-site-wide direction
carries every pair twice):
    H = sum_b [ -t (b+_a b_c + b+_c b_a) + V n_a n_c - (mu/4)(n_a + n_c) ],
which is -t sum(b+b + h.c.) + V sum n n - mu sum_i n_i on the square lattice
(each site ends 4 bonds), and Q = sum_i (b_i + b+_i) (the worm source term).
Thermal averages at inverse temperature beta from numpy's eigh.
"""
import numpy as np


def bonds(Lx, Ly):
    out = []
    for y in range(Ly):
        for x in range(Lx):
            a = x + Lx * y
            out.append((a, (x + 1) % Lx + Lx * y))
            out.append((a, x + Lx * ((y + 1) % Ly)))
    return out


def _ops(N):
    dim = 1 << N
    states = np.arange(dim)
    occ = [((states >> i) & 1).astype(np.float64) for i in range(N)]
    return dim, states, occ


def hamiltonians(Lx, Ly, t, V, mu, eta):
    """Dense H (model only) and Q; H_eta = H - eta Q."""
    N = Lx * Ly
    dim, states, occ = _ops(N)
    H = np.zeros((dim, dim))
    diag = np.zeros(dim)
    for a, c in bonds(Lx, Ly):
        diag += V * occ[a] * occ[c] - (mu / 4.0) * (occ[a] + occ[c])
        # hopping: |..1_a..0_c..> <-> |..0_a..1_c..>
        m = (occ[a] == 1) & (occ[c] == 0)
        src = states[m]
        dst = src ^ (1 << a) ^ (1 << c)
        H[dst, src] += -t
        H[src, dst] += -t
    H[np.arange(dim), np.arange(dim)] += diag
    Q = np.zeros((dim, dim))
    for i in range(N):
        src = states
        dst = states ^ (1 << i)
        Q[dst, src] += 1.0
    return H, Q


def thermal(Lx, Ly, beta, t, V, mu, eta, slices_r=True):
    """Exact thermal averages: E/N (of H), <n>, <Q>/N, <b+b+h.c.> per bond,
    G_QQ(r) = <Q_i Q_{i+r x^}> averaged over i, r = 1..Lx-1, and the plaquette
    4-point function <Q_i Q_{i+x} Q_{i+y} Q_{i+x+y}> averaged over i."""
    N = Lx * Ly
    H, Q = hamiltonians(Lx, Ly, t, V, mu, eta)
    Heta = H - eta * Q
    w, U = np.linalg.eigh(Heta)
    w0 = w.min()
    p = np.exp(-beta * (w - w0))
    Z = p.sum()

    def avg(A):
        diag = np.einsum("ik,ik->k", U, A @ U)   # <k|A|k> in the eigenbasis
        return float(p @ diag / Z)

    dim, states, occ = _ops(N)
    nop = np.diag(sum(occ))
    Hkin = H - np.diag(np.diag(H))
    out = dict(E=avg(H) / N, n=avg(nop) / N, Q=avg(Q) / N,
               kin=avg(-Hkin) / (t * 2 * N) if t > 0 else 0.0)
    if slices_r:
        G = []
        Qi = []
        for i in range(N):
            A = np.zeros((dim, dim))
            A[states ^ (1 << i), states] = 1.0
            Qi.append(A)
        # 4-point function on a plaquette: <Q_i Q_{i+x} Q_{i+y} Q_{i+x+y}>
        acc = 0.0
        for y in range(Ly):
            for x in range(Lx):
                s0 = x + Lx * y
                s1 = (x + 1) % Lx + Lx * y
                s2 = x + Lx * ((y + 1) % Ly)
                s3 = (x + 1) % Lx + Lx * ((y + 1) % Ly)
                acc += avg(Qi[s0] @ Qi[s1] @ Qi[s2] @ Qi[s3])
        out["plaq"] = acc / N
        for r in range(1, Lx):
            acc = 0.0
            for y in range(Ly):
                for x in range(Lx):
                    i = x + Lx * y
                    j = (x + r) % Lx + Lx * y
                    acc += avg(Qi[i] @ Qi[j])
            G.append(acc / N)
        out["G"] = np.array(G)
    return out


def green_tau(Lx, Ly, beta, t, V, mu, eta, K, rmax):
    """Exact single-particle Green function of H_eta at unequal times,
        G_d(r, dk) = (1/N) sum_i Tr[e^{-(beta - tau) H_eta} b_j e^{-tau H_eta} b+_i] / Z,
    j = i + r e_d (d = x, y), tau = dk beta / K, for r = 0..rmax and
    dk = 0..K-1, as an array (2, rmax + 1, K); the entry r = dk = 0 (the two
    operators at one point) is left 0.  In the eigenbasis of H_eta
    (energies w, shifted by their minimum) the trace is
    sum_{m,n} e^{-(beta - tau) w_m - tau w_n} <m|b_j|n> <m|b_i|n>."""
    N = Lx * Ly
    H, Q = hamiltonians(Lx, Ly, t, V, mu, eta)
    w, U = np.linalg.eigh(H - eta * Q)
    w = w - w.min()
    Z = np.exp(-beta * w).sum()
    dim, states, occ = _ops(N)
    B = []
    for i in range(N):
        b = np.zeros((dim, dim))
        src = states[((states >> i) & 1) == 1]
        b[src ^ (1 << i), src] = 1.0
        B.append(U.T @ b @ U)
    G = np.zeros((2, rmax + 1, K))
    for dk in range(K):
        tau = dk * beta / K
        W = np.exp(-(beta - tau) * w[:, None] - tau * w[None, :]) / Z
        for r in range(rmax + 1):
            if r == 0 and dk == 0:
                continue
            for d in range(2):
                acc = 0.0
                for i in range(N):
                    x, y = i % Lx, i // Lx
                    j = (x + r) % Lx + Lx * y if d == 0 else x + Lx * ((y + r) % Ly)
                    acc += float((W * B[j] * B[i]).sum())
                G[d, r, dk] = acc / N
    return G


def correlator(Lx, Ly, beta, t, V, mu, eta, ops):
    """Exact time-ordered correlator of H_eta,
        < T prod_k Q_ak(tau_k) >  with Q_0 = b_i, Q_1 = b+_i at site i,
    ops = [(site, tau, a), ...] with 0 <= tau < beta (operators at equal
    times must sit on different sites, where they commute):
        Tr[e^{-(beta - tau_n) H} O_n e^{-(tau_n - tau_{n-1}) H} ... O_1 e^{-tau_1 H}] / Z
    for the operators sorted by time, tau_1 <= ... <= tau_n, H = H_eta, from
    the eigendecomposition (energies shifted by their minimum)."""
    N = Lx * Ly
    H, Q = hamiltonians(Lx, Ly, t, V, mu, eta)
    w, U = np.linalg.eigh(H - eta * Q)
    w = w - w.min()
    Z = np.exp(-beta * w).sum()
    dim, states, occ = _ops(N)
    order = sorted(range(len(ops)), key=lambda k: ops[k][1])
    M = np.diag(np.exp(-ops[order[0]][1] * w))           # e^{-tau_1 H}
    prev = ops[order[0]][1]
    for j, k in enumerate(order):
        i, tau, a = ops[k]
        if j:
            M = np.diag(np.exp(-(tau - prev) * w)) @ M
            prev = tau
        b = np.zeros((dim, dim))
        if a == 0:   # b_i: 1 -> 0
            src = states[((states >> i) & 1) == 1]
        else:        # b+_i: 0 -> 1
            src = states[((states >> i) & 1) == 0]
        b[src ^ (1 << i), src] = 1.0
        M = (U.T @ b @ U) @ M
    M = np.diag(np.exp(-(beta - prev) * w)) @ M
    return float(np.trace(M) / Z)


def single_site(beta, mu, eta):
    """Closed form at t = 0, V = 0, where the sites decouple.  Each site is
    h = -mu n - eta (b + b+) = -mu/2 + (mu/2) sz - eta sx (sz = 1 - 2n), a spin
    in a field of size D = sqrt(mu^2/4 + eta^2), so
        <n> = 1/2 + (mu / (4 D)) tanh(beta D),  <Q_i> = (eta / D) tanh(beta D),
    and E/N = -mu <n>."""
    D = np.sqrt(mu * mu / 4.0 + eta * eta)
    th = np.tanh(beta * D)
    n = 0.5 + (mu / (4.0 * D)) * th
    Q = (eta / D) * th
    return dict(n=n, Q=Q, E=-mu * n)


def thermal_lowest(Lx, Ly, beta, t, V, mu, eta, k=60):
    """Thermal averages (E/N of H, <n>, <Q>/N, <b+b + h.c.> per bond) from
    the k lowest eigenstates of H_eta (sparse Lanczos, scipy's eigsh), for
    lattices too large for dense diagonalisation at low temperature.  The
    Boltzmann weight of the highest state kept is returned as p_last; the
    truncation is valid when it is negligible (e.g. < 1e-30)."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as sla
    N = Lx * Ly
    dim, states, occ = _ops(N)
    diag = np.zeros(dim)
    rows, cols, vals = [], [], []
    for a, c in bonds(Lx, Ly):
        diag += V * occ[a] * occ[c] - (mu / 4.0) * (occ[a] + occ[c])
        m = (occ[a] == 1) & (occ[c] == 0)
        src = states[m]
        dst = src ^ (1 << a) ^ (1 << c)
        rows += [dst, src]
        cols += [src, dst]
        vals += [np.full(len(src), -t)] * 2
    Hk = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(dim, dim))
    H = Hk + sp.diags(diag)
    Q = sp.csr_matrix((np.ones(N * dim), (np.concatenate([states ^ (1 << i) for i in range(N)]),
                                           np.tile(states, N))), shape=(dim, dim))
    nop = sp.diags(np.sum(occ, axis=0))
    w, U = sla.eigsh(H - eta * Q, k=k, which="SA", tol=1e-12)
    order = np.argsort(w)
    w, U = w[order], U[:, order]
    p = np.exp(-beta * (w - w[0]))
    Z = p.sum()

    def avg(A):
        return float(p @ np.einsum("ik,ik->k", U, A @ U) / Z)

    return dict(E=avg(H) / N, n=avg(nop) / N, Q=avg(Q) / N,
                kin=avg(-Hk) / (t * 2 * N) if t > 0 else 0.0, p_last=float(p[-1] / Z))
