"""ctypes binding of the plain C oracle (pmwa_oracle.c).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  The oracle follows the
paper's Steps 2-6 (Masaki-Kato et al., "Parallelized Quantum Monte Carlo
Algorithm with Nonlocal Worm Updates": Eqs. 1, 2, 4, 5 and Supplement S-I) in
the deterministic arithmetic the GPU path also implements.
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pmwa_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle_pmwa.so")


def build(force=False):
    """Compile the oracle with gcc (no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(_SRC),
                                              os.path.getmtime(os.path.join(_HERE, "pmwa_oracle.h")))):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared",
                           "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class Params(C.Structure):
    _fields_ = [("Lx", C.c_int32), ("Ly", C.c_int32),
                ("beta", C.c_double), ("t", C.c_double), ("V", C.c_double),
                ("mu", C.c_double), ("eta", C.c_double),
                ("seed", C.c_uint64),
                ("dom_x", C.c_int32), ("dom_y", C.c_int32),
                ("exchange_every", C.c_int32), ("n_cycle", C.c_int32),
                ("sub_block", C.c_int32), ("init", C.c_int32),
                ("init_seed", C.c_uint64), ("c_off", C.c_double),
                ("replica", C.c_uint32), ("dom_tau", C.c_int32), ("vertex_window", C.c_double)]


class Row(C.Structure):
    _fields_ = [("sweep", C.c_uint64), ("n_v", C.c_uint64), ("n_k", C.c_uint64),
                ("n_w", C.c_uint64), ("occ_lo", C.c_uint64), ("occ_hi", C.c_uint64),
                ("q_impr", C.c_double), ("w_dom_min", C.c_uint32), ("dom_empty", C.c_uint32)]


ROW_DTYPE = np.dtype([("sweep", "<u8"), ("n_v", "<u8"), ("n_k", "<u8"), ("n_w", "<u8"),
                      ("occ_lo", "<u8"), ("occ_hi", "<u8"), ("q_impr", "<f8"), ("w_dom_min", "<u4"),
                      ("dom_empty", "<u4")])

DEFAULTS = dict(Lx=4, Ly=4, beta=2.0, t=1.0, V=0.0, mu=0.0, eta=0.2, seed=1,
                dom_x=0, dom_y=0, exchange_every=2, n_cycle=8, sub_block=0,
                init=1, init_seed=1, c_off=-1.0, replica=0, dom_tau=1, vertex_window=0.0)

_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        L.or_create.argtypes = [P(Params), P(C.c_void_p)]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_sweep.argtypes = [C.c_void_p, C.c_int64]
        L.or_boundary.argtypes = [C.c_void_p]
        L.or_temporal.argtypes = [C.c_void_p]
        L.or_pdom.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_uint64, C.c_double, C.c_void_p]
        L.or_tile.argtypes = [C.c_void_p, C.c_int]
        L.or_check.argtypes = [C.c_void_p]
        L.or_rows.argtypes = [C.c_void_p, C.c_void_p, C.c_int64]
        L.or_rows.restype = C.c_int64
        L.or_export_bytes.argtypes = [C.c_void_p]
        L.or_export_bytes.restype = C.c_size_t
        L.or_export.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
        L.or_import.argtypes = [C.c_void_p, C.c_void_p, C.c_size_t]
        L.or_sweep_index.argtypes = [C.c_void_p]
        L.or_sweep_index.restype = C.c_uint64
        L.or_set_sweep_index.argtypes = [C.c_void_p, C.c_uint64]
        L.or_rho_slices.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
        L.or_rho_alpha.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p]
        L.or_rho_pair.argtypes = [C.c_void_p, C.c_int32, C.c_void_p]
        L.or_npoint_alpha.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p]
        L.or_interval_density.argtypes = [C.c_int, C.c_int, C.c_uint64, C.c_int, C.c_void_p, C.c_void_p,
                                          C.c_double, C.c_double]
        L.or_interval_density.restype = C.c_double
        L.or_philox4x32_10.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_exp_det.argtypes = [C.c_double]
        L.or_exp_det.restype = C.c_double
        L.or_expm1_det.argtypes = [C.c_double]
        L.or_expm1_det.restype = C.c_double
        L.or_zig_tables.argtypes = [C.c_void_p] * 6
        L.or_exp_deviates.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.c_int64, C.c_void_p]
        L.or_sample_worms.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.c_uint64, C.c_int, C.c_double, C.c_void_p, C.c_int]
        L.or_tables.argtypes = [P(Params)] + [C.c_void_p] * 6
        _lib = L
    return _lib


def make_params(**kw):
    d = dict(DEFAULTS)
    d.update(kw)
    for k in ("cap_site", "rows_cap", "legs_hint"):  # device capacities: no meaning here
        d.pop(k, None)
    if not d["dom_x"]:
        d["dom_x"] = d["Lx"]
    if not d["dom_y"]:
        d["dom_y"] = d["Ly"]
    if not d["dom_tau"]:
        d["dom_tau"] = 1
    return Params(**d)


class Oracle:
    """One PMWA instance on the CPU."""

    def __init__(self, **kw):
        self.params = make_params(**kw)
        self.h = C.c_void_p()
        rc = lib().or_create(C.byref(self.params), C.byref(self.h))
        if rc:
            raise ValueError("or_create failed with status %d" % rc)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_destroy(self.h)
            self.h = None

    def _ok(self, rc, what):
        if rc:
            raise RuntimeError("%s failed with status %d" % (what, rc))

    def sweep(self, n=1):
        self._ok(lib().or_sweep(self.h, n), "or_sweep")

    def boundary(self):
        self._ok(lib().or_boundary(self.h), "or_boundary")

    def temporal(self):
        self._ok(lib().or_temporal(self.h), "or_temporal")

    def tile(self, stop_after=6):
        self._ok(lib().or_tile(self.h, stop_after), "or_tile")

    def check(self):
        return lib().or_check(self.h)

    @property
    def sweep_index(self):
        return lib().or_sweep_index(self.h)

    @sweep_index.setter
    def sweep_index(self, v):
        lib().or_set_sweep_index(self.h, v)

    def rows(self, max_rows=1 << 24):
        out = np.zeros(max_rows, dtype=ROW_DTYPE) if max_rows < 4096 else None
        chunks = []
        while True:
            buf = np.zeros(min(max_rows, 65536), dtype=ROW_DTYPE)
            n = lib().or_rows(self.h, buf.ctypes.data, len(buf))
            chunks.append(buf[:n])
            if n < len(buf):
                break
        del out
        return np.concatenate(chunks)

    def export(self):
        n = lib().or_export_bytes(self.h)
        buf = np.zeros(n // 8, dtype=np.uint64)
        self._ok(lib().or_export(self.h, buf.ctypes.data, n), "or_export")
        return buf

    def import_(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint64)
        self._ok(lib().or_import(self.h, buf.ctypes.data, buf.nbytes), "or_import")

    def rho_slices(self, K):
        N = self.params.Lx * self.params.Ly
        out = np.zeros((N, K), dtype=np.float64)
        self._ok(lib().or_rho_slices(self.h, K, out.ctypes.data), "or_rho_slices")
        return out

    def npoint(self, K, tuples):
        """Supplement S-I for n distinct sites at equal time:
        <Q_i1(tau) ... Q_in(tau)> = eta^-n <rho_i1(tau) ... rho_in(tau)>,
        averaged over the K slices, for each row of `tuples` (m x n site
        indices).  Distinct sites never share an interval, so the densities
        multiply.  Per tuple: for each slice the product over the sites in
        row order from 1.0, summed over the slices in order, divided by K and
        then by eta^n (eta multiplied n times from 1.0)."""
        t = np.asarray(tuples, dtype=np.int64)
        m, n = t.shape
        rho = self.rho_slices(K)
        eta = self.params.eta
        acc = np.zeros(m)
        for k in range(K):
            p = np.ones(m)
            for c in range(n):
                p = p * rho[t[:, c], k]
            acc = acc + p
        etan = 1.0
        for _ in range(n):
            etan = etan * eta
        return (acc / float(K)) / etan

    def rho_alpha(self, K):
        """(rho (N, K, 2) with [..., 0] for b and [..., 1] for b+, iv (N, K))."""
        N = self.params.Lx * self.params.Ly
        out = np.zeros((N, K, 2), dtype=np.float64)
        iv = np.zeros((N, K), dtype=np.int32)
        self._ok(lib().or_rho_alpha(self.h, K, out.ctypes.data, iv.ctypes.data), "or_rho_alpha")
        return out, iv

    def rho_pair(self, K):
        """(N, K, K, 2, 2): Q_a1 at slice k1 and Q_a2 at slice k2 on one site."""
        N = self.params.Lx * self.params.Ly
        out = np.zeros((N, K, K, 2, 2), dtype=np.float64)
        self._ok(lib().or_rho_pair(self.h, K, out.ctypes.data), "or_rho_pair")
        return out

    def npoint_alpha(self, K, pts):
        """<Q_a1(X_1) ... Q_an(X_n)> for each tuple of n points (site, slice,
        component) in pts (m, n, 3), averaged over the K cyclic shifts of the
        slices: an array (m,)."""
        a = np.ascontiguousarray(pts, dtype=np.int32)
        m, n = a.shape[0], a.shape[1]
        out = np.zeros(m)
        self._ok(lib().or_npoint_alpha(self.h, K, n, m, a.ctypes.data, out.ctypes.data), "or_npoint_alpha")
        return out

    def green_tau(self, K, rmax):
        """Supplement S-I: G_d(r, dk) = <b_{i + r e_d}(tau_k + dk beta/K) b+_i(tau_k)>
        estimated as the average over sites i and slices k of the two-point
        density / eta^2, for d = x, y, r = 0..rmax, dk = 0..K-1 (0 at r = dk = 0,
        where the two operators meet).  Returns an array (2, rmax + 1, K)."""
        p = self.params
        Lx, Ly, N, eta = p.Lx, p.Ly, p.Lx * p.Ly, p.eta
        rho, _ = self.rho_alpha(K)
        pair = self.rho_pair(K)
        idx = np.arange(N)
        x, y = idx % Lx, idx // Lx
        G = np.zeros((2, rmax + 1, K))
        for dk in range(K):
            k2 = (np.arange(K) + dk) % K
            same = pair[:, np.arange(K), k2, 1, 0]            # b+ at k, b at k + dk
            G[:, 0, dk] = same.sum() / (N * K) / eta ** 2
            for r in range(1, rmax + 1):
                for d, j in ((0, (x + r) % Lx + Lx * y), (1, x + Lx * ((y + r) % Ly))):
                    G[d, r, dk] = (rho[j][:, k2, 0] * rho[:, :, 1]).sum() / (N * K) / eta ** 2
        return G


def tile_config(buf, L, T):
    """A configuration of the L x L lattice repeated T x T times on the
    (T L) x (T L) lattice: every site copies its event list, and the legs of
    the bonds that wrapped round the small torus take the tags of the bonds
    they become on the large one (class 2 only at the last column or row).
    A way to start a large lattice from a locally thermalised state that the
    oracle reaches in seconds on the small one."""
    N = L * L
    lists, k = [], 1
    for s in range(N):
        n = int(buf[k] & np.uint64(0x7fffffff))
        lists.append((buf[k], buf[k + 1:k + 1 + n].copy()))
        k += 1 + n
    LL = T * L
    out = [np.array([LL * LL], dtype=np.uint64)]
    for y in range(LL):
        for x in range(LL):
            hd, ev = lists[(x % L) + L * (y % L)]
            ev = ev.copy()
            tag = (ev >> np.uint64(2)) & np.uint64(7)
            for d, c in ((0, x), (1, y)):
                # the wrap bond of the small torus joins c = L-1 (mod L) to c = 0
                # (mod L); on the large torus only c = LL-1 / 0 keeps class 2
                if (c % L == L - 1 and c != LL - 1) or (c % L == 0 and c != 0):
                    m = tag == np.uint64(3 * d + 2)
                    ev[m] = (ev[m] & ~np.uint64(7 << 2)) | np.uint64((3 * d + 1) << 2)
            out.append(np.array([hd], dtype=np.uint64))
            out.append(ev)
    return np.concatenate(out)


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(c.ctypes.data, k.ctypes.data, o.ctypes.data)
    return o


def interval_density(p, q, M, M1, a, eta, XW):
    """Joint density of the operators Q_a[j] at the points with M1[j] worm
    points below them on one interval (p < 0: a site without legs, M1 = pk)."""
    m1 = np.ascontiguousarray(M1, dtype=np.uint64)
    aa = np.ascontiguousarray(a, dtype=np.int32)
    return lib().or_interval_density(p, q, M, len(m1), m1.ctypes.data, aa.ctypes.data, eta, XW)


def pdom(p, q, M1, M2, XW):
    """Step 1's probabilities (P(s'=0), P(s'=1)) of the new boundary state."""
    out = np.zeros(2)
    lib().or_pdom(p, q, M1, M2, XW, out.ctypes.data)
    return out


def zig_tables():
    X = np.zeros(257); F = np.zeros(257); W = np.zeros(256)
    K = np.zeros(256, dtype=np.uint64); R = C.c_double(); v = C.c_double()
    lib().or_zig_tables(X.ctypes.data, F.ctypes.data, W.ctypes.data, K.ctypes.data,
                        C.byref(R), C.byref(v))
    return dict(X=X, F=F, W=W, K=K, R=R.value, v=v.value)


def exp_deviates(n, seed=1, unit=0, c2=0, sweep=0):
    out = np.zeros(n)
    rc = lib().or_exp_deviates(seed, unit, c2, sweep, n, out.ctypes.data)
    if rc:
        raise RuntimeError("or_exp_deviates status %d" % rc)
    return out


def sample_worms(M, sigma, SW, seed=1, unit=0, c2=0, sweep=0, maxn=4096):
    offs = np.zeros(maxn, dtype=np.uint64)
    n = lib().or_sample_worms(seed, unit, c2, sweep, M, sigma, SW, offs.ctypes.data, maxn)
    if n < 0:
        raise RuntimeError("or_sample_worms failed")
    return offs[:n]


def tables(**kw):
    p = make_params(**kw)
    d4 = np.zeros(4); D = C.c_double(); TV = np.zeros(4, dtype=np.uint64)
    TH = np.zeros(256, dtype=np.uint64); SV = C.c_double(); SW = C.c_double()
    lib().or_tables(C.byref(p), d4.ctypes.data, C.byref(D), TV.ctypes.data, TH.ctypes.data,
                    C.byref(SV), C.byref(SW))
    return dict(d=d4, D=D.value, TV=TV, TH=TH.reshape(16, 4, 4), SV=SV.value, SW=SW.value)


def observables(rows, p):
    """Per-sweep physical observables from measured rows (Step 6).

    E/N = (N_b C - n_v / beta) / N with C = max E(s) + c_off; density from the
    occupied time; <Q>/N raw = n_w / (beta eta N), improved = sum x g(x) /
    (beta eta N); kinetic <b+_i b_j + h.c.> per bond = n_k / (beta t N_b).
    """
    N = p.Lx * p.Ly
    Nb = 2 * N
    c_off = 0.5 * p.t if p.c_off < 0 else p.c_off
    E = [p.V * (s & 1) * (s >> 1) - (p.mu / 4.0) * ((s & 1) + (s >> 1)) for s in range(4)]
    Cc = max(E) + c_off
    nv = rows["n_v"].astype(np.float64)
    occ = rows["occ_lo"].astype(np.float64) + rows["occ_hi"].astype(np.float64) * 2.0 ** 64
    out = dict(
        E=(Nb * Cc - nv / p.beta) / N,
        n=occ / (2.0 ** 62 * N),
        Q_raw=rows["n_w"].astype(np.float64) / (p.beta * p.eta * N),
        Q_impr=rows["q_impr"] / (p.beta * p.eta * N),
    )
    if p.t > 0:
        out["kin"] = rows["n_k"].astype(np.float64) / (p.beta * p.t * Nb)
    return out


def binned(x, nbins=32):
    """Mean and standard error from nbins equal bins of the series."""
    x = np.asarray(x, dtype=np.float64)
    m = len(x) // nbins
    b = x[: m * nbins].reshape(nbins, m).mean(axis=1)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(nbins))
