"""ctypes binding of libpmwa.so (C ABI in include/pmwa.h).

Argument marshalling only: every step of the sweep runs in the library's
CUDA kernels.  Loading fails loudly when the library is missing; there is no
fallback path.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

PMWA_OK, PMWA_EINVAL, PMWA_ECAPACITY, PMWA_ETIMEOUT = 0, 1, 2, 3
PMWA_ECUDA, PMWA_EINVARIANT, PMWA_EROWS = 4, 5, 6


class PmwaError(RuntimeError):
    def __init__(self, call, status):
        super().__init__("%s: %s (status %d)" % (call, pmwa_strerror(status), status))
        self.status = status


class Params(C.Structure):
    _fields_ = [("Lx", C.c_int32), ("Ly", C.c_int32),
                ("beta", C.c_double), ("t", C.c_double), ("V", C.c_double),
                ("mu", C.c_double), ("eta", C.c_double),
                ("seed", C.c_uint64),
                ("dom_x", C.c_int32), ("dom_y", C.c_int32),
                ("exchange_every", C.c_int32), ("n_cycle", C.c_int32),
                ("sub_block", C.c_int32), ("init", C.c_int32),
                ("init_seed", C.c_uint64), ("c_off", C.c_double),
                ("replica", C.c_uint32), ("cap_site", C.c_int32),
                ("rows_cap", C.c_int32), ("legs_hint", C.c_int32), ("dom_tau", C.c_int32),
                ("reserved", C.c_int32 * 1), ("vertex_window", C.c_double)]


ROW_DTYPE = np.dtype([("sweep", "<u8"), ("n_v", "<u8"), ("n_k", "<u8"), ("n_w", "<u8"),
                      ("occ_lo", "<u8"), ("occ_hi", "<u8"), ("q_impr", "<f8"), ("w_dom_min", "<u4"),
                      ("dom_empty", "<u4")])

class Obs(C.Structure):
    _fields_ = [("rows", C.c_int64), ("bins", C.c_int32), ("pad", C.c_int32)] + [
        (k, C.c_double) for k in ("E", "E_err", "E_eta", "E_eta_err", "n", "n_err", "Q_raw", "Q_raw_err",
                                  "Q_impr", "Q_impr_err", "kin", "kin_err", "n_v", "n_w", "w_dom_mean",
                                  "w_dom_min", "dom_empty_frac")]


SERIES = ("E", "E_eta", "n", "Q_raw", "Q_impr", "kin")

DEFAULTS = dict(Lx=8, Ly=8, beta=2.0, t=1.0, V=0.0, mu=0.0, eta=0.2, seed=1, dom_x=0, dom_y=0,
                exchange_every=2, n_cycle=8, sub_block=0, init=1, init_seed=1, c_off=-1.0,
                replica=0, cap_site=0, rows_cap=0, legs_hint=0, dom_tau=1, vertex_window=0.0)

_lib = None


def load(build=True):
    """Load libpmwa.so (building it with nvcc first if it is stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError("libpmwa.so not found at %s; run __graft_entry__.build()" % path)
    L = C.CDLL(path)
    P, vp, sz = C.POINTER, C.c_void_p, C.c_size_t
    sig = {
        "pmwa_footprint": (sz, [P(Params)]),
        "pmwa_create": (C.c_int, [P(Params), vp, sz, vp, P(vp)]),
        "pmwa_sweep": (C.c_int, [vp, C.c_int64]),
        "pmwa_boundary": (C.c_int, [vp]),
        "pmwa_temporal": (C.c_int, [vp]),
        "pmwa_tile": (C.c_int, [vp, C.c_int32]),
        "pmwa_measure": (C.c_int, [vp, vp, C.c_int64, P(C.c_int64)]),
        "pmwa_rho_slices": (C.c_int, [vp, C.c_int32, vp]),
        "pmwa_rho_slices_static": (C.c_int, [vp, C.c_int32, vp]),
        "pmwa_green": (C.c_int, [vp, C.c_int32, C.c_int32, vp, vp, vp]),
        "pmwa_export_bytes": (C.c_int, [vp, P(sz)]),
        "pmwa_export": (C.c_int, [vp, vp, sz]),
        "pmwa_import": (C.c_int, [vp, vp, sz]),
        "pmwa_check": (C.c_int, [vp, P(C.c_int64), P(C.c_int32)]),
        "pmwa_rho_alpha": (C.c_int, [vp, C.c_int32, vp, vp]),
        "pmwa_slot_capacity": (C.c_int, [P(Params), P(C.c_int32)]),
        "pmwa_green_tau": (C.c_int, [vp, C.c_int32, C.c_int32, vp]),
        "pmwa_npoint": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int64, vp, vp]),
        "pmwa_npoint_alpha": (C.c_int, [vp, C.c_int32, C.c_int32, C.c_int64, vp, vp]),
        "pmwa_get_sweep": (C.c_int, [vp, P(C.c_uint64)]),
        "pmwa_set_sweep": (C.c_int, [vp, C.c_uint64]),
        "pmwa_destroy": (C.c_int, [vp]),
        "pmwa_tables": (C.c_int, [P(Params)] + [vp] * 10),
        "pmwa_strerror": (C.c_char_p, [C.c_int]),
        "pmwa_profile": (C.c_int, [vp, C.c_int32]),
        "pmwa_set_n_cycle": (C.c_int, [vp, C.c_int32]),
        "pmwa_tile_plan": (C.c_int, [P(Params), vp, vp, vp]),
        "pmwa_tile_smem": (C.c_int32, [P(Params)]),
        "pmwa_batch_footprint": (sz, [vp, C.c_int32]),
        "pmwa_batch_create": (C.c_int, [vp, C.c_int32, vp, sz, vp, P(vp)]),
        "pmwa_batch_sweep": (C.c_int, [vp, C.c_int64]),
        "pmwa_batch_graph": (C.c_int, [vp, C.c_int32]),
        "pmwa_batch_instance": (C.c_int, [vp, C.c_int32, P(vp)]),
        "pmwa_batch_set_active": (C.c_int, [vp, C.c_int32, C.c_int32]),
        "pmwa_batch_set_n_cycle": (C.c_int, [vp, C.c_int32, C.c_int32]),
        "pmwa_batch_last_ms": (C.c_int, [vp, P(C.c_double)]),
        "pmwa_batch_destroy": (C.c_int, [vp]),
        "pmwa_batch_tables_bytes": (sz, [vp, C.c_int32]),
        "pmwa_batch_from_handles": (C.c_int, [vp, C.c_int32, vp, sz, vp, P(vp)]),
        "pmwa_profile_read": (C.c_int, [vp, vp, vp, C.c_int32]),
        "pmwa_profile_phases": (C.c_int, [vp, vp, C.c_int32]),
        "pmwa_row_observables": (C.c_int, [P(Params), vp, C.c_int64, vp]),
        "pmwa_observables": (C.c_int, [P(Params), vp, C.c_int64, C.c_int32, P(Obs)]),
        "pmwa_n_cycle": (C.c_int, [P(Params), vp, C.c_int64, P(C.c_int32)]),
        "pmwa_set_loop_caps": (C.c_int, [vp, C.c_int32, C.c_int32]),
        "pmwa_philox_blocks": (C.c_int, [vp, C.c_int64, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    _lib = L
    return L


def make_params(**kw):
    d = dict(DEFAULTS)
    unknown = set(kw) - set(d)
    if unknown:
        raise TypeError("unknown parameters: %s" % sorted(unknown))
    d.update(kw)
    p = Params()
    for k, v in d.items():
        setattr(p, k, v)
    return p


def _check(call, rc):
    if rc:
        raise PmwaError(call, rc)


# -- thin wrappers with the C names ------------------------------------------
def pmwa_strerror(status):
    return load().pmwa_strerror(status).decode()


def pmwa_footprint(p):
    return load().pmwa_footprint(C.byref(p))


def pmwa_create(p, arena_ptr, arena_bytes, stream_ptr):
    h = C.c_void_p()
    _check("pmwa_create", load().pmwa_create(C.byref(p), arena_ptr, arena_bytes, stream_ptr, C.byref(h)))
    return h


def pmwa_sweep(h, n):
    _check("pmwa_sweep", load().pmwa_sweep(h, n))


def pmwa_boundary(h):
    _check("pmwa_boundary", load().pmwa_boundary(h))


def pmwa_temporal(h):
    _check("pmwa_temporal", load().pmwa_temporal(h))


def pmwa_tile(h, stop_after):
    _check("pmwa_tile", load().pmwa_tile(h, stop_after))


def pmwa_measure(h, max_rows=1 << 20):
    """Drain up to max_rows pending measurement rows (oldest first)."""
    chunks = []
    while True:
        buf = np.empty(min(max_rows, 4096), dtype=ROW_DTYPE)
        n = C.c_int64()
        _check("pmwa_measure", load().pmwa_measure(h, buf.ctypes.data, len(buf), C.byref(n)))
        chunks.append(buf[: n.value])
        if n.value < len(buf):
            break
    return np.concatenate(chunks)


def pmwa_rho_slices(h, N, K):
    out = np.zeros((N, K), dtype=np.float64)
    _check("pmwa_rho_slices", load().pmwa_rho_slices(h, K, out.ctypes.data))
    return out


def pmwa_green(h, K, rmax):
    """Equal-time <Q_i Q_{i+r}> along x and y (r = 1..rmax) and the plaquette
    4-point function, from the worm densities of the current configuration."""
    gx = np.zeros(rmax)
    gy = np.zeros(rmax)
    pl = C.c_double()
    _check("pmwa_green", load().pmwa_green(h, K, rmax, gx.ctypes.data, gy.ctypes.data, C.byref(pl)))
    return gx, gy, pl.value


def pmwa_rho_alpha(h, N, K):
    """(rho (N, K, 2): [..., 0] for b, [..., 1] for b+; iv (N, K) int32)."""
    rho = np.zeros((N, K, 2), dtype=np.float64)
    iv = np.zeros((N, K), dtype=np.int32)
    _check("pmwa_rho_alpha", load().pmwa_rho_alpha(h, K, rho.ctypes.data, iv.ctypes.data))
    return rho, iv


def pmwa_green_tau(h, K, rmax):
    """G_d(r, dk) as an array (2, rmax + 1, K)."""
    g = np.zeros((2, rmax + 1, K), dtype=np.float64)
    _check("pmwa_green_tau", load().pmwa_green_tau(h, K, rmax, g.ctypes.data))
    return g


def pmwa_npoint(h, K, tuples):
    """<Q_i1 ... Q_in> at equal time for each row of `tuples` (m x n distinct
    sites), averaged over K slices: an array (m,)."""
    t = np.ascontiguousarray(tuples, dtype=np.int32)
    if t.ndim != 2:
        raise ValueError("tuples must be an (m, n) array of site indices")
    out = np.zeros(t.shape[0], dtype=np.float64)
    _check("pmwa_npoint", load().pmwa_npoint(h, K, t.shape[1], t.shape[0], t.ctypes.data, out.ctypes.data))
    return out


def pmwa_npoint_alpha(h, K, pts):
    """<T Q_a1(X_1) ... Q_an(X_n)> for each tuple of n points (site, slice,
    component) in pts (m, n, 3), averaged over the K cyclic shifts of the
    slices: an array (m,)."""
    a = np.ascontiguousarray(pts, dtype=np.int32)
    if a.ndim != 3 or a.shape[2] != 3:
        raise ValueError("pts must be an (m, n, 3) array of (site, slice, component)")
    out = np.zeros(a.shape[0], dtype=np.float64)
    _check("pmwa_npoint_alpha", load().pmwa_npoint_alpha(h, K, a.shape[1], a.shape[0], a.ctypes.data,
                                                         out.ctypes.data))
    return out


def pmwa_rho_slices_static(h, N, K):
    """rho slices with the library's own fixed device scratch (no allocation)."""
    out = np.zeros((N, K), dtype=np.float64)
    _check("pmwa_rho_slices_static", load().pmwa_rho_slices_static(h, K, out.ctypes.data))
    return out


def pmwa_export_bytes(h):
    n = C.c_size_t()
    _check("pmwa_export_bytes", load().pmwa_export_bytes(h, C.byref(n)))
    return n.value


def pmwa_export(h):
    n = pmwa_export_bytes(h)
    buf = np.zeros(n // 8, dtype=np.uint64)
    _check("pmwa_export", load().pmwa_export(h, buf.ctypes.data, n))
    return buf


def pmwa_import(h, buf):
    buf = np.ascontiguousarray(buf, dtype=np.uint64)
    _check("pmwa_import", load().pmwa_import(h, buf.ctypes.data, buf.nbytes))


CHECK_NAMES = {1: "capacity", 2: "tag", 3: "order", 4: "continuity", 5: "base", 6: "bond", 7: "partner",
               8: "conservation"}


def pmwa_check(h):
    """None when every invariant of the current configuration holds, else
    (site, code) of the lowest failing site (code as PMWA_CHECK_*, names in
    CHECK_NAMES; site -1 on a handle whose configuration is undefined)."""
    site, what = C.c_int64(), C.c_int32()
    rc = load().pmwa_check(h, C.byref(site), C.byref(what))
    if rc == 5:
        return (site.value, what.value)
    _check("pmwa_check", rc)
    return None


def pmwa_get_sweep(h):
    s = C.c_uint64()
    _check("pmwa_get_sweep", load().pmwa_get_sweep(h, C.byref(s)))
    return s.value


def pmwa_set_sweep(h, s):
    _check("pmwa_set_sweep", load().pmwa_set_sweep(h, s))


def pmwa_tile_smem(**kw):
    return int(load().pmwa_tile_smem(C.byref(make_params(**kw))))


def pmwa_slot_capacity(**kw):
    c = C.c_int32()
    _check("pmwa_slot_capacity", load().pmwa_slot_capacity(C.byref(make_params(**kw)), C.byref(c)))
    return c.value


def pmwa_tile_plan(**kw):
    """Shared-memory plan of a domain: dict(smem, legcap, oldcap)."""
    a, b, c = C.c_int32(), C.c_int32(), C.c_int32()
    _check("pmwa_tile_plan", load().pmwa_tile_plan(C.byref(make_params(**kw)), C.byref(a), C.byref(b), C.byref(c)))
    return dict(smem=a.value, legcap=b.value, oldcap=c.value)


def pmwa_set_n_cycle(h, n):
    _check("pmwa_set_n_cycle", load().pmwa_set_n_cycle(h, n))


def pmwa_destroy(h):
    _check("pmwa_destroy", load().pmwa_destroy(h))


KERNELS = ("boundary", "tile", "temporal", "unused3", "unused4", "rho", "sweep")


def pmwa_profile(h, enable):
    _check("pmwa_profile", load().pmwa_profile(h, 1 if enable else 0))


def pmwa_profile_read(h):
    ms = np.zeros(8)
    n = np.zeros(8, dtype=np.int64)
    _check("pmwa_profile_read", load().pmwa_profile_read(h, ms.ctypes.data, n.ctypes.data, 8))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KERNELS)}


PHASES = ("vertex_candidates", "leg_merge", "worm_creation", "scatter", "output_measure",
          "scatter_pass_setup", "scatter_moves", "scatter_rounds")


def pmwa_profile_phases(h):
    c = np.zeros(8, dtype=np.uint64)
    _check("pmwa_profile_phases", load().pmwa_profile_phases(h, c.ctypes.data, 8))
    return {k: int(c[i]) for i, k in enumerate(PHASES)}


def pmwa_tables(**kw):
    """Host tables the library derives from the parameters (no GPU needed)."""
    p = make_params(**kw)
    d4 = np.zeros(4); D = C.c_double(); tv = np.zeros(4, dtype=np.uint64)
    th = np.zeros(256, dtype=np.uint64); sv = C.c_double(); sw = C.c_double()
    zx = np.zeros(257); zf = np.zeros(257); zw = np.zeros(256); zk = np.zeros(256, dtype=np.uint64)
    _check("pmwa_tables", load().pmwa_tables(C.byref(p), d4.ctypes.data, C.byref(D), tv.ctypes.data,
                                             th.ctypes.data, C.byref(sv), C.byref(sw), zx.ctypes.data,
                                             zf.ctypes.data, zw.ctypes.data, zk.ctypes.data))
    return dict(d=d4, D=D.value, TV=tv, TH=th.reshape(16, 4, 4), SV=sv.value, SW=sw.value,
                X=zx, F=zf, W=zw, K=zk)


class Sim:
    """One PMWA instance whose configuration lives in a torch-allocated arena."""

    def __init__(self, device="cuda", stream=None, **kw):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: libpmwa has no CPU path")
        self.params = make_params(**kw)
        nbytes = pmwa_footprint(self.params)
        if nbytes == 0:
            raise PmwaError("pmwa_footprint", PMWA_EINVAL)
        self.arena = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.arena.device)
        self.h = pmwa_create(self.params, self.arena.data_ptr(), nbytes, self.stream.cuda_stream)
        self.N = self.params.Lx * self.params.Ly

    def close(self):
        if getattr(self, "h", None):
            pmwa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def sweep(self, n=1):
        pmwa_sweep(self.h, n)

    def boundary(self):
        pmwa_boundary(self.h)

    def temporal(self):
        pmwa_temporal(self.h)

    def tile(self, stop_after=6):
        pmwa_tile(self.h, stop_after)

    def rows(self):
        return pmwa_measure(self.h)

    def export(self):
        return pmwa_export(self.h)

    def import_(self, buf):
        pmwa_import(self.h, buf)

    def rho_slices(self, K):
        return pmwa_rho_slices(self.h, self.N, K)

    def check(self):
        return pmwa_check(self.h)

    def rho_alpha(self, K):
        return pmwa_rho_alpha(self.h, self.N, K)

    def green_tau(self, K, rmax):
        return pmwa_green_tau(self.h, K, rmax)

    def npoint(self, K, tuples):
        return pmwa_npoint(self.h, K, tuples)

    def npoint_alpha(self, K, pts):
        return pmwa_npoint_alpha(self.h, K, pts)

    @property
    def sweep_index(self):
        return pmwa_get_sweep(self.h)

    @sweep_index.setter
    def sweep_index(self, s):
        pmwa_set_sweep(self.h, s)


class Batch:
    """Many independent instances advanced together, one launch per kernel
    per sweep (pmwa_batch_*).  Instance i is exposed as a handle for the
    per-instance calls (rows, export, import, plain sweeps)."""

    def __init__(self, params_list, device="cuda", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: libpmwa has no CPU path")
        self.params = [make_params(**kw) for kw in params_list]
        n = len(self.params)
        arr = (Params * n)(*self.params)
        self._arr = arr
        nbytes = load().pmwa_batch_footprint(arr, n)
        if nbytes == 0:
            raise PmwaError("pmwa_batch_footprint", PMWA_EINVAL)
        self.arena = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.arena.device)
        b = C.c_void_p()
        _check("pmwa_batch_create", load().pmwa_batch_create(arr, n, self.arena.data_ptr(), nbytes,
                                                             self.stream.cuda_stream, C.byref(b)))
        self.b = b
        self.n = n
        self.handles = []
        for i in range(n):
            h = C.c_void_p()
            _check("pmwa_batch_instance", load().pmwa_batch_instance(b, i, C.byref(h)))
            self.handles.append(h)

    def sweep(self, n=1):
        _check("pmwa_batch_sweep", load().pmwa_batch_sweep(self.b, n))

    def graph(self, sweeps):
        _check("pmwa_batch_graph", load().pmwa_batch_graph(self.b, sweeps))

    def set_active(self, i, on):
        _check("pmwa_batch_set_active", load().pmwa_batch_set_active(self.b, i, 1 if on else 0))

    def set_n_cycle(self, i, n):
        _check("pmwa_batch_set_n_cycle", load().pmwa_batch_set_n_cycle(self.b, i, n))

    def last_ms(self):
        v = C.c_double()
        _check("pmwa_batch_last_ms", load().pmwa_batch_last_ms(self.b, C.byref(v)))
        return v.value

    def rows(self, i):
        return pmwa_measure(self.handles[i])

    def export(self, i):
        return pmwa_export(self.handles[i])

    def check(self, i):
        return pmwa_check(self.handles[i])

    def close(self):
        if getattr(self, "b", None):
            load().pmwa_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _rows_arg(rows):
    rows = np.ascontiguousarray(rows, dtype=ROW_DTYPE)
    return rows, (rows.ctypes.data if len(rows) else None)


def observables(rows, p):
    """The Step-6 observables of every measured sweep (pmwa_row_observables):
    a dict of arrays E, E_eta, n, Q_raw, Q_impr and, when t > 0, kin."""
    rows, ptr = _rows_arg(rows)
    out = np.zeros((len(rows), len(SERIES)), dtype=np.float64)
    _check("pmwa_row_observables", load().pmwa_row_observables(C.byref(p), ptr, len(rows),
                                                               out.ctypes.data if len(rows) else None))
    d = {k: out[:, i].copy() for i, k in enumerate(SERIES)}
    if p.t <= 0:
        del d["kin"]
    return d


def summary(rows, p, bins=32):
    """Means with binned standard errors and the worms-per-domain figures
    (pmwa_observables), as a dict."""
    rows, ptr = _rows_arg(rows)
    o = Obs()
    _check("pmwa_observables", load().pmwa_observables(C.byref(p), ptr, len(rows), bins, C.byref(o)))
    return {k: getattr(o, k) for k, _ in Obs._fields_ if k != "pad"}


def n_cycle(p, rows=None):
    """N_cycle by the library's rule: from measured rows, else a priori."""
    nc = C.c_int32()
    if rows is None or len(rows) == 0:
        _check("pmwa_n_cycle", load().pmwa_n_cycle(C.byref(p), None, 0, C.byref(nc)))
    else:
        rows, ptr = _rows_arg(rows)
        _check("pmwa_n_cycle", load().pmwa_n_cycle(C.byref(p), ptr, len(rows), C.byref(nc)))
    return nc.value


def pmwa_set_loop_caps(h, zig_words=64, worm_tries=128):
    _check("pmwa_set_loop_caps", load().pmwa_set_loop_caps(h, zig_words, worm_tries))


def pmwa_philox_blocks(h, ctr_key):
    """Device Philox4x32-10 of each row (c0, c1, c2, c3, k0, k1): an (n, 4) array."""
    a = np.ascontiguousarray(ctr_key, dtype=np.uint32).reshape(-1, 6)
    out = np.zeros((len(a), 4), dtype=np.uint32)
    _check("pmwa_philox_blocks", load().pmwa_philox_blocks(h, len(a), a.ctypes.data, out.ctypes.data))
    return out
