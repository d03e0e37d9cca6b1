"""Continuous-batching serving loop for PMWA simulation jobs.

Jobs (lattice parameters and a number of sweeps) arrive over time.  A job is
admitted as soon as its device footprint fits the free HBM budget and a slot
is free; its configuration then stays resident in its own arena for the whole
job.  Every step all resident jobs advance together, one launch per kernel per
sweep, through a batch built over their handles (pmwa_batch_from_handles,
rebuilt only when the resident set changes).  Finished jobs hand their
measurement rows back and release their memory, which admits the next waiting
jobs while the others keep running.  A job's result does not depend on what
runs beside it: every random draw is keyed by the job's own seed, replica id,
sweep and unit.
"""
import ctypes as C
import time

import numpy as np

from . import _lib
from . import autotune


class Job:
    def __init__(self, jid, params, sweeps, arrival=0.0):
        self.id = jid
        self.params = dict(params)
        self.sweeps = int(sweeps)
        self.arrival = float(arrival)
        self.admitted = None
        self.finished = None
        self.done = 0
        self.rows = []
        self.sim = None

    def result(self):
        return np.concatenate(self.rows) if self.rows else np.zeros(0, dtype=_lib.ROW_DTYPE)


def n_cycle_estimate(p):
    """The library's a-priori N_cycle (pmwa_n_cycle without rows) for a job
    that names none."""
    return _lib.n_cycle(_lib.make_params(**{k: v for k, v in p.items() if k in _lib.DEFAULTS}))


def admission(waiting, used, budget, slots, busy, max_bypass):
    """The waiting jobs to admit now, in arrival order: every job whose
    footprint fits the memory left and a free slot (first fit), so that a
    large job at the head of the queue does not hold back small ones behind
    it.  A job passed over `max_bypass` times blocks the jobs behind it until
    it is admitted (no starvation).  With nothing resident the head job is
    admitted even if it alone exceeds the budget.  Counts each pass-over on
    the job (job.bypassed)."""
    picked = []
    for job in waiting:
        if len(picked) >= slots:
            break
        fits = used + job.footprint <= budget or (not busy and not picked and job is waiting[0])
        if fits:
            picked.append(job)
            used += job.footprint
            continue
        job.bypassed = getattr(job, "bypassed", 0) + 1
        if job.bypassed > max_bypass:
            break
    return picked


class Server:
    def __init__(self, budget_bytes, max_jobs=64, chunk=8, device="cuda", max_bypass=8):
        import torch
        self.torch = torch
        self.budget = int(budget_bytes)
        self.max_jobs = int(max_jobs)
        self.max_bypass = int(max_bypass)
        self.chunk = int(chunk)
        self.device = device
        self.waiting = []
        self.resident = []
        self.finished = []
        self.used = 0
        self.batch = None
        self.batch_arena = None
        self.stream = torch.cuda.current_stream()
        self.vertices = 0
        self.busy_s = 0.0

    # -- admission ----------------------------------------------------------
    def submit(self, job):
        p = dict(job.params)
        p.setdefault("rows_cap", max(64, self.chunk * 2))
        if "dom_x" not in p:
            p.update(autotune.tune(p))
        p.setdefault("n_cycle", n_cycle_estimate(p))
        job.params = p
        job.footprint = _lib.pmwa_footprint(_lib.make_params(**p))
        if job.footprint == 0:
            raise _lib.PmwaError("pmwa_footprint", _lib.PMWA_EINVAL)
        self.waiting.append(job)

    def _admit(self, now):
        picked = admission(self.waiting, self.used, self.budget, self.max_jobs - len(self.resident),
                           bool(self.resident), self.max_bypass)
        for job in picked:
            self.waiting.remove(job)
            job.sim = _lib.Sim(device=self.device, stream=self.stream, **job.params)
            self.used += job.footprint
            job.admitted = now
            self.resident.append(job)
        return bool(picked)

    def _rebuild(self):
        self._drop_batch()
        if not self.resident:
            return
        n = len(self.resident)
        hs = (C.c_void_p * n)(*[j.sim.h.value for j in self.resident])
        lib = _lib.load()
        nbytes = lib.pmwa_batch_tables_bytes(hs, n)
        self.batch_arena = self.torch.empty(nbytes, dtype=self.torch.uint8, device=self.device)
        b = C.c_void_p()
        _lib._check("pmwa_batch_from_handles",
                    lib.pmwa_batch_from_handles(hs, n, self.batch_arena.data_ptr(), nbytes,
                                                self.stream.cuda_stream, C.byref(b)))
        self.batch = b

    def _drop_batch(self):
        if self.batch is not None:
            _lib.load().pmwa_batch_destroy(self.batch)
            self.batch = None
            self.batch_arena = None

    # -- one step -------------------------------------------------------------
    def step(self, now):
        """Admit what fits, advance every resident job, harvest the finished."""
        if self._admit(now) or (self.batch is None and self.resident):
            self._rebuild()
        if not self.resident:
            return False
        s = min(self.chunk, min(j.sweeps - j.done for j in self.resident))
        t0 = time.perf_counter()
        _lib._check("pmwa_batch_sweep", _lib.load().pmwa_batch_sweep(self.batch, s))
        self.busy_s += time.perf_counter() - t0
        done = []
        for j in self.resident:
            r = _lib.pmwa_measure(j.sim.h)
            j.rows.append(r)
            j.done += s
            self.vertices += int(r["n_v"].sum())
            if j.done >= j.sweeps:
                done.append(j)
        if done:
            self._drop_batch()
            for j in done:
                j.finished = time.perf_counter()
                self.resident.remove(j)
                self.used -= j.footprint
                j.sim.close()
                j.sim = None
                self.finished.append(j)
        return True

    def close(self):
        self._drop_batch()
        for j in self.resident:
            if j.sim is not None:
                j.sim.close()


def run_trace(jobs, budget_bytes, max_jobs=64, chunk=8, device="cuda", realtime=True):
    """Serve a trace of Jobs whose `arrival` is in seconds from the start;
    returns per-job latency (finish - arrival), p50/p99 and the aggregate
    vertex-update rate over the wall time of the run."""
    srv = Server(budget_bytes, max_jobs=max_jobs, chunk=chunk, device=device)
    pending = sorted(jobs, key=lambda j: j.arrival)
    t_start = time.perf_counter()
    while pending or srv.waiting or srv.resident:
        now = time.perf_counter() - t_start
        while pending and (pending[0].arrival <= now or not realtime):
            j = pending.pop(0)
            if not realtime:
                j.arrival = now
            srv.submit(j)
        if not srv.step(now):
            if pending:
                time.sleep(max(0.0, min(0.01, pending[0].arrival - now)))
    wall = time.perf_counter() - t_start
    srv.close()
    lat = np.array([(j.finished - t_start) - j.arrival for j in srv.finished])
    return dict(jobs=len(srv.finished), wall_s=wall,
                p50_s=float(np.percentile(lat, 50)), p99_s=float(np.percentile(lat, 99)),
                vertex_updates_per_s=srv.vertices / wall, busy_s=srv.busy_s,
                finished=srv.finished)


def poisson_trace(n=400, rate=20.0, seed=5, sweep_scale=1.0, L_max=1024):
    """The serving workload: Poisson arrivals at `rate` jobs/s; L uniform on
    {32, 64, ..., L_max}, beta t from {2, 4, 8, 16}, mu uniform in [-1, 1],
    eta = 0.1, sweeps uniform in {1000..10000} times sweep_scale (at least 1),
    all drawn with numpy's Philox keyed by `seed`."""
    rng = np.random.Generator(np.random.Philox(seed))
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    Ls = rng.choice(np.arange(32, L_max + 1, 32), n)
    betas = rng.choice([2.0, 4.0, 8.0, 16.0], n)
    mus = rng.uniform(-1.0, 1.0, n)
    sweeps = rng.integers(1000, 10001, n)
    jobs = []
    for i in range(n):
        p = dict(Lx=int(Ls[i]), Ly=int(Ls[i]), beta=float(betas[i]), t=1.0, V=0.0, mu=float(mus[i]),
                 eta=0.1, seed=500000 + i, replica=i % 65536, init=1, init_seed=600000 + i)
        jobs.append(Job(i, p, max(1, int(round(sweeps[i] * sweep_scale))), float(t[i])))
    return jobs
