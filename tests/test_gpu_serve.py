"""Serving loop: jobs that arrive while others run are admitted as memory and
slots free up, advance together with the resident ones, and each job's
result is exactly the one it has when run alone (bit-exact integer counters,
FP64 estimator within 1e-12) and the one the CPU oracle computes for the same
job (the same parameters, domains, sub-blocks and N_cycle)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_1307_0328_gb300 as P  # noqa: E402
from oracle import oracle as O  # noqa: E402
from paper_1307_0328_gb300 import serve  # noqa: E402

ROW_FIELDS = ("sweep", "n_v", "n_k", "n_w", "occ_lo", "occ_hi", "w_dom_min", "dom_empty")


def _jobs():
    specs = [
        (dict(Lx=16, Ly=16, beta=2.0, eta=0.2, mu=0.3), 13, 0.00),
        (dict(Lx=32, Ly=32, beta=4.0, eta=0.1, mu=-0.4), 9, 0.00),
        (dict(Lx=8, Ly=8, beta=1.0, eta=0.3), 21, 0.02),
        (dict(Lx=24, Ly=24, beta=8.0, eta=0.1, mu=0.9), 6, 0.05),
        (dict(Lx=16, Ly=16, beta=16.0, eta=0.1, mu=-1.0), 5, 0.05),
        (dict(Lx=12, Ly=12, beta=2.0, eta=0.2, V=1.0, mu=0.5), 17, 0.10),
        (dict(Lx=32, Ly=32, beta=2.0, eta=0.1), 11, 0.12),
    ]
    jobs = []
    for i, (p, sw, t) in enumerate(specs):
        p = dict(p, seed=900 + i, replica=i, init=1, init_seed=700 + i)
        jobs.append(serve.Job(i, p, sw, t))
    return jobs


def test_each_job_same_alone_and_in_the_mix():
    jobs = _jobs()
    # a budget that holds only some jobs at a time, so admission waits for memory
    fps = []
    for j in _jobs():
        p = dict(j.params)
        p.update(serve.autotune.tune(p))
        fps.append(P.pmwa_footprint(P.make_params(**p)))
    budget = int(sorted(fps)[-1] * 2.5)
    out = serve.run_trace(jobs, budget, max_jobs=4, chunk=4, realtime=False)
    assert out["jobs"] == len(jobs)
    assert out["p99_s"] >= out["p50_s"] > 0
    for j in out["finished"]:
        got = j.result()
        assert len(got) == j.sweeps
        alone = P.Sim(**j.params)
        alone.sweep(j.sweeps)
        want = alone.rows()
        for f in ROW_FIELDS:
            assert np.array_equal(got[f], want[f]), (j.id, f)
        assert np.allclose(got["q_impr"], want["q_impr"], rtol=1e-12, atol=0), j.id
        # the served job against the oracle run of the same job
        o = O.Oracle(**j.params)
        o.sweep(j.sweeps)
        ref = o.rows()
        for f in ROW_FIELDS:
            assert np.array_equal(got[f], ref[f]), (j.id, f, "oracle")
        assert np.allclose(got["q_impr"], ref["q_impr"], rtol=1e-12, atol=0), (j.id, "oracle")
        assert np.array_equal(alone.export(), o.export()), (j.id, "configuration")
