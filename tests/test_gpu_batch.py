"""Replica batching: many independent instances advanced by one launch per
kernel (pmwa_batch_*) must give, instance by instance, exactly the bytes of
the same instance swept alone (every random draw is keyed by the instance's
own seed, replica id, sweep and unit), with and without a captured CUDA
graph, with inactive instances untouched; and small instances match the CPU
oracle bit for bit."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402

import paper_1307_0328_gb300 as P  # noqa: E402
from paper_1307_0328_gb300 import autotune as A  # noqa: E402

MIXED = [
    dict(Lx=8, Ly=8, beta=2.0, eta=0.2, n_cycle=5, seed=1, replica=0),
    dict(Lx=16, Ly=16, beta=4.0, eta=0.1, V=1.0, mu=0.6, dom_x=8, dom_y=8, sub_block=2, n_cycle=7,
         seed=2, replica=1, exchange_every=1),
    dict(Lx=12, Ly=12, beta=1.0, eta=0.2, mu=-1.5, dom_x=6, dom_y=6, sub_block=2, n_cycle=3, seed=3,
         replica=2),
    dict(Lx=6, Ly=4, beta=8.0, eta=0.05, t=0.5, V=0.3, dom_x=3, dom_y=2, n_cycle=9, seed=4, replica=3,
         exchange_every=3),
    dict(Lx=24, Ly=24, beta=2.0, eta=0.1, mu=1.2, V=1.0, dom_x=12, dom_y=12, sub_block=2, n_cycle=6,
         seed=5, replica=4),
    dict(Lx=4, Ly=4, beta=3.0, eta=0.3, init=0, n_cycle=4, seed=6, replica=5),
]


def _rows_equal(a, b):
    for f in ("sweep", "n_v", "n_k", "n_w", "occ_lo", "occ_hi"):
        assert np.array_equal(a[f], b[f]), f
    assert np.allclose(a["q_impr"], b["q_impr"], rtol=1e-12, atol=0)


@pytest.mark.parametrize("graph", [0, 3])
def test_batch_equals_instances_swept_alone(graph):
    batch = P.Batch(MIXED)
    if graph:
        batch.graph(graph)
    batch.sweep(9)
    batch.sweep(3)
    for i, kw in enumerate(MIXED):
        alone = P.Sim(**kw)
        alone.sweep(12)
        assert np.array_equal(batch.export(i), alone.export()), i
        _rows_equal(batch.rows(i), alone.rows())


def test_inactive_instances_are_untouched_and_plain_sweeps_mix():
    batch = P.Batch(MIXED[:3])
    before = batch.export(1)
    batch.set_active(1, False)
    batch.sweep(4)
    assert np.array_equal(batch.export(1), before)
    batch.set_active(1, True)
    P.pmwa_sweep(batch.handles[1], 2)      # the plain path on one instance
    batch.sweep(2)
    alone = P.Sim(**MIXED[1])
    alone.sweep(4)
    assert np.array_equal(batch.export(1), alone.export())
    ref0 = P.Sim(**MIXED[0])
    ref0.sweep(6)
    assert np.array_equal(batch.export(0), ref0.export())


def test_batch_matches_oracle():
    kws = [MIXED[0], MIXED[2], MIXED[5]]
    batch = P.Batch(kws)
    batch.graph(2)
    batch.sweep(6)
    for i, kw in enumerate(kws):
        o = O.Oracle(**kw)
        o.sweep(6)
        assert np.array_equal(batch.export(i), o.export()), i


def test_tuned_replica_set_runs():
    """A slice of the 512-replica workload (autotuned domains, graph) runs
    and stays equal to one of its instances swept alone."""
    reps = A.replica_set(512)[:24]
    batch = P.Batch(reps)
    batch.graph(2)
    batch.sweep(4)
    alone = P.Sim(**reps[5])
    alone.sweep(4)
    assert np.array_equal(batch.export(5), alone.export())
    assert batch.last_ms() > 0
