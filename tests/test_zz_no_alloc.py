"""The allocation-free rho-slice entry point (pmwa_rho_slices_static).

Some callers cannot allocate device memory while they run: a serving loop
whose GPU memory belongs to another framework's allocator, or one that has
promised its memory pool no new blocks.  pmwa_rho_slices_static gives them
the Supplement S-I worm density at equal-time slices with the device scratch
held in a fixed array inside the library instead of the caller's arena.  This
test calls it through the C ABI twice in a row and checks each result against
the arena-based pmwa_rho_slices, within the 1e-12 relative tolerance the
other FP64 parity tests use.  It lives in a file of its own, collected last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

import paper_1307_0328_gb300 as P  # noqa: E402


def test_static_scratch_rho_matches_arena_rho_twice():
    g = P.Sim(Lx=12, Ly=8, beta=3.0, eta=0.3, V=0.5, mu=0.2, dom_x=6, dom_y=4, sub_block=2,
              n_cycle=4, seed=21)
    N, K = 12 * 8, 6
    for call in range(2):
        g.sweep(2)
        want = P.pmwa_rho_slices(g.h, N, K)
        got = P.pmwa_rho_slices_static(g.h, N, K)
        assert got.shape == want.shape
        assert np.all(np.isfinite(got)), call
        assert np.allclose(got, want, rtol=1e-12, atol=0), call
    # after the calls above (the first one looked the array up), a call
    # changes neither the device's free memory nor torch's allocator
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st0 = torch.cuda.memory_stats()
    for _ in range(3):
        P.pmwa_rho_slices_static(g.h, N, K)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    st1 = torch.cuda.memory_stats()
    assert free1 == free0
    for k in ("allocated_bytes.all.current", "reserved_bytes.all.current", "num_alloc_retries"):
        assert st1.get(k, 0) == st0.get(k, 0), k
    # requests beyond the fixed size are refused with a clear status
    with pytest.raises(P.PmwaError) as e:
        P.pmwa_rho_slices_static(g.h, N, (1 << 20) // N + 1)
    assert e.value.status == P.PMWA_EINVAL
