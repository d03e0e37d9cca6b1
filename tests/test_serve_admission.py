"""Host logic of the serving loop's admission (no GPU): first fit in arrival
order with a bounded number of pass-overs, so that small jobs are not held
back by a large one at the head of the queue and no job starves."""
from paper_1307_0328_gb300 import serve


class J:
    def __init__(self, name, fp):
        self.name, self.footprint = name, fp


def _names(js):
    return [j.name for j in js]


def test_first_fit_admits_small_jobs_behind_a_large_one():
    w = [J("big", 80), J("a", 10), J("b", 30), J("c", 5)]
    got = serve.admission(w, used=50, budget=100, slots=8, busy=True, max_bypass=3)
    assert _names(got) == ["a", "b", "c"]  # 50 + 10 + 30 + 5 <= 100; the 80 does not fit
    assert w[0].bypassed == 1


def test_slots_and_budget_are_respected():
    w = [J(str(i), 10) for i in range(10)]
    got = serve.admission(w, used=0, budget=45, slots=3, busy=False, max_bypass=3)
    assert _names(got) == ["0", "1", "2"]
    got = serve.admission(w, used=0, budget=45, slots=8, busy=False, max_bypass=3)
    assert _names(got) == ["0", "1", "2", "3"]


def test_a_job_passed_over_too_often_blocks_the_queue():
    big = J("big", 90)
    w = [big, J("a", 10), J("b", 10)]
    for k in range(3):
        got = serve.admission(w, used=50, budget=100, slots=8, busy=True, max_bypass=3)
        assert _names(got) == ["a", "b"], k
    got = serve.admission(w, used=50, budget=100, slots=8, busy=True, max_bypass=3)
    assert got == []  # the fourth pass-over exceeds the allowance: the head waits for memory
    got = serve.admission(w, used=0, budget=100, slots=8, busy=True, max_bypass=3)
    assert _names(got) == ["big", "a"]


def test_an_oversized_head_runs_alone_when_nothing_is_resident():
    w = [J("huge", 500), J("a", 10)]
    got = serve.admission(w, used=0, budget=100, slots=8, busy=False, max_bypass=3)
    assert _names(got) == ["huge"]
