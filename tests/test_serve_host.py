"""Host-side logic of the request loop (no GPU): percentiles and request bookkeeping."""
import pytest

from paper_2602_09527_gb300 import serve


def test_percentile_interpolates_order_statistics():
    v = [5.0, 1.0, 3.0, 2.0, 4.0]
    assert serve.percentile(v, 0) == 1.0
    assert serve.percentile(v, 100) == 5.0
    assert serve.percentile(v, 50) == 3.0
    assert serve.percentile(v, 25) == 2.0
    assert serve.percentile([1.0, 2.0], 50) == pytest.approx(1.5)
    assert serve.percentile([], 50) != serve.percentile([], 50)   # NaN


def test_request_defaults():
    r = serve.Request(key=1, b=None, arrival=0.5, alpha=0.01, gamma=1.0, seed=3)
    assert r.admitted is None and r.finished is None and r.n_subsets == 0 and r.storage == "FP32"


class _FakeBatch:
    """Stands in for the device batch: a job finishes after max_iters ticks."""
    live = []

    def __init__(self, graphs=True, **kw):
        self.left, self.next_id, self.running_max = {}, 0, 0
        _FakeBatch.live.append(self)

    def submit(self, g, b, *, max_iters, x_out, **kw):
        jid = self.next_id
        self.next_id += 1
        self.left[jid] = max_iters
        self.running_max = max(self.running_max, sum(v > 0 for v in self.left.values()))
        return jid

    def step(self, ticks=1):
        for j in self.left:
            self.left[j] = max(0, self.left[j] - ticks)
        return sum(v > 0 for v in self.left.values())

    def poll(self, jid):
        done = self.left[jid] == 0
        return done, ({"iterations": 1} if done else None)

    def release(self, jid):
        del self.left[jid]

    def close(self):
        pass


class _G:
    def __init__(self, n, nbytes):
        self.n, self.nbytes = n, nbytes


@pytest.fixture
def fake_engine(monkeypatch):
    import torch
    from paper_2602_09527_gb300 import _binding as vb
    _FakeBatch.live = []
    monkeypatch.setattr(vb, "Batch", _FakeBatch)
    monkeypatch.setattr(vb, "job_footprint", lambda g, max_iters, storage="FP32": g.nbytes)
    return torch


def _reqs(torch, keys, iters):
    return [serve.Request(key=k, b=torch.zeros(4), arrival=0.0, alpha=0.01, gamma=1.0, seed=i, max_iters=it)
            for i, (k, it) in enumerate(zip(keys, iters))]


def test_admission_by_footprint_and_handles(fake_engine):
    """Admission in arrival order while a handle of the request's class is free and the summed
    footprint stays within the budget; memory and handles return when a job finishes."""
    torch = fake_engine
    pools = {"a": [_G(4, 100), _G(4, 100), _G(4, 100)], "b": [_G(4, 250)]}
    srv = serve.BatchServer(pools, budget_bytes=300, ticks_per_step=1)
    reqs = _reqs(torch, ["a", "a", "b", "a", "b", "a"], [3, 5, 2, 4, 1, 2])
    st = srv.run(reqs)
    assert st.completed == len(reqs)
    assert st.peak_bytes <= 300
    assert _FakeBatch.live[0].running_max <= 3
    assert all(r.admitted is not None and r.finished >= r.admitted for r in reqs)
    # arrival order within a class: a request is never admitted before an earlier one of its class
    for key in ("a", "b"):
        adm = [r.admitted for r in reqs if r.key == key]
        assert adm == sorted(adm)
    assert srv.used == 0 and len(srv.free["a"]) == 3 and len(srv.free["b"]) == 1


def test_single_job_larger_than_budget_still_runs(fake_engine):
    """A job whose footprint alone exceeds the budget is admitted when nothing else runs."""
    torch = fake_engine
    srv = serve.BatchServer({"big": [_G(4, 10_000)]}, budget_bytes=10, ticks_per_step=2)
    st = srv.run(_reqs(torch, ["big", "big"], [3, 3]))
    assert st.completed == 2 and st.peak_jobs == 1


def test_mixed_server_splits_and_merges(fake_engine):
    """2D and 3D requests go to two batch servers (the 3D one in a worker thread) sharing one
    clock; the merged statistics count every request."""
    torch = fake_engine
    srv = serve.MixedServer({"2d": [_G(4, 10), _G(4, 10)]}, {"3d": [_G(8, 10)]}, budget_bytes=100)
    reqs = _reqs(torch, ["2d", "3d", "2d", "3d", "2d"], [4, 6, 2, 3, 5])
    st = srv.run(reqs)
    srv.close()
    assert st.completed == 5 and len(st.latencies) == 5
    assert len(_FakeBatch.live) == 2
    assert sum(b.next_id for b in _FakeBatch.live) == 5
    assert all(r.finished is not None for r in reqs)


class _Clock:
    """Deterministic clock: every reading advances time by `dt` seconds."""

    def __init__(self, dt=0.001):
        self.t, self.dt = 0.0, dt

    def __call__(self):
        self.t += self.dt
        return self.t


def test_later_request_of_free_class_admitted_past_blocked_head(fake_engine):
    """The head request waits for a handle of its class (the only one is busy); a later request
    of another class with a free handle and room in the budget is admitted at once instead of
    queueing behind it."""
    torch = fake_engine
    pools = {"big": [_G(4, 100)], "small": [_G(4, 10)]}
    srv = serve.BatchServer(pools, budget_bytes=1000, ticks_per_step=1)
    reqs = _reqs(torch, ["big", "big", "small"], [50, 5, 3])
    st = srv.run(reqs, clock=_Clock())
    assert st.completed == 3
    first_big, second_big, small = reqs
    assert small.admitted < second_big.admitted          # went past the blocked head
    assert small.finished < first_big.finished
    assert second_big.admitted >= first_big.finished      # waited for the class's only handle


def test_request_waiting_for_memory_holds_later_ones(fake_engine):
    """Memory is shared: a request that does not fit the budget is not overtaken (no starvation
    of large jobs by a stream of small ones)."""
    torch = fake_engine
    pools = {"big": [_G(4, 600), _G(4, 600)], "small": [_G(4, 10), _G(4, 10)]}
    srv = serve.BatchServer(pools, budget_bytes=1000, ticks_per_step=1)
    reqs = _reqs(torch, ["big", "big", "small"], [20, 5, 3])
    st = srv.run(reqs, clock=_Clock())
    assert st.completed == 3
    _, second_big, small = reqs
    assert small.admitted >= second_big.admitted


def test_max_running_caps_concurrent_jobs(fake_engine):
    """With max_running the batch never holds more jobs at once, whatever handles and memory
    would allow; every request still completes."""
    torch = fake_engine
    pools = {"a": [_G(4, 1) for _ in range(8)]}
    srv = serve.BatchServer(pools, budget_bytes=10_000, ticks_per_step=1, max_running=3)
    st = srv.run(_reqs(torch, ["a"] * 10, [4, 2, 6, 3, 5, 1, 2, 3, 4, 5]), clock=_Clock())
    assert st.completed == 10 and st.peak_jobs == 3
    assert _FakeBatch.live[0].running_max == 3
