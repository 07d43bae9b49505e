"""Host logic of the continuous-batching server (serve.py) on the CPU, with
fake CUDA streams/events and a fake library: admission in arrival order,
at most one request per lane at a time, in-flight output bytes within the
admission budget, every request completed; latency statistics; Poisson
arrivals."""
import numpy as np
import pytest

from paper_2407_13055_gb300 import serve


class FakeStream:
    _next = 1000

    def __init__(self):
        FakeStream._next += 1
        self.cuda_stream = FakeStream._next


class FakeEvent:
    """Completes after a few polls, like work that takes a while."""

    def __init__(self):
        self.polls = 0

    def record(self, stream):
        pass

    def query(self):
        self.polls += 1
        return self.polls >= 3


class FakeK:
    """Fake library: operations are recorded; request footprints follow the
    library's rule (inputs + output ciphertexts + lane scratch); the admission
    pool is a plain counter with the library's refusal rule."""
    CKKS_RESCALE = 1
    CKKS_OP_HMULT, CKKS_OP_HROT = 1, 2
    SCRATCH = 5000

    def __init__(self, n=64):
        self.calls = []
        self.n = n
        self.pools = {}

    def ckks_request_bytes(self, ctx, op, level):
        ct = 2 * (level + 1) * self.n * 4
        return (3 if op == self.CKKS_OP_HMULT else 2) * ct + self.SCRATCH

    def ckks_pool_create(self, budget):
        h = len(self.pools) + 1
        self.pools[h] = [budget, 0]
        return h

    def ckks_pool_acquire(self, h, nbytes):
        budget, used = self.pools[h]
        if used + nbytes > budget:
            return False
        self.pools[h][1] = used + nbytes
        return True

    def ckks_pool_release(self, h, nbytes):
        assert 0 <= nbytes <= self.pools[h][1]
        self.pools[h][1] -= nbytes

    def ckks_pool_destroy(self, h):
        del self.pools[h]

    def ckks_ctx_clone(self, ctx, stream):
        return ("lane", stream)

    def ckks_ctx_destroy(self, c):
        pass

    def ckks_hmult(self, lane, a, b, evk, flags, out):
        assert flags == self.CKKS_RESCALE
        self.calls.append(("hmult", lane, out))

    def ckks_hrot(self, lane, a, r, evk, out):
        self.calls.append(("hrot", lane, out))


@pytest.fixture
def fake_cuda(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)


@pytest.mark.parametrize("lanes,budget_reqs", [(1, 4), (3, 10), (4, 2)])
def test_admission_invariants(fake_cuda, lanes, budget_reqs):
    rng = np.random.default_rng(lanes)
    n = 64
    reqs = [serve.Request(i, "hmult" if i % 2 else "hrot", int(rng.integers(1, 40)), rot=1, arrival=0.0)
            for i in range(30)]
    K = FakeK(n)
    resident = 12345
    budget = resident + budget_reqs * K.ckks_request_bytes(None, K.CKKS_OP_HMULT, 39)
    srv = serve.Server(K, ctx="ctx", lanes=lanes, budget_bytes=budget, n=n, resident_bytes=resident)
    pool = srv._pool
    done = srv.run(reqs, inputs_for=lambda r: ("a", "b"), key_for=lambda r: "evk",
                   out_for=lambda r, li: ("out", r.rid))
    assert K.pools[pool][1] == resident  # every request released what it acquired
    srv.close()
    assert pool not in K.pools
    assert sorted(d.rid for d in done) == list(range(30))
    by_id = {r.rid: r for r in reqs}
    # admission in arrival order (ties: list order), each on a free lane
    starts = sorted(done, key=lambda d: d.start)
    assert [d.rid for d in sorted(done, key=lambda d: (d.start, d.rid))] == sorted(d.rid for d in starts)
    for li in range(lanes):
        spans = sorted((d.start, d.end) for d in done if d.lane == li)
        for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
            assert s1 >= e0
    # resident bytes plus the in-flight requests' footprints never exceed the budget
    for d in done:
        t = d.start
        held = sum(srv.footprint(by_id[x.rid]) for x in done if x.start <= t < x.end)
        assert resident + held <= srv.budget_bytes
    assert all(d.end >= d.start >= d.arrival for d in done)
    assert len(K.calls) == 30 and all(c[0] == by_id[c[2][1]].op for c in K.calls)


def test_resident_bytes_above_the_budget_are_refused(fake_cuda):
    K = FakeK()
    with pytest.raises(ValueError):
        serve.Server(K, ctx="ctx", lanes=2, budget_bytes=1000, n=64, resident_bytes=1001)
    assert not K.pools


def test_a_request_larger_than_the_budget_is_an_error(fake_cuda):
    """A request that could never be admitted raises instead of waiting forever."""
    K = FakeK()
    srv = serve.Server(K, ctx="ctx", lanes=2, budget_bytes=1000, n=64)
    try:
        with pytest.raises(ValueError):
            srv.run([serve.Request(0, "hmult", 3)], lambda r: ("a", "b"), lambda r: "evk", lambda r, li: "out")
    finally:
        srv.close()


def test_latency_stats():
    done = [serve.Done(i, arrival=0.0, start=0.0, end=(i + 1) * 1e-3, lane=0) for i in range(100)]
    st = serve.latency_stats(done)
    assert st["completed"] == 100
    assert st["p50_ms"] == pytest.approx(50.5)
    assert st["p99_ms"] == pytest.approx(99.01)
    assert st["throughput_ops_s"] == pytest.approx(100 / 0.1)


def test_poisson_arrivals_rate():
    rng = np.random.default_rng(5)
    t = serve.poisson_arrivals(rng, 20000, 250.0)
    gaps = np.diff([0.0] + t)
    assert np.all(gaps > 0)
    assert np.mean(gaps) == pytest.approx(1 / 250.0, rel=0.03)
