"""Host logic of the continuous-batching server on the CPU: the library's
native serving loop (ckks_serve_run) and admission pool with the device work
replaced by host hooks, behind serve.Server with fake streams and contexts:
admission in arrival order, at most one request per lane at a time, bytes in
flight within the admission budget, every request completed, refusals and
failures reported; latency statistics; Poisson arrivals."""
import numpy as np
import pytest

from paper_2407_13055_gb300 import serve


class FakeStream:
    _next = 1000

    def __init__(self):
        FakeStream._next += 1
        self.cuda_stream = FakeStream._next


class FakeK:
    """The library's admission pool and serving loop (ckks_serve_run, native)
    with the device work replaced by host hooks: a request "runs" until its
    lane has been polled three times. Contexts and streams are fakes;
    request footprints follow the library's rule (inputs + output
    ciphertexts + lane scratch)."""
    CKKS_RESCALE = 1
    CKKS_OP_HMULT, CKKS_OP_HROT = 1, 2
    SCRATCH = 5000

    def __init__(self, K, n=64):
        self.K = K
        self.calls = []
        self.n = n
        self.pools = []
        self.in_use_at_issue = []

    def ckks_request_bytes(self, ctx, op, level):
        ct = 2 * (level + 1) * self.n * 4
        return (3 if op == self.CKKS_OP_HMULT else 2) * ct + self.SCRATCH

    def ckks_pool_create(self, budget):
        h = self.K.ckks_pool_create(budget)
        self.pools.append(h)
        return h

    def ckks_pool_acquire(self, h, nbytes):
        return self.K.ckks_pool_acquire(h, nbytes)

    def ckks_pool_destroy(self, h):
        self.pools = [p for p in self.pools if p.value != h.value]
        self.K.ckks_pool_destroy(h)

    def ckks_ctx_clone(self, ctx, stream):
        return ("lane", stream)

    def ckks_ctx_destroy(self, c):
        pass

    def ckks_serve_run(self, lanes, pool, reqs, lane_outs=None):
        polls = {}

        def issue(i, lane):
            r = reqs[i]
            self.calls.append(("hmult" if r["op"] == self.CKKS_OP_HMULT else "hrot", lane, r["out"]))
            self.in_use_at_issue.append(self.K.ckks_pool_in_use(pool))
            polls[lane] = 0
            return 0

        def query(lane):
            polls[lane] += 1
            return 1 if polls[lane] >= 3 else 0

        bare = [dict(op=r["op"], r=r["r"], arrival=r["arrival"], bytes=r["bytes"]) for r in reqs]
        return self.K.ckks_serve_run(None, pool, bare, hooks=(issue, query), n_lanes=len(lanes))


@pytest.fixture
def K():
    from paper_2407_13055_gb300 import ckks
    return ckks


@pytest.fixture
def fake_cuda(monkeypatch):
    import torch
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)


@pytest.mark.parametrize("lanes,budget_reqs", [(1, 4), (3, 10), (4, 2)])
def test_admission_invariants(fake_cuda, K, lanes, budget_reqs):
    rng = np.random.default_rng(lanes)
    n = 64
    reqs = [serve.Request(i, "hmult" if i % 2 else "hrot", int(rng.integers(1, 40)), rot=1, arrival=0.0)
            for i in range(30)]
    F = FakeK(K, n)
    resident = 12345
    budget = resident + budget_reqs * F.ckks_request_bytes(None, F.CKKS_OP_HMULT, 39)
    srv = serve.Server(F, ctx="ctx", lanes=lanes, budget_bytes=budget, n=n, resident_bytes=resident)
    pool = srv._pool
    done = srv.run(reqs, inputs_for=lambda r: ("a", "b"), key_for=lambda r: "evk",
                   out_for=lambda r: ("out", r.rid))
    assert K.ckks_pool_in_use(pool) == resident  # every request released what it acquired
    assert max(F.in_use_at_issue) <= budget
    srv.close()
    assert not F.pools
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
    assert len(F.calls) == 30 and all(c[0] == by_id[c[2][1]].op for c in F.calls)
    # every lane takes part when the budget holds a request per lane
    used = {d.lane for d in done}
    assert used <= set(range(lanes)) and (budget_reqs < lanes or used == set(range(lanes)))


def test_resident_bytes_above_the_budget_are_refused(fake_cuda, K):
    F = FakeK(K)
    with pytest.raises(ValueError):
        serve.Server(F, ctx="ctx", lanes=2, budget_bytes=1000, n=64, resident_bytes=1001)
    assert not F.pools


def test_a_request_larger_than_the_budget_is_an_error(fake_cuda, K):
    """A request that could never be admitted is refused instead of waiting forever."""
    F = FakeK(K)
    srv = serve.Server(F, ctx="ctx", lanes=2, budget_bytes=1000, n=64)
    try:
        with pytest.raises(K.CkksError) as e:
            srv.run([serve.Request(0, "hmult", 3)], lambda r: ("a", "b"), lambda r: "evk", lambda r: "out")
        assert e.value.code == K.CKKS_EINVAL
        assert not F.calls
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


class Device:
    """Host stand-in for the lanes: request i runs for `polls[i]` polls of its
    lane; issue / query may be told to fail."""

    def __init__(self, polls, fail_issue=None, fail_query=None):
        self.polls, self.fail_issue, self.fail_query = polls, fail_issue, fail_query
        self.left, self.started = {}, []

    def issue(self, i, lane):
        if i == self.fail_issue:
            return -6
        self.left[lane] = (i, self.polls[i])
        self.started.append((i, lane))
        return 0

    def query(self, lane):
        i, n = self.left[lane]
        if i == self.fail_query:
            return -6
        self.left[lane] = (i, n - 1)
        return 1 if n <= 1 else 0


def _reqs(K, arrivals, nbytes=100):
    return [dict(op=K.CKKS_OP_HMULT if i % 2 else K.CKKS_OP_HROT, arrival=t, bytes=nbytes)
            for i, t in enumerate(arrivals)]


def test_native_loop_waits_for_arrivals_and_reports_completion_order(K):
    pool = K.ckks_pool_create(10 ** 6)
    try:
        arrivals = [0.0, 0.0, 0.002, 0.004, 0.004]
        dev = Device([50, 2, 2, 2, 2])
        done, order = K.ckks_serve_run(None, pool, _reqs(K, arrivals), hooks=(dev.issue, dev.query), n_lanes=2)
        for (start, end, lane), t in zip(done, arrivals):
            assert t <= start <= end and lane in (0, 1)
        assert sorted(order) == list(range(5))
        assert order.index(1) < order.index(0)  # the short request finished before the long one
        assert [i for i, _ in dev.started] == list(range(5))  # admitted in arrival order
        assert K.ckks_pool_in_use(pool) == 0
    finally:
        K.ckks_pool_destroy(pool)


def test_native_loop_refuses_bad_lists(K):
    pool = K.ckks_pool_create(1000)
    dev = Device([1] * 3)
    hooks = (dev.issue, dev.query)
    try:
        for reqs in (_reqs(K, [0.0, 0.2, 0.1]),                                     # not sorted by arrival
                     [dict(op=K.CKKS_OP_PMULT, arrival=0.0, bytes=1)],                 # not a served op
                     _reqs(K, [0.0], nbytes=1001)):                                   # can never be admitted
            with pytest.raises(K.CkksError) as e:
                K.ckks_serve_run(None, pool, reqs, hooks=hooks, n_lanes=2)
            assert e.value.code == K.CKKS_EINVAL
        assert not dev.started
        assert K.ckks_pool_acquire(pool, 600)   # resident bytes: what is left is the limit
        with pytest.raises(K.CkksError):
            K.ckks_serve_run(None, pool, _reqs(K, [0.0], nbytes=401), hooks=hooks, n_lanes=1)
        K.ckks_serve_run(None, pool, _reqs(K, [0.0], nbytes=400), hooks=hooks, n_lanes=1)
        assert K.ckks_pool_in_use(pool) == 600
    finally:
        K.ckks_pool_destroy(pool)


@pytest.mark.parametrize("where", ["issue", "query"])
def test_native_loop_stops_at_the_first_failure_after_draining(K, where):
    pool = K.ckks_pool_create(10 ** 6)
    try:
        dev = Device([3] * 8, fail_issue=4 if where == "issue" else None, fail_query=4 if where == "query" else None)
        with pytest.raises(K.CkksError) as e:
            K.ckks_serve_run(None, pool, _reqs(K, [0.0] * 8), hooks=(dev.issue, dev.query), n_lanes=2)
        assert e.value.code == -6
        assert K.ckks_pool_in_use(pool) == 0            # everything admitted was released
        assert max(i for i, _ in dev.started) == (3 if where == "issue" else 5)
    finally:
        K.ckks_pool_destroy(pool)
