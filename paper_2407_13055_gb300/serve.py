"""Served form: continuous batching of single HMult / HRot requests.

Requests arrive over time (a Poisson process in the benchmark). The host
scheduler admits a request as soon as (1) its arrival time has passed,
(2) an execution lane (a context clone with its own CUDA stream and scratch)
is free, and (3) the device memory the request holds while it runs (its
input and output ciphertexts and its lane's key-switching scratch,
ckks_request_bytes) fits in the admission budget next to the resident
evaluation keys and the requests already in flight; the budget is the
library's admission pool (ckks_pool_acquire refuses with CKKS_EBUSY).
Admitted requests run on their lane's stream, so the work of several
requests overlaps on the GPU; requests that arrive meanwhile are admitted as
lanes and memory free up. Completion is detected by polling a CUDA event per
request; latency is completion minus arrival on the host clock.

With one lane this is the plain one-operation-at-a-time server.
"""
from __future__ import annotations

import collections
import time
from dataclasses import dataclass, field


@dataclass
class Request:
    rid: int
    op: str            # "hmult" (with rescaling) or "hrot"
    level: int
    rot: int = 0       # rotation distance (hrot)
    arrival: float = 0.0


@dataclass
class Done:
    rid: int
    arrival: float
    start: float
    end: float
    lane: int


@dataclass
class _Slot:
    req: Request | None = None
    event: object = None
    start: float = 0.0
    bytes: int = 0


def poisson_arrivals(rng, count: int, rate: float):
    """Arrival times (seconds) of a Poisson process of the given rate."""
    t, out = 0.0, []
    for _ in range(count):
        t += rng.exponential(1.0 / rate)
        out.append(t)
    return out


@dataclass
class Server:
    """Continuous-batching server over `lanes` execution lanes of `ctx`."""
    K: object
    ctx: object
    lanes: int
    budget_bytes: int
    n: int                       # ring degree N
    resident_bytes: int = 0      # evaluation keys kept on the device, charged for the server's lifetime
    _streams: list = field(default_factory=list)
    _ctxs: list = field(default_factory=list)
    _pool: object = None

    def __post_init__(self):
        import torch
        self._pool = self.K.ckks_pool_create(self.budget_bytes)
        if not self.K.ckks_pool_acquire(self._pool, self.resident_bytes):
            self.K.ckks_pool_destroy(self._pool)
            self._pool = None
            raise ValueError(f"resident bytes {self.resident_bytes} exceed the admission budget {self.budget_bytes}")
        self._streams = [torch.cuda.Stream() for _ in range(self.lanes)]
        self._ctxs = [self.K.ckks_ctx_clone(self.ctx, s.cuda_stream) for s in self._streams]

    def close(self):
        for c in self._ctxs:
            self.K.ckks_ctx_destroy(c)
        self._ctxs = []
        if self._pool is not None:
            self.K.ckks_pool_destroy(self._pool)
            self._pool = None

    def footprint(self, req: Request) -> int:
        op = self.K.CKKS_OP_HMULT if req.op == "hmult" else self.K.CKKS_OP_HROT
        return self.K.ckks_request_bytes(self.ctx, op, req.level)

    def run(self, requests, inputs_for, key_for, out_for):
        """Serve `requests` (sorted by arrival). inputs_for(req) -> (a, b)
        ciphertext handles (b ignored for hrot); key_for(req) -> evk handle;
        out_for(req, lane) -> output ciphertext handle. Returns Done records
        in completion order."""
        import torch
        K = self.K
        pending = collections.deque(sorted(requests, key=lambda r: r.arrival))
        slots = [_Slot() for _ in range(self.lanes)]
        inflight = 0
        done = []
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        while pending or any(s.req for s in slots):
            now = time.perf_counter() - t0
            for li, s in enumerate(slots):
                if s.req is not None and s.event.query():
                    done.append(Done(s.req.rid, s.req.arrival, s.start, now, li))
                    inflight -= s.bytes
                    K.ckks_pool_release(self._pool, s.bytes)
                    slots[li] = _Slot()
            while pending and pending[0].arrival <= now:
                req = pending[0]
                need = self.footprint(req)
                if need > self.budget_bytes - self.resident_bytes:
                    raise ValueError(f"request {req.rid} needs {need} bytes, more than the budget leaves "
                                     f"({self.budget_bytes} - {self.resident_bytes} resident)")
                free = [li for li, s in enumerate(slots) if s.req is None]
                if not free or not K.ckks_pool_acquire(self._pool, need):
                    break
                pending.popleft()
                li = free[0]
                lane = self._ctxs[li]
                a, b = inputs_for(req)
                out = out_for(req, li)
                if req.op == "hmult":
                    K.ckks_hmult(lane, a, b, key_for(req), K.CKKS_RESCALE, out)
                else:
                    K.ckks_hrot(lane, a, req.rot, key_for(req), out)
                ev = torch.cuda.Event()
                ev.record(self._streams[li])
                slots[li] = _Slot(req, ev, now, need)
                inflight += need
        return done


def latency_stats(done):
    import numpy as np
    lat = np.array([d.end - d.arrival for d in done])
    span = max(d.end for d in done) - min(d.arrival for d in done)
    return {
        "completed": len(done),
        "throughput_ops_s": len(done) / span if span > 0 else None,
        "p50_ms": float(np.percentile(lat, 50) * 1e3),
        "p99_ms": float(np.percentile(lat, 99) * 1e3),
        "mean_ms": float(lat.mean() * 1e3),
    }
