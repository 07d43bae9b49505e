"""Served form: continuous batching of single HMult / HRot requests.

Requests arrive over time (a Poisson process in the benchmark). The
library's serving loop (ckks_serve_run, native, on the calling thread)
admits a request as soon as (1) its arrival time has passed, (2) an
execution lane (a context clone with its own CUDA stream and scratch) is
idle, and (3) the device memory the request holds while it runs (its input
and output ciphertexts and its lane's key-switching scratch,
ckks_request_bytes) fits in the admission pool next to the resident
evaluation keys and the requests already in flight. Admitted requests run on
their lane's stream, so the work of several requests overlaps on the GPU;
requests that arrive meanwhile are admitted as lanes and memory free up.
Completion is a CUDA event per request polled by the loop; latency is
completion minus arrival on the host's steady clock.

With one lane this is the plain one-operation-at-a-time server.
"""
from __future__ import annotations

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

    def run(self, requests, inputs_for, key_for, out_for=None, lane_outs=None):
        """Serve `requests` in arrival order. inputs_for(req) -> (a, b)
        ciphertext handles (b ignored for hrot); key_for(req) -> evk handle;
        out_for(req) -> the request's output ciphertext, or lane_outs: one
        output ciphertext per lane that every request on that lane writes.
        Returns Done records in completion order."""
        import torch
        K = self.K
        reqs = sorted(requests, key=lambda r: r.arrival)
        native = []
        for r in reqs:   # a request larger than the budget leaves is refused (CKKS_EINVAL)
            a, b = inputs_for(r)
            native.append(dict(op=K.CKKS_OP_HMULT if r.op == "hmult" else K.CKKS_OP_HROT, r=r.rot,
                               arrival=r.arrival, a=a, b=b if r.op == "hmult" else None, evk=key_for(r),
                               out=out_for(r) if out_for is not None else None, bytes=self.footprint(r)))
        torch.cuda.synchronize()
        times, order = K.ckks_serve_run(self._ctxs, self._pool, native, lane_outs=lane_outs)
        return [Done(reqs[i].rid, reqs[i].arrival, times[i][0], times[i][1], times[i][2]) for i in order]


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
