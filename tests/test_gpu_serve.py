"""Served form (continuous batching over execution lanes): every request's
result is the same alone and in the mix, bit for bit, and the scheduler
respects its admission budget."""
import numpy as np
import pytest

from paper_2407_13055_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2407_13055_gb300 import ckks
    return ckks


def test_results_same_alone_and_in_the_mix(K, O):
    from paper_2407_13055_gb300.serve import Request, Server, latency_stats
    log_n, L, dnum = 12, 8, 2
    P = O.make_params(log_n, L, dnum)
    ctx = K.ckks_ctx_create(log_n, P.q, P.p, dnum, scale=2.0**28)
    handles = []
    try:
        sk = K.ckks_keygen_secret(ctx, 1)
        rk = K.ckks_keygen_relin(ctx, sk, 2)
        rots = [1, 3, 7, 100]
        gks = {r: K.ckks_keygen_rot(ctx, sk, r, 10 + r) for r in rots}
        handles += [sk, rk] + list(gks.values())
        pool = {}
        for lv in range(1, L):
            pool[lv] = [K.ckks_encrypt(ctx, sk, K.ckks_encode(ctx, inputs.messages(30 + 2 * lv + t, P.n // 2), lv,
                                                               2.0**28), 40 + 2 * lv + t) for t in range(2)]
            handles += pool[lv]
        rng = np.random.default_rng(5)
        reqs = []
        for i in range(24):
            op = "hmult" if i % 2 == 0 else "hrot"
            reqs.append(Request(i, op, int(rng.integers(1, L)), rots[i % len(rots)] if op == "hrot" else 0, 0.0))
        outs = {r.rid: K.ckks_ct_create(ctx, L - 1) for r in reqs}
        alone = {r.rid: K.ckks_ct_create(ctx, L - 1) for r in reqs}
        handles += list(outs.values()) + list(alone.values())
        inputs_for = lambda r: (pool[r.level][0], pool[r.level][1])
        key_for = lambda r: rk if r.op == "hmult" else gks[r.rot]
        # in the mix: all arrive at once on three lanes; the budget holds the
        # resident keys and two top-level requests (inputs, output, lane
        # scratch), so the footprint check limits admission too
        keys = (len(gks) + 1) * P.dnum * 2 * (L + P.alpha) * P.n * 4
        top = K.ckks_request_bytes(ctx, K.CKKS_OP_HMULT, L - 1)
        assert top > 3 * 2 * L * P.n * 4  # more than the input and output ciphertexts: the lane scratch
        budget = keys + 2 * top
        srv = Server(K, ctx, 3, budget, P.n, resident_bytes=keys)
        try:
            done = srv.run(reqs, inputs_for, key_for, out_for=lambda r: outs[r.rid])
            fp = {r.rid: srv.footprint(r) for r in reqs}
        finally:
            srv.close()
        assert sorted(d.rid for d in done) == list(range(24))
        # the bytes held by admitted requests never exceeded the budget, and
        # requests did overlap (more than one in flight at some point)
        events = sorted([(d.start, 1, d.rid) for d in done] + [(d.end, -1, d.rid) for d in done],
                        key=lambda e: (e[0], e[1]))
        live = peak = count = max_count = 0
        for _, delta, rid in events:
            live += delta * fp[rid]
            count += delta
            peak = max(peak, live)
            max_count = max(max_count, count)
        assert keys + peak <= budget and max_count >= 2
        stats = latency_stats(done)
        assert stats["completed"] == 24 and stats["p99_ms"] >= stats["p50_ms"] > 0
        # alone: one request at a time on the context itself
        for r in reqs:
            a, b = inputs_for(r)
            if r.op == "hmult":
                K.ckks_hmult(ctx, a, b, rk, K.CKKS_RESCALE, alone[r.rid])
            else:
                K.ckks_hrot(ctx, a, r.rot, gks[r.rot], alone[r.rid])
            K.ckks_sync(ctx)
        for r in reqs:
            x = K.ckks_ct_export(ctx, outs[r.rid], P.n)
            y = K.ckks_ct_export(ctx, alone[r.rid], P.n)
            assert x[1] == y[1] and np.array_equal(x[0], y[0]), r
    finally:
        for h in handles:
            K.ckks_free(h)
        K.ckks_ctx_destroy(ctx)


def test_memory_limit_refuses_allocations_with_enomem(K, O):
    """Admission by memory footprint on the device side: with a limit on the
    bytes a context's objects may hold (shared with its clones), an
    allocation beyond it fails with CKKS_ENOMEM before any CUDA allocation,
    freeing an object makes room again, and the request footprint the
    server admits by covers inputs, output and the lane's scratch."""
    import torch
    log_n, L, dnum = 12, 4, 4
    P = O.make_params(log_n, L, dnum, 1)
    ctx = K.ckks_ctx_create(log_n, P.q, P.p, dnum, scale=2.0**28)
    lane = K.ckks_ctx_clone(ctx, torch.cuda.Stream().cuda_stream)
    held = []
    try:
        base = K.ckks_memory_in_use(ctx)
        held.append(K.ckks_ct_create(ctx, L - 1))
        one = K.ckks_memory_in_use(ctx) - base
        assert one == 2 * L * P.n * 4
        K.ckks_set_memory_limit(ctx, base + one + one // 2)
        with pytest.raises(K.CkksError) as e:
            K.ckks_ct_create(ctx, L - 1)
        assert e.value.code == K.CKKS_ENOMEM
        with pytest.raises(K.CkksError) as e:
            K.ckks_ct_create(lane, L - 1)   # the clone shares the budget
        assert e.value.code == K.CKKS_ENOMEM
        assert K.ckks_memory_in_use(ctx) == base + one
        K.ckks_free(held.pop())
        assert K.ckks_memory_in_use(lane) == base
        held.append(K.ckks_ct_create(lane, L - 1))
        K.ckks_set_memory_limit(ctx, 0)
        held.append(K.ckks_ct_create(ctx, L - 1))
        ct = 2 * L * P.n * 4
        assert K.ckks_request_bytes(ctx, K.CKKS_OP_HMULT, L - 1) == 3 * ct + K.lib.ckks_ctx_device_bytes(lane)
        assert K.ckks_request_bytes(ctx, K.CKKS_OP_HADD, L - 1) == 3 * ct
        assert K.ckks_request_bytes(ctx, 99, L - 1) == 0
    finally:
        for h in held:
            K.ckks_free(h)
        K.ckks_ctx_destroy(lane)
        K.ckks_ctx_destroy(ctx)
