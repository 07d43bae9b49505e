"""Stage-major batched form with one persistent kernel (CKKS_BATCH_PERSISTENT):
every operation's ModUp on its lane, ONE persistent launch for the KeyMult +
MAC of all key switches and every element-wise operation (work items from a
device queue, admitted operations only), then the ModDown tails. Outputs at
mixed levels equal the oracle's bit for bit, direct and as a CUDA graph, on
one and on several lanes; an operation that is never admitted makes the
bounded admission wait expire (CKKS_ETIMEOUT) and the batch works again
afterwards; operations admitted while the kernel runs are picked up."""
import numpy as np
import pytest

from paper_2407_13055_gb300 import inputs

pytestmark = pytest.mark.gpu

PARAMS = {
    "n16d3": (16, 40, 3, 14),
    "toyT1": (12, 4, 4, 1),
}
_ctx = {}


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2407_13055_gb300 import ckks
    yield ckks
    for ctx, _ in _ctx.values():
        ckks.ckks_ctx_destroy(ctx)
    _ctx.clear()


def get(K, O, name):
    if name not in _ctx:
        log_n, L, dnum, alpha = PARAMS[name]
        P = O.make_params(log_n, L, dnum, alpha)
        _ctx[name] = (K.ckks_ctx_create(log_n, P.q, P.p, dnum, scale=2.0**30), P)
    return _ctx[name]


def rand_ct(P, n_q, seed):
    return np.stack([inputs.uniform_residues(seed, P.q[:n_q], P.n, s) for s in (0, 1)])


def rand_evk(P, seed):
    allp = P.all_primes()
    return np.stack([np.stack([inputs.uniform_residues(seed, allp, P.n, 10 * j + t) for t in range(2)])
                     for j in range(P.dnum)])


def mixed_batch(K, O, ctx, P, seed, count, max_level):
    """Independent operations of every kind at levels drawn from 1..max_level."""
    rng = np.random.default_rng(seed)
    relin, rotk = rand_evk(P, seed + 1), rand_evk(P, seed + 2)
    k1, kc = O.rot_k(1, P.log_n), O.conj_k(P.log_n)
    ek_r = K.ckks_evk_import(ctx, relin, 0)
    ek_g = K.ckks_evk_import(ctx, rotk, k1)
    ek_c = K.ckks_evk_import(ctx, rotk, kc)
    kinds = ["hmult_rs", "hrot", "pmult", "hadd", "hmult", "hconj", "rescale", "padd", "hmult_merged"]
    handles, ops, want = [ek_r, ek_g, ek_c], [], []
    for i in range(count):
        kind = kinds[i % len(kinds)]
        n_q = int(rng.integers(2, max_level + 2))
        a = rand_ct(P, n_q, seed + 100 + i)
        ha = K.ckks_ct_import(ctx, a, n_q - 1, 2.0**30)
        out = K.ckks_ct_create(ctx, n_q - 1)
        handles += [ha, out]
        if kind in ("hmult_rs", "hmult", "hadd", "hmult_merged"):
            b = rand_ct(P, n_q, seed + 200 + i)
            hb = K.ckks_ct_import(ctx, b, n_q - 1, 2.0**30)
            handles.append(hb)
            if kind == "hadd":
                ops.append(dict(op=K.CKKS_OP_HADD, a=ha, b=hb, out=out))
                want.append(O.hadd(a, b, P.q[:n_q]))
            elif kind == "hmult_merged":
                ops.append(dict(op=K.CKKS_OP_HMULT, a=ha, b=hb, evk=ek_r, flags=K.CKKS_RESCALE_MERGED, out=out))
                want.append(O.hmult_merged(P, a, b, relin))
            else:
                rs = kind == "hmult_rs"
                ops.append(dict(op=K.CKKS_OP_HMULT, a=ha, b=hb, evk=ek_r, flags=K.CKKS_RESCALE if rs else 0, out=out))
                want.append(O.hmult(P, a, b, relin, rescale=rs))
        elif kind == "hrot":
            ops.append(dict(op=K.CKKS_OP_HROT, a=ha, r=1, evk=ek_g, out=out))
            want.append(O.hrot(P, a, k1, rotk))
        elif kind == "hconj":
            ops.append(dict(op=K.CKKS_OP_HCONJ, a=ha, evk=ek_c, out=out))
            want.append(O.hrot(P, a, kc, rotk))
        elif kind in ("pmult", "padd"):
            pt = inputs.uniform_residues(seed + 300 + i, P.q[:n_q], P.n, 0)
            hp = K.ckks_pt_import(ctx, pt, n_q - 1, 2.0**30)
            handles.append(hp)
            if kind == "pmult":
                ops.append(dict(op=K.CKKS_OP_PMULT, a=ha, pt=hp, out=out))
                want.append(O.pmult(a, pt, P.q[:n_q]))
            else:
                ops.append(dict(op=K.CKKS_OP_PADD, a=ha, pt=hp, out=out))
                want.append(O.hadd(a, np.stack([pt, np.zeros_like(pt)]), P.q[:n_q]))
        else:
            ops.append(dict(op=K.CKKS_OP_RESCALE, a=ha, out=out))
            want.append(O.rescale(a, P.q[:n_q]))
    return ops, want, handles


def check_outputs(K, ctx, P, ops, want):
    for i, (o, w) in enumerate(zip(ops, want)):
        assert np.array_equal(K.ckks_ct_export(ctx, o["out"], P.n)[0], w), i


@pytest.mark.parametrize("name,lanes,graph", [("n16d3", 1, False), ("n16d3", 3, False), ("n16d3", 4, True),
                                              ("toyT1", 2, True)])
def test_persistent_batch_matches_oracle(K, O, name, lanes, graph):
    ctx, P = get(K, O, name)
    ops, want, handles = mixed_batch(K, O, ctx, P, 701, 12, min(P.L - 1, 39) if name == "toyT1" else 12)
    mode = K.CKKS_BATCH_PERSISTENT | (K.CKKS_BATCH_GRAPH if graph else 0)
    batch = K.ckks_batch_create(ctx, ops, lanes, mode)
    try:
        for _ in range(2):
            K.ckks_batch_run(ctx, batch)
            K.ckks_sync(ctx)
            check_outputs(K, ctx, P, ops, want)
    finally:
        K.ckks_batch_destroy(batch)
        for h in handles:
            K.ckks_free(h)


def test_persistent_batch_withheld_operation_times_out(K, O):
    """The last operation is never admitted: its KeyMult items wait for
    admission until the (shortened) wait limit expires; the kernel stops,
    the next synchronizing call returns CKKS_ETIMEOUT once, and a full run of
    the same batch afterwards is exact."""
    ctx, P = get(K, O, "n16d3")
    ops, want, handles = mixed_batch(K, O, ctx, P, 711, 6, 10)
    assert ops[-1]["op"] in (K.CKKS_OP_HMULT, K.CKKS_OP_HROT, K.CKKS_OP_HCONJ, K.CKKS_OP_PMULT, K.CKKS_OP_HADD)
    K.ckks_set_wait_limit(ctx, 2_000_000)  # about a millisecond; the lanes inherit it
    batch = K.ckks_batch_create(ctx, ops, 2, K.CKKS_BATCH_PERSISTENT | K.CKKS_BATCH_GRAPH)
    try:
        K.ckks_batch_run_admit(ctx, batch, len(ops) - 1)
        with pytest.raises(K.CkksError) as e:
            K.ckks_sync(ctx)
        assert e.value.code == K.CKKS_ETIMEOUT
        K.ckks_sync(ctx)
        K.ckks_batch_run(ctx, batch)
        K.ckks_sync(ctx)
        check_outputs(K, ctx, P, ops, want)
        with pytest.raises(K.CkksError):
            K.ckks_batch_admit(ctx, batch, 0)  # admission never shrinks
        with pytest.raises(K.CkksError):
            K.ckks_batch_run_admit(ctx, batch, len(ops) + 1)
    finally:
        K.ckks_batch_destroy(batch)
        K.ckks_set_wait_limit(ctx, 1 << 32)
        for h in handles:
            K.ckks_free(h)


def test_persistent_batch_admits_while_running(K, O):
    """Launched with nothing admitted, then every operation admitted from the
    host while the kernel runs: the waiting items pick the admission up and
    every output equals the oracle's."""
    ctx, P = get(K, O, "n16d3")
    ops, want, handles = mixed_batch(K, O, ctx, P, 721, 9, 20)
    batch = K.ckks_batch_create(ctx, ops, 3, K.CKKS_BATCH_PERSISTENT | K.CKKS_BATCH_GRAPH)
    try:
        K.ckks_batch_run_admit(ctx, batch, 0)
        for k in range(1, len(ops) + 1):
            K.ckks_batch_admit(ctx, batch, k)
        K.ckks_sync(ctx)
        check_outputs(K, ctx, P, ops, want)
        with pytest.raises(K.CkksError):
            K.ckks_batch_run_admit(ctx, None, 0)
    finally:
        K.ckks_batch_destroy(batch)
        for h in handles:
            K.ckks_free(h)


def test_admission_calls_need_a_persistent_batch(K, O):
    ctx, P = get(K, O, "toyT1")
    a = K.ckks_ct_import(ctx, rand_ct(P, 3, 731), 2, 2.0**30)
    b = K.ckks_ct_import(ctx, rand_ct(P, 3, 732), 2, 2.0**30)
    out = K.ckks_ct_create(ctx, 2)
    batch = K.ckks_batch_create(ctx, [dict(op=K.CKKS_OP_HADD, a=a, b=b, out=out)], 1, True)
    try:
        with pytest.raises(K.CkksError):
            K.ckks_batch_run_admit(ctx, batch, 1)
        with pytest.raises(K.CkksError):
            K.ckks_batch_admit(ctx, batch, 1)
        with pytest.raises(K.CkksError):
            K.ckks_batch_create(ctx, [dict(op=K.CKKS_OP_HADD, a=a, b=b, out=out)], 1, 4)  # unknown mode flag
    finally:
        K.ckks_batch_destroy(batch)
        for h in (a, b, out):
            K.ckks_free(h)
