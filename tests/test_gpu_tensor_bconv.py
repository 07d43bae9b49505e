"""Tensor-core BConv (Eq. 2 as an exact fp16 matrix product over byte planes,
tcgen05 kind::f16) inside the ModUp, ModDown and fused-rescale column kernels:
every tensor-core launch shape reproduces the oracle's HMult (with and
without rescaling), HRot and HConj bit for bit, on random and on extreme
residues; conversions with more than 16 sources fall back to the CUDA-core
kernels."""
import numpy as np
import pytest

from paper_2407_13055_gb300 import inputs

pytestmark = pytest.mark.gpu

# name: (log_n, L, dnum, alpha)
PARAMS = {
    "n16d3": (16, 40, 3, 14),
    "n16d5": (16, 40, 5, 8),
    "toyT1": (12, 4, 4, 1),
    "toyT2": (12, 4, 1, 4),
    "wide": (12, 20, 1, 20),    # 20 sources per conversion: above the tensor-core limit of 16
}
# (tc, sl, z, tp): tp = targets per MMA chunk
TC_SHAPES = [(8, 2, 1, 8), (8, 2, 1, 16), (8, 4, 1, 8), (8, 4, 1, 16),
             (4, 4, 1, 8), (4, 4, 1, 16), (4, 8, 1, 8), (4, 8, 1, 16)]

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


def set_shape(K, ctx, level, shape):
    for kern in (K.CKKS_COL_MODUP, K.CKKS_COL_MODDOWN, K.CKKS_COL_RS_FUSED):
        K.ckks_tune_set(ctx, kern, level, *shape)


def run_ops(K, O, ctx, P, c1, c2, evk, rk, k):
    """HMult + rescale (when the level allows), HMult, HRot(1) and HConj outputs."""
    n_q = c1.shape[1]
    a = K.ckks_ct_import(ctx, c1, n_q - 1, 2.0**30)
    b = K.ckks_ct_import(ctx, c2, n_q - 1, 2.0**30)
    ek = K.ckks_evk_import(ctx, evk, 0)
    er = K.ckks_evk_import(ctx, rk, k)
    ec = K.ckks_evk_import(ctx, rk, O.conj_k(P.log_n))
    out = K.ckks_ct_create(ctx, n_q - 1)
    res = {}
    try:
        if n_q > 1:
            K.ckks_hmult(ctx, a, b, ek, K.CKKS_RESCALE, out)
            res["hmult_rs"] = K.ckks_ct_export(ctx, out, P.n)[0]
        K.ckks_hmult(ctx, a, b, ek, 0, out)
        res["hmult"] = K.ckks_ct_export(ctx, out, P.n)[0]
        K.ckks_hrot(ctx, a, 1, er, out)
        res["hrot"] = K.ckks_ct_export(ctx, out, P.n)[0]
        K.ckks_hconj(ctx, a, ec, out)
        res["hconj"] = K.ckks_ct_export(ctx, out, P.n)[0]
    finally:
        for h in (a, b, ek, er, ec, out):
            K.ckks_free(h)
    return res


def oracle_ops(O, P, c1, c2, evk, rk, k):
    n_q = c1.shape[1]
    want = {}
    if n_q > 1:
        want["hmult_rs"] = O.hmult(P, c1, c2, evk, rescale=True)
    want["hmult"] = O.hmult(P, c1, c2, evk, rescale=False)
    want["hrot"] = O.hrot(P, c1, k, rk)
    want["hconj"] = O.hrot(P, c1, O.conj_k(P.log_n), rk)
    return want


@pytest.mark.parametrize("name,n_q", [("n16d3", 40), ("n16d3", 21), ("n16d3", 2), ("n16d5", 40), ("n16d5", 9),
                                      ("toyT1", 4), ("toyT2", 4), ("toyT2", 2), ("wide", 20)])
def test_tensor_core_shapes_match_oracle(K, O, name, n_q):
    ctx, P = get(K, O, name)
    c1, c2 = rand_ct(P, n_q, 601), rand_ct(P, n_q, 603)
    evk, rk = rand_evk(P, 605), rand_evk(P, 607)
    k = O.rot_k(1, P.log_n)
    want = oracle_ops(O, P, c1, c2, evk, rk, k)
    try:
        for shape in TC_SHAPES:
            set_shape(K, ctx, n_q - 1, shape)
            got = run_ops(K, O, ctx, P, c1, c2, evk, rk, k)
            for op in want:
                assert np.array_equal(got[op], want[op]), (shape, op)
    finally:
        set_shape(K, ctx, n_q - 1, (0, 4, 1, 1))


def _extreme_ct(P, n_q, kind, seed):
    q = P.q[:n_q].astype(np.uint64)[None, :, None]
    base = np.zeros((2, n_q, P.n), dtype=np.uint64)
    if kind == "q-1":
        v = base + q - 1
    elif kind == "half-":
        v = base + (q - 1) // 2
    elif kind == "half+":
        v = base + (q + 1) // 2
    else:  # alternating q - 1 and 0 along the coefficients, then random limbs mixed in
        v = np.where((np.arange(P.n) % 2 == 0)[None, None, :], base + q - 1, base)
        r = rand_ct(P, n_q, seed).astype(np.uint64)
        v[:, ::3, :] = r[:, ::3, :]
    return v.astype(np.uint32)


@pytest.mark.parametrize("kind", ["q-1", "half-", "half+", "mixed"])
def test_tensor_core_extreme_residues(K, O, kind):
    """Residues at q - 1 and (q +- 1) / 2 put the centered sources at their
    extremes (and, through the NTTs, spread extremes over the conversions):
    tensor-core and CUDA-core forms both equal the oracle."""
    ctx, P = get(K, O, "n16d3")
    n_q = 40
    c1, c2 = _extreme_ct(P, n_q, kind, 611), _extreme_ct(P, n_q, kind, 613)
    evk = rand_evk(P, 615)
    if kind == "q-1":
        allp = P.all_primes().astype(np.uint64)[None, None, :, None]
        evk = (np.zeros(evk.shape, dtype=np.uint64) + allp - 1).astype(np.uint32)
    k = O.rot_k(1, P.log_n)
    want = oracle_ops(O, P, c1, c2, evk, evk, k)
    try:
        for shape in [(8, 4, 1, 16), (4, 8, 1, 8), (0, 4, 1, 1)]:
            set_shape(K, ctx, n_q - 1, shape)
            got = run_ops(K, O, ctx, P, c1, c2, evk, evk, k)
            for op in want:
                assert np.array_equal(got[op], want[op]), (shape, op)
    finally:
        set_shape(K, ctx, n_q - 1, (0, 4, 1, 1))


def test_tensor_core_step_modup_and_moddown(K, O):
    """The step entry points (ModUp, ModUp + KeyMult, ModDown) run the tuned
    column kernels too: with a tensor-core shape they equal the oracle."""
    ctx, P = get(K, O, "n16d3")
    n_q = 40
    d = inputs.uniform_residues(621, P.q[:n_q], P.n, 0)
    acc = np.stack([inputs.uniform_residues(623, P.ext_primes(n_q), P.n, t) for t in (0, 1)])
    try:
        set_shape(K, ctx, n_q - 1, (8, 4, 1, 16))
        assert np.array_equal(K.ckks_step_modup(ctx, d, P.alpha), O.modup(P, d, n_q))
        assert np.array_equal(K.ckks_step_moddown(ctx, acc, n_q), O.moddown(P, acc, n_q))
    finally:
        set_shape(K, ctx, n_q - 1, (0, 4, 1, 1))


def test_tuner_with_tensor_shapes_keeps_results(K, O):
    """With CKKS_TUNE_TENSOR the fine-tuner also times the tensor-core shapes;
    whatever it records, the operations still equal the oracle."""
    ctx, P = get(K, O, "n16d3")
    n_q = 21
    K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL | K.CKKS_TUNE_TENSOR)
    try:
        K.ckks_tune(ctx, n_q - 1, 2)
        for kern in (K.CKKS_COL_MODUP, K.CKKS_COL_MODDOWN, K.CKKS_COL_RS_FUSED):
            tc, sl, z, tp, us = K.ckks_tune_get(ctx, kern, n_q - 1)
            assert tc in (4, 8) and tp in (1, 2, 8, 16) and us > 0
        c1, c2 = rand_ct(P, n_q, 641), rand_ct(P, n_q, 643)
        evk, rk = rand_evk(P, 645), rand_evk(P, 647)
        k = O.rot_k(1, P.log_n)
        want = oracle_ops(O, P, c1, c2, evk, rk, k)
        got = run_ops(K, O, ctx, P, c1, c2, evk, rk, k)
        for op in want:
            assert np.array_equal(got[op], want[op]), op
    finally:
        K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL)
        set_shape(K, ctx, n_q - 1, (0, 4, 1, 1))
        K.ckks_tune_set(ctx, K.CKKS_ROW_PASSES, n_q - 1, 0, 1, 1, 1)
