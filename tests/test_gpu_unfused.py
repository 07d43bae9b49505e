"""Unfused one-step-per-launch form (CKKS_LAUNCH_UNFUSED, the mechanism
baseline of the fusion ablation): HMult with and without rescaling, HRot and
HConj equal the oracle bit for bit, i.e. the same residues as the fused
pipeline; the forms it does not cover are refused."""
import numpy as np
import pytest

from paper_2407_13055_gb300 import inputs

pytestmark = pytest.mark.gpu

PARAMS = {"n16d3": (16, 40, 3, 14), "toyT1": (12, 4, 4, 1), "toyT2": (12, 4, 1, 4), "tiny": (8, 6, 3, 2)}
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


@pytest.mark.parametrize("name,n_q", [("n16d3", 40), ("n16d3", 21), ("n16d3", 2), ("n16d3", 15), ("toyT1", 4),
                                      ("toyT2", 4), ("tiny", 6), ("tiny", 3)])
def test_unfused_form_matches_oracle(K, O, name, n_q):
    ctx, P = get(K, O, name)
    c1, c2 = rand_ct(P, n_q, 801), rand_ct(P, n_q, 803)
    evk, rk = rand_evk(P, 805), rand_evk(P, 807)
    k, kc = O.rot_k(1, P.log_n), O.conj_k(P.log_n)
    a = K.ckks_ct_import(ctx, c1, n_q - 1, 2.0**30)
    b = K.ckks_ct_import(ctx, c2, n_q - 1, 2.0**30)
    ek = K.ckks_evk_import(ctx, evk, 0)
    er = K.ckks_evk_import(ctx, rk, k)
    ec = K.ckks_evk_import(ctx, rk, kc)
    out = K.ckks_ct_create(ctx, n_q - 1)
    K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL | K.CKKS_LAUNCH_UNFUSED)
    try:
        if n_q > 1:
            K.ckks_hmult(ctx, a, b, ek, K.CKKS_RESCALE, out)
            got, level, _ = K.ckks_ct_export(ctx, out, P.n)
            assert level == n_q - 2 and np.array_equal(got, O.hmult(P, c1, c2, evk, rescale=True))
            with pytest.raises(K.CkksError):
                K.ckks_hmult(ctx, a, b, ek, K.CKKS_RESCALE_MERGED, out)
        K.ckks_hmult(ctx, a, b, ek, 0, out)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.hmult(P, c1, c2, evk, rescale=False))
        K.ckks_hrot(ctx, a, 1, er, out)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.hrot(P, c1, k, rk))
        K.ckks_hconj(ctx, a, ec, out)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.hrot(P, c1, kc, rk))
    finally:
        K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL)
        for h in (a, b, ek, er, ec, out):
            K.ckks_free(h)


def test_unfused_flag_refused_with_level_windows(K, O):
    q, p, levels = K.ckks_gen_prime_system_2530(12, 5)
    ctx = K.ckks_ctx_create(12, q, p, 3, scale=2.0**40, levels=levels)
    try:
        with pytest.raises(K.CkksError) as e:
            K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_UNFUSED)
        assert e.value.code == K.CKKS_EINVAL
    finally:
        K.ckks_ctx_destroy(ctx)
