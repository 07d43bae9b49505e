"""Checked launch mode (CKKS_LAUNCH_CHECKED): every operation checks on the
device that its operands' residues lie below their primes, and its result
after it ran; imports check what they wrote. A residue out of range surfaces
as CKKS_ERANGE at the next synchronizing call and the context stays usable.
Out-of-range residues are data, never indices, so the unchecked kernels only
compute wrong values from them."""
import numpy as np
import pytest

from paper_2407_13055_gb300 import inputs

pytestmark = pytest.mark.gpu

PARAMS = {"toyT1": (12, 4, 4, 1), "n16d3": (16, 40, 3, 14)}
_cache = {}


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2407_13055_gb300 import ckks
    yield ckks
    for ctx, _ in _cache.values():
        ckks.ckks_set_launch_flags(ctx, ckks.CKKS_LAUNCH_PDL)
        ckks.ckks_ctx_destroy(ctx)
    _cache.clear()


def get(K, O, name):
    if name not in _cache:
        log_n, L, dnum, alpha = PARAMS[name]
        P = O.make_params(log_n, L, dnum, alpha)
        ctx = K.ckks_ctx_create(log_n, P.q, P.p, dnum, scale=2.0**30, secret_hw=192 if log_n == 16 else 0)
        _cache[name] = (ctx, P)
    return _cache[name]


def rand_ct(P, n_q, seed):
    return np.stack([inputs.uniform_residues(seed, P.q[:n_q], P.n, t) for t in range(2)])


def rand_evk(P, seed):
    allp = P.all_primes()
    return np.stack([np.stack([inputs.uniform_residues(seed, allp, P.n, 10 * j + t) for t in range(2)])
                     for j in range(P.dnum)])


def _set(K, ctx, checked):
    K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL | (K.CKKS_LAUNCH_CHECKED if checked else 0))


@pytest.mark.parametrize("name,n_q", [("toyT1", 4), ("n16d3", 5)])
def test_checked_mode_keeps_results(K, O, name, n_q):
    """With in-range operands the checked mode changes no residue and raises
    nothing: HMult + rescale, HRot, HAdd, PMult and rescale against the oracle."""
    ctx, P = get(K, O, name)
    c1, c2 = rand_ct(P, n_q, 501), rand_ct(P, n_q, 503)
    evk = rand_evk(P, 505)
    k = O.rot_k(1, P.log_n)
    pt = inputs.uniform_residues(507, P.q[:n_q], P.n, 0)
    _set(K, ctx, True)
    hs = []
    try:
        a = K.ckks_ct_import(ctx, c1, n_q - 1, 2.0**30)
        b = K.ckks_ct_import(ctx, c2, n_q - 1, 2.0**30)
        rk = K.ckks_evk_import(ctx, evk, 0)
        gk = K.ckks_evk_import(ctx, evk, k)
        p = K.ckks_pt_import(ctx, pt, n_q - 1, 2.0**30)
        out = K.ckks_ct_create(ctx, n_q - 1)
        hs += [a, b, rk, gk, p, out]
        K.ckks_hmult(ctx, a, b, rk, K.CKKS_RESCALE, out)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.hmult(P, c1, c2, evk, rescale=True))
        K.ckks_hrot(ctx, a, 1, gk, out)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.hrot(P, c1, k, evk))
        K.ckks_hadd(ctx, a, b, out)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.hadd(c1, c2, P.q[:n_q]))
        K.ckks_pmult(ctx, a, p, out)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.pmult(c1, pt, P.q[:n_q]))
        K.ckks_rescale(ctx, a, out)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.rescale(c1, P.q[:n_q]))
        K.ckks_sync(ctx)
    finally:
        _set(K, ctx, False)
        for h in hs:
            K.ckks_free(h)


def test_out_of_range_residue_raises_erange_and_the_context_recovers(K, O):
    ctx, P = get(K, O, "toyT1")
    n_q = 4
    c1, c2 = rand_ct(P, n_q, 511), rand_ct(P, n_q, 513)
    bad = c1.copy()
    bad[1, 2, 77] = P.q[2]            # one residue equal to its prime
    evk = rand_evk(P, 515)
    hs = []
    try:
        rk = K.ckks_evk_import(ctx, evk, 0)
        b = K.ckks_ct_import(ctx, c2, n_q - 1, 2.0**30)
        out = K.ckks_ct_create(ctx, n_q - 1)
        hs += [rk, b, out]
        # unchecked: the import and an operation on it raise nothing
        a_bad = K.ckks_ct_import(ctx, bad, n_q - 1, 2.0**30)
        hs.append(a_bad)
        K.ckks_hmult(ctx, a_bad, b, rk, K.CKKS_RESCALE, out)
        K.ckks_sync(ctx)
        _set(K, ctx, True)
        # checked: the import itself reports it
        with pytest.raises(K.CkksError) as e:
            K.ckks_ct_import(ctx, bad, n_q - 1, 2.0**30)
        assert e.value.code == K.CKKS_ERANGE
        # an operation on the operand imported unchecked reports it at the next sync
        K.ckks_hmult(ctx, a_bad, b, rk, K.CKKS_RESCALE, out)
        with pytest.raises(K.CkksError) as e:
            K.ckks_sync(ctx)
        assert e.value.code == K.CKKS_ERANGE
        # the mark was cleared: the context goes on with in-range operands
        a = K.ckks_ct_import(ctx, c1, n_q - 1, 2.0**30)
        hs.append(a)
        K.ckks_hmult(ctx, a, b, rk, K.CKKS_RESCALE, out)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.hmult(P, c1, c2, evk, rescale=True))
        # a key with an auxiliary-limb residue at its prime
        bad_evk = evk.copy()
        bad_evk[0, 1, P.L, 5] = P.p[0]
        with pytest.raises(K.CkksError) as e:
            K.ckks_evk_import(ctx, bad_evk, 0)
        assert e.value.code == K.CKKS_ERANGE
        K.ckks_sync(ctx)
    finally:
        _set(K, ctx, False)
        for h in hs:
            K.ckks_free(h)
