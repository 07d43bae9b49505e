"""The 25-30 prime system on the GPU (Sec. 3.2, Table 2): levels are windows
of the prime list, rescaling is rational, one evaluation key serves every
level. Residues equal the oracle's bit for bit; a squaring chain through the
rescaling cycle decrypts within 1e-3."""
import math

import numpy as np
import pytest

from paper_2407_13055_gb300 import inputs

pytestmark = pytest.mark.gpu

_cache = {}


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2407_13055_gb300 import ckks
    yield ckks
    for ctx, _, _ in _cache.values():
        ckks.ckks_ctx_destroy(ctx)
    _cache.clear()


def system(K, O, log_n):
    if log_n not in _cache:
        P, levels = O.prime_system_2530(log_n, 5)
        ctx = K.ckks_ctx_create(log_n, P.q, P.p, P.dnum, scale=2.0**40, secret_hw=192 if log_n == 16 else 0,
                                levels=levels)
        _cache[log_n] = (ctx, P, levels)
    return _cache[log_n]


def rand_ct(P, lv, seed):
    s, n = lv
    primes = [int(v) for v in P.q[s:s + n]]
    return np.stack([inputs.uniform_residues(seed, primes, P.n, t) for t in range(2)])


def rand_evk(P, seed):
    allp = P.all_primes()
    return np.stack([np.stack([inputs.uniform_residues(seed, allp, P.n, 10 * j + t) for t in range(2)])
                     for j in range(P.dnum)])


@pytest.mark.parametrize("log_n", [12, 16])
@pytest.mark.parametrize("level", [1, 2, 3, 4, 5, 8])
def test_rational_rescale_matches_oracle(K, O, log_n, level):
    ctx, P, levels = system(K, O, log_n)
    (s0, n0), (s1, n1) = levels[level], levels[level - 1]
    c = rand_ct(P, levels[level], 300 + level)
    a = K.ckks_ct_import(ctx, c, level, 2.0**40)
    out = K.ckks_ct_create(ctx, level)
    try:
        K.ckks_rescale(ctx, a, out)
        got, lv, scale = K.ckks_ct_export(ctx, out, P.n)
        assert lv == level - 1
        assert np.array_equal(got, O.rescale_rational(P, c, s0, n0, s1, n1))
        drop = [int(P.q[g]) for g in range(s0, s0 + n0) if not s1 <= g < s1 + n1]
        add = [int(P.q[g]) for g in range(s1, s1 + n1) if not s0 <= g < s0 + n0]
        assert scale == pytest.approx(2.0**40 * math.prod(add) / math.prod(drop), rel=1e-12)
    finally:
        K.ckks_free(a)
        K.ckks_free(out)


@pytest.mark.parametrize("log_n", [12, 16])
@pytest.mark.parametrize("level", [0, 1, 2, 3, 4, 6, 8])
def test_hmult_hrot_at_windows_match_oracle(K, O, log_n, level):
    _check_hmult_hrot(K, O, log_n, level)


@pytest.mark.parametrize("level", [4, 8])
@pytest.mark.parametrize("passes", [2, 4, 6])
def test_row_forms_at_windows_match_oracle(K, O, level, passes):
    """The row-phase forms other than the default one (two passes, bulk-staged
    forward rows, twiddles in shared memory) at windows of the 25-30 system:
    the rational rescale's and the merged form's row epilogues included."""
    ctx, P, levels = system(K, O, 16)
    K.ckks_tune_set(ctx, K.CKKS_ROW_PASSES, level, passes, 1, 1, 1)
    try:
        _check_hmult_hrot(K, O, 16, level)
    finally:
        K.ckks_tune_set(ctx, K.CKKS_ROW_PASSES, level, 0, 1, 1, 1)


def _check_hmult_hrot(K, O, log_n, level):
    ctx, P, levels = system(K, O, log_n)
    s0, n0 = levels[level]
    c1, c2 = rand_ct(P, levels[level], 310 + level), rand_ct(P, levels[level], 320 + level)
    evk = rand_evk(P, 330)
    k = O.rot_k(3, P.log_n)
    a = K.ckks_ct_import(ctx, c1, level, 2.0**40)
    b = K.ckks_ct_import(ctx, c2, level, 2.0**40)
    rk = K.ckks_evk_import(ctx, evk, 0)
    gk = K.ckks_evk_import(ctx, evk, k)
    out = K.ckks_ct_create(ctx, level)
    try:
        K.ckks_hmult(ctx, a, b, rk, 0, out)
        want_m = O.hmult(P, c1, c2, evk, rescale=False, base=s0)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], want_m)
        K.ckks_hrot(ctx, a, 3, gk, out)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.hrot(P, c1, k, evk, base=s0))
        if level >= 1:
            K.ckks_hmult(ctx, a, b, rk, K.CKKS_RESCALE, out)
            s1, n1 = levels[level - 1]
            got, lv, _ = K.ckks_ct_export(ctx, out, P.n)
            assert lv == level - 1
            assert np.array_equal(got, O.rescale_rational(P, want_m, s0, n0, s1, n1))
            # ModDown merged into the rational rescaling (Sec. 6)
            K.ckks_hmult(ctx, a, b, rk, K.CKKS_RESCALE_MERGED, out)
            got, lv, _ = K.ckks_ct_export(ctx, out, P.n)
            assert lv == level - 1
            assert np.array_equal(got, O.hmult_merged(P, c1, c2, evk, base=s0, new=(s1, n1)))
    finally:
        for h in (a, b, rk, gk, out):
            K.ckks_free(h)


@pytest.mark.parametrize("level", [3, 7])
def test_hoisted_and_linear_transform_at_windows_match_oracle(K, O, level):
    ctx, P, levels = system(K, O, 12)
    s0, n0 = levels[level]
    c = rand_ct(P, levels[level], 340 + level)
    rs = [0, 1, 5]
    evks = [rand_evk(P, 350 + i) if r else None for i, r in enumerate(rs)]
    primes_ext = [int(v) for v in P.q[s0:s0 + n0]] + [int(v) for v in P.p]
    pts = [inputs.uniform_residues(360 + i, primes_ext, P.n, 7) for i in range(len(rs))]
    a = K.ckks_ct_import(ctx, c, level, 2.0**40)
    eks = [K.ckks_evk_import(ctx, e, O.rot_k(r, P.log_n)) if r else None for e, r in zip(evks, rs)]
    dps = [K.ckks_pt_import_ext(ctx, pt, level, 2.0**20) for pt in pts]
    outs = [K.ckks_ct_create(ctx, level) for _ in range(3)]
    try:
        K.ckks_hrot_hoisted(ctx, a, rs[1:], eks[1:], outs[:2])
        for r, e, o in zip(rs[1:], evks[1:], outs[:2]):
            assert np.array_equal(K.ckks_ct_export(ctx, o, P.n)[0], O.hrot(P, c, O.rot_k(r, P.log_n), e, base=s0))
        K.ckks_linear_transform(ctx, a, rs, eks, dps, outs[2])
        assert np.array_equal(K.ckks_ct_export(ctx, outs[2], P.n)[0],
                              O.linear_transform(P, c, rs, evks, pts, base=s0))
    finally:
        for h in [a] + [e for e in eks if e] + dps + outs:
            K.ckks_free(h)


@pytest.mark.parametrize("merged", [False, True])
@pytest.mark.parametrize("log_n", [12, 16])
def test_squaring_through_the_rescaling_cycle_decrypts(K, O, log_n, merged):
    """Library keys and encryption at level 4 (Delta = 2^40); HMult + rational
    rescaling (or ModDown merged into it, Sec. 6) down to level 0: each
    decryption is u^(2^k) within 1e-3 and the scale stays within 0.1 bits of
    2^40 (Sec. 3.2)."""
    ctx, P, levels = system(K, O, log_n)
    sk = K.ckks_keygen_secret(ctx, 21)
    rk = K.ckks_keygen_relin(ctx, sk, 22)
    gk = K.ckks_keygen_rot(ctx, sk, 5, 23)
    u = 0.9 * inputs.messages(24, P.n // 2)
    handles = [sk, rk, gk]
    try:
        pt = K.ckks_encode(ctx, u, 4, 2.0**40)
        ct = K.ckks_encrypt(ctx, sk, pt, 25)
        handles += [pt, ct]
        want = u.copy()
        for lv in range(4, 0, -1):
            out = K.ckks_ct_create(ctx, lv - 1)
            handles.append(out)
            K.ckks_hmult(ctx, ct, ct, rk, K.CKKS_RESCALE_MERGED if merged else K.CKKS_RESCALE, out)
            ct = out
            want = want * want
            _, scale = K.ckks_ct_info(ct)[:2]
            assert abs(math.log2(scale) - 40) < 0.1
            dec = K.ckks_decrypt(ctx, sk, ct)
            got = K.ckks_decode(ctx, dec, P.n // 2)
            K.ckks_free(dec)
            assert np.max(np.abs(got - want)) < 1e-3, lv
        # rotation at level 3 with the same (all-prime) key
        pt3 = K.ckks_encode(ctx, u, 3, 2.0**40)
        c3 = K.ckks_encrypt(ctx, sk, pt3, 26)
        r3 = K.ckks_ct_create(ctx, 3)
        handles += [pt3, c3, r3]
        K.ckks_hrot(ctx, c3, 5, gk, r3)
        dec = K.ckks_decrypt(ctx, sk, r3)
        got = K.ckks_decode(ctx, dec, P.n // 2)
        K.ckks_free(dec)
        assert np.max(np.abs(got - np.roll(u, -5))) < 1e-3
    finally:
        for h in handles:
            K.ckks_free(h)
