"""GPU parity: every step of the key-switch path through the C ABI, compared
element by element with the CPU oracle on the same seeded inputs. Integer
path: bit-exact. Decrypted slots: max-abs error <= 1e-3."""
import numpy as np
import pytest

from paper_2407_13055_gb300 import inputs

pytestmark = pytest.mark.gpu

# name: (log_n, L, dnum, alpha)
PARAMS = {
    "tiny": (8, 6, 3, 2),        # ragged digits {0,1} {2,3} {4,5}; N = 2^8
    "toyT1": (12, 4, 4, 1),      # toy configuration, one auxiliary prime, per-prime digits
    "toyT2": (12, 4, 1, 4),      # toy configuration, one digit, four auxiliary primes
    "n16d3": (16, 40, 3, 14),    # single-op configuration at N = 2^16, dnum = 3
}

_ctx_cache = {}


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2407_13055_gb300 import ckks
    yield ckks
    for ctx, _ in _ctx_cache.values():
        ckks.ckks_ctx_destroy(ctx)
    _ctx_cache.clear()


def get(K, O, name):
    if name not in _ctx_cache:
        log_n, L, dnum, alpha = PARAMS[name]
        P = O.make_params(log_n, L, dnum, alpha)
        ctx = K.ckks_ctx_create(log_n, P.q, P.p, dnum, scale=2.0**30, secret_hw=192 if log_n == 16 else 0)
        _ctx_cache[name] = (ctx, P)
    return _ctx_cache[name]


def rand_poly(P, primes, seed, stream=0):
    return inputs.uniform_residues(seed, primes, P.n, stream)


def rand_ct(P, n_q, seed, stream=0):
    return np.stack([rand_poly(P, P.q[:n_q], seed, stream), rand_poly(P, P.q[:n_q], seed, stream + 1)])


def rand_evk(P, seed):
    allp = P.all_primes()
    return np.stack([np.stack([rand_poly(P, allp, seed, 10 * j + t) for t in range(2)]) for j in range(P.dnum)])


# ---------------------------------------------------------------- a1: SMR ---

def test_smr_matches_oracle(K, O):
    ctx, P = get(K, O, "toyT1")
    rng = np.random.default_rng(0)
    for pid in (0, 1, P.L):
        q = int(P.all_primes()[pid])
        lo, hi = -q * 2**31, q * 2**31 - 1
        x = np.concatenate([[lo, hi, 0, -1, 1], rng.integers(lo, hi, 20000, dtype=np.int64)]).astype(np.int64)
        y = K.ckks_step_smr(ctx, x, pid)
        want = np.array([O.smr(int(v), q) for v in x[:2000]], np.int32)
        assert np.array_equal(y[:2000], want)
        assert np.all(np.abs(y.astype(np.int64)) < q)
        assert np.all(((y.astype(object) * 2**32 - x.astype(object)) % q) == 0)


# ---------------------------------------------------------------- a2: NTT ---

@pytest.mark.parametrize("name", ["tiny", "toyT1", "n16d3"])
def test_ntt_matches_oracle(K, O, name):
    ctx, P = get(K, O, name)
    ids = [0, 1, P.L - 1, P.L, P.L + P.alpha - 1]
    primes = P.all_primes()[ids]
    a = np.stack([inputs.uniform_residues(7, [p], P.n)[0] for p in primes])
    got = K.ckks_step_ntt(ctx, a, ids, inverse=False)
    assert np.array_equal(got, O.ntt(a, primes))
    got_i = K.ckks_step_ntt(ctx, a, ids, inverse=True)
    assert np.array_equal(got_i, O.intt(a, primes))


def test_ntt_edge_values(K, O):
    ctx, P = get(K, O, "n16d3")
    ids = [0, 1, P.L]
    primes = P.all_primes()[ids]
    a = np.zeros((3, P.n), np.uint32)
    a[:, 0] = primes - 1
    a[:, -1] = primes - 1
    a[1, :] = primes[1] - 1         # every coefficient q - 1
    for inv in (False, True):
        want = O.intt(a, primes) if inv else O.ntt(a, primes)
        assert np.array_equal(K.ckks_step_ntt(ctx, a, ids, inverse=inv), want)


# ------------------------------------------------------------- a3: tensor ---

@pytest.mark.parametrize("name,n_q", [("toyT1", 4), ("n16d3", 3)])
def test_tensor_matches_oracle(K, O, name, n_q):
    ctx, P = get(K, O, name)
    c1, c2 = rand_ct(P, n_q, 1), rand_ct(P, n_q, 2)
    assert np.array_equal(K.ckks_step_tensor(ctx, c1, c2), O.tensor(c1, c2, P.q[:n_q]))


# -------------------------------------------------------------- a4: BConv ---

@pytest.mark.parametrize("variant", [0, 1])
@pytest.mark.parametrize("k_src,m_dst", [(1, 3), (2, 5), (8, 40), (14, 40), (40, 40)])
def test_bconv_matches_oracle(K, O, variant, k_src, m_dst):
    ctx, P = get(K, O, "n16d3")
    allp = P.all_primes()
    src = list(range(k_src))
    dst = list(range(P.L, P.L + P.alpha)) + list(range(k_src, P.L))
    dst = dst[:m_dst]
    x = np.stack([inputs.uniform_residues(k_src, [allp[i]], P.n)[0] for i in src])
    # extreme columns: all (q-1)/2, all (q+1)/2, all 0, all q-1
    half = ((allp[src] - 1) // 2).astype(np.uint32)
    x[:, 0], x[:, 1], x[:, 2], x[:, 3] = half, half + 1, 0, allp[src] - 1
    got = K.ckks_step_bconv(ctx, x, src, dst, variant)
    assert np.array_equal(got, O.bconv(x, allp[src], allp[dst]))


def test_bconv_tensor_core_equals_cuda_core(K, O):
    ctx, P = get(K, O, "toyT2")
    allp = P.all_primes()
    x = np.stack([inputs.uniform_residues(3, [allp[i]], P.n)[0] for i in range(4)])
    a = K.ckks_step_bconv(ctx, x, [0, 1, 2, 3], [4, 5, 6, 7], 0)
    b = K.ckks_step_bconv(ctx, x, [0, 1, 2, 3], [4, 5, 6, 7], 1)
    assert np.array_equal(a, b)


# ------------------------------------------------------------- a4: ModUp ---

@pytest.mark.parametrize("name,n_q", [("tiny", 6), ("tiny", 5), ("tiny", 1), ("toyT1", 4), ("toyT2", 3),
                                      ("n16d3", 40), ("n16d3", 21), ("n16d3", 2)])
def test_modup_matches_oracle(K, O, name, n_q):
    ctx, P = get(K, O, name)
    d = rand_poly(P, P.q[:n_q], 11)
    assert np.array_equal(K.ckks_step_modup(ctx, d, P.alpha), O.modup(P, d, n_q))


# -------------------------------------------------- a5: KeyMult + MAC ---

@pytest.mark.parametrize("name,n_q", [("tiny", 6), ("tiny", 3), ("toyT2", 4), ("n16d3", 40), ("n16d3", 15)])
def test_keyswitch_acc_matches_oracle(K, O, name, n_q):
    ctx, P = get(K, O, name)
    d = rand_poly(P, P.q[:n_q], 12)
    evk = rand_evk(P, 13)
    ek = K.ckks_evk_import(ctx, evk, 0)
    try:
        got = K.ckks_step_keyswitch_acc(ctx, d, ek, P.alpha)
    finally:
        K.ckks_free(ek)
    assert np.array_equal(got, O.keymult(P, O.modup(P, d, n_q), n_q, evk))


# ------------------------------------------------------ a6: automorphism ---

@pytest.mark.parametrize("name", ["tiny", "toyT1", "n16d3"])
def test_automorph_matches_oracle(K, O, name):
    ctx, P = get(K, O, name)
    a = rand_poly(P, P.q[:3], 14)
    for k in (O.rot_k(1, P.log_n), O.rot_k(5, P.log_n), O.rot_k(12345, P.log_n), O.conj_k(P.log_n)):
        assert np.array_equal(K.ckks_step_automorph(ctx, a, k), O.automorph_ntt(a, k))


# ------------------------------------------------------------ a7: ModDown ---

@pytest.mark.parametrize("name,n_q", [("tiny", 6), ("toyT1", 2), ("toyT2", 4), ("n16d3", 40), ("n16d3", 2)])
def test_moddown_matches_oracle(K, O, name, n_q):
    ctx, P = get(K, O, name)
    ext = P.ext_primes(n_q)
    acc = np.stack([rand_poly(P, ext, 15, t) for t in range(2)])
    assert np.array_equal(K.ckks_step_moddown(ctx, acc, n_q), O.moddown(P, acc, n_q))


# ------------------------------------------------------------ a8: rescale ---

@pytest.mark.parametrize("name,n_q", [("tiny", 6), ("tiny", 2), ("toyT1", 4), ("n16d3", 40), ("n16d3", 2)])
def test_rescale_matches_oracle(K, O, name, n_q):
    ctx, P = get(K, O, name)
    c = rand_ct(P, n_q, 16)
    ct = K.ckks_ct_import(ctx, c, n_q - 1, 2.0**60)
    out = K.ckks_ct_create(ctx, n_q - 2)
    try:
        K.ckks_rescale(ctx, ct, out)
        got, level, scale = K.ckks_ct_export(ctx, out, P.n)
    finally:
        K.ckks_free(ct)
        K.ckks_free(out)
    assert level == n_q - 2 and scale == 2.0**60 / float(P.q[n_q - 1])
    assert np.array_equal(got, O.rescale(c, P.q[:n_q]))


# ----------------------------------------------------- a9: HAdd / PMult ---

def test_hadd_pmult_padd_match_oracle(K, O):
    ctx, P = get(K, O, "n16d3")
    n_q = 5
    x, y = rand_ct(P, n_q, 17), rand_ct(P, n_q, 19)
    pt = rand_poly(P, P.q[:n_q], 21)
    cx, cy = K.ckks_ct_import(ctx, x, n_q - 1, 2.0**30), K.ckks_ct_import(ctx, y, n_q - 1, 2.0**30)
    p = K.ckks_pt_import(ctx, pt, n_q - 1, 2.0**30)
    out = K.ckks_ct_create(ctx, n_q - 1)
    try:
        K.ckks_hadd(ctx, cx, cy, out)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.hadd(x, y, P.q[:n_q]))
        K.ckks_pmult(ctx, cx, p, out)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.pmult(x, pt, P.q[:n_q]))
        K.ckks_padd(ctx, cx, p, out)
        zero = np.zeros_like(pt)
        assert np.array_equal(K.ckks_ct_export(ctx, out, P.n)[0], O.hadd(x, np.stack([pt, zero]), P.q[:n_q]))
        K.ckks_hadd(ctx, cx, cy, cx)   # in place
        assert np.array_equal(K.ckks_ct_export(ctx, cx, P.n)[0], O.hadd(x, y, P.q[:n_q]))
    finally:
        for h in (cx, cy, p, out):
            K.ckks_free(h)


# -------------------------------------------------- full HMult / HRot ---

def _run_hmult(K, ctx, P, c1, c2, evk, rescale, flags=None):
    n_q = c1.shape[1]
    a = K.ckks_ct_import(ctx, c1, n_q - 1, 2.0**30)
    b = K.ckks_ct_import(ctx, c2, n_q - 1, 2.0**30)
    ek = K.ckks_evk_import(ctx, evk, 0)
    out = K.ckks_ct_create(ctx, n_q - 1)
    if flags is None:
        flags = K.CKKS_RESCALE if rescale else 0
    try:
        K.ckks_hmult(ctx, a, b, ek, flags, out)
        return K.ckks_ct_export(ctx, out, P.n)
    finally:
        for h in (a, b, ek, out):
            K.ckks_free(h)


def _run_hrot(K, O, ctx, P, c, evk, r=None):
    n_q = c.shape[1]
    k = O.conj_k(P.log_n) if r is None else O.rot_k(r, P.log_n)
    a = K.ckks_ct_import(ctx, c, n_q - 1, 2.0**30)
    ek = K.ckks_evk_import(ctx, evk, k)
    out = K.ckks_ct_create(ctx, n_q - 1)
    try:
        if r is None:
            K.ckks_hconj(ctx, a, ek, out)
        else:
            K.ckks_hrot(ctx, a, r, ek, out)
        return K.ckks_ct_export(ctx, out, P.n)[0], k
    finally:
        for h in (a, ek, out):
            K.ckks_free(h)


@pytest.mark.parametrize("name,n_q,rescale", [("tiny", 6, True), ("tiny", 4, False), ("tiny", 1, False),
                                              ("toyT1", 4, True), ("toyT2", 4, True), ("toyT2", 2, False),
                                              ("n16d3", 40, True), ("n16d3", 21, True), ("n16d3", 2, True)])
def test_hmult_matches_oracle(K, O, name, n_q, rescale):
    ctx, P = get(K, O, name)
    c1, c2 = rand_ct(P, n_q, 31), rand_ct(P, n_q, 33)
    evk = rand_evk(P, 35)
    got, level, _ = _run_hmult(K, ctx, P, c1, c2, evk, rescale)
    assert level == n_q - 1 - int(rescale)
    assert np.array_equal(got, O.hmult(P, c1, c2, evk, rescale=rescale))


@pytest.mark.parametrize("name,n_q", [("tiny", 6), ("tiny", 2), ("toyT1", 4), ("toyT2", 3), ("toyT2", 2),
                                      ("n16d3", 40), ("n16d3", 17), ("n16d3", 2)])
def test_hmult_merged_matches_oracle(K, O, name, n_q):
    """ModDown merged into the rescaling (Sec. 6): residues equal the oracle's
    merged definition bit for bit; level and scale as with CKKS_RESCALE."""
    ctx, P = get(K, O, name)
    c1, c2 = rand_ct(P, n_q, 131), rand_ct(P, n_q, 133)
    evk = rand_evk(P, 135)
    got, level, scale = _run_hmult(K, ctx, P, c1, c2, evk, True, K.CKKS_RESCALE_MERGED)
    assert level == n_q - 2
    assert scale == pytest.approx(2.0**60 / float(P.q[n_q - 1]), rel=1e-12)
    assert np.array_equal(got, O.hmult_merged(P, c1, c2, evk))
    # both flags together mean the merged form
    got2, _, _ = _run_hmult(K, ctx, P, c1, c2, evk, True, K.CKKS_RESCALE | K.CKKS_RESCALE_MERGED)
    assert np.array_equal(got2, got)


@pytest.mark.parametrize("name,n_q,r", [("tiny", 6, 1), ("tiny", 1, 3), ("toyT1", 4, 1), ("toyT2", 4, 7),
                                        ("toyT2", 4, None), ("n16d3", 40, 1), ("n16d3", 21, 5),
                                        ("n16d3", 2, 12345), ("n16d3", 40, None)])
def test_hrot_matches_oracle(K, O, name, n_q, r):
    ctx, P = get(K, O, name)
    c = rand_ct(P, n_q, 41)
    evk = rand_evk(P, 43)
    got, k = _run_hrot(K, O, ctx, P, c, evk, r)
    assert np.array_equal(got, O.hrot(P, c, k, evk))


@pytest.mark.parametrize("dnum", [1, 5])
def test_hmult_full_size_other_dnum(K, O, dnum):
    """N = 2^16, 40 primes, top level, dnum in {1, 5}: bit-exact HMult+rescale and HRot."""
    P = O.make_params(16, 40, dnum)
    ctx = K.ckks_ctx_create(16, P.q, P.p, dnum, scale=2.0**30)
    try:
        c1, c2 = rand_ct(P, 40, 51), rand_ct(P, 40, 53)
        evk = rand_evk(P, 55)
        got, _, _ = _run_hmult(K, ctx, P, c1, c2, evk, True)
        assert np.array_equal(got, O.hmult(P, c1, c2, evk, rescale=True))
        got, _, _ = _run_hmult(K, ctx, P, c1, c2, evk, True, K.CKKS_RESCALE_MERGED)
        assert np.array_equal(got, O.hmult_merged(P, c1, c2, evk))
        got, k = _run_hrot(K, O, ctx, P, c1, evk, 1)
        assert np.array_equal(got, O.hrot(P, c1, k, evk))
    finally:
        K.ckks_ctx_destroy(ctx)


def test_more_auxiliary_than_ciphertext_primes(K, O):
    """alpha > L (one digit, five auxiliary primes, three ciphertext primes):
    HMult with rescaling and HRot stay bit-exact."""
    P = O.make_params(12, 3, 1, 5)
    ctx = K.ckks_ctx_create(12, P.q, P.p, 1, scale=2.0**30)
    try:
        c1, c2 = rand_ct(P, 3, 57), rand_ct(P, 3, 59)
        evk = rand_evk(P, 61)
        got, _, _ = _run_hmult(K, ctx, P, c1, c2, evk, True)
        assert np.array_equal(got, O.hmult(P, c1, c2, evk, rescale=True))
        got, _, _ = _run_hmult(K, ctx, P, c1, c2, evk, True, K.CKKS_RESCALE_MERGED)
        assert np.array_equal(got, O.hmult_merged(P, c1, c2, evk))
        got, k = _run_hrot(K, O, ctx, P, c1, evk, 3)
        assert np.array_equal(got, O.hrot(P, c1, k, evk))
    finally:
        K.ckks_ctx_destroy(ctx)


# ------------------------------------------------- hoisted rotations ---

@pytest.mark.parametrize("name,n_q,rs", [("tiny", 6, [1, 2, 5]), ("tiny", 1, [3]), ("toyT1", 4, [1, 7, 100]),
                                         ("toyT2", 3, [2, 9]), ("n16d3", 40, [1, 2, 3, 17]),
                                         ("n16d3", 21, [5, 12345]), ("n16d3", 2, [1, 4])])
def test_hrot_hoisted_matches_oracle(K, O, name, n_q, rs):
    """One ModUp shared by several rotations (Par. 5): every output equals the
    oracle's separate HRot bit for bit."""
    ctx, P = get(K, O, name)
    c = rand_ct(P, n_q, 91)
    evks = [rand_evk(P, 93 + i) for i in range(len(rs))]
    a = K.ckks_ct_import(ctx, c, n_q - 1, 2.0**30)
    eks = [K.ckks_evk_import(ctx, e, O.rot_k(r, P.log_n)) for e, r in zip(evks, rs)]
    outs = [K.ckks_ct_create(ctx, n_q - 1) for _ in rs]
    try:
        K.ckks_hrot_hoisted(ctx, a, rs, eks, outs)
        for r, e, o in zip(rs, evks, outs):
            got, level, _ = K.ckks_ct_export(ctx, o, P.n)
            assert level == n_q - 1
            assert np.array_equal(got, O.hrot(P, c, O.rot_k(r, P.log_n), e)), r
    finally:
        for h in [a] + eks + outs:
            K.ckks_free(h)


def test_hrot_hoisted_rejects_bad_calls(K, O):
    ctx, P = get(K, O, "tiny")
    c = rand_ct(P, 4, 97)
    a = K.ckks_ct_import(ctx, c, 3, 2.0**30)
    e1 = K.ckks_evk_import(ctx, rand_evk(P, 98), O.rot_k(1, P.log_n))
    o1, o2 = K.ckks_ct_create(ctx, 3), K.ckks_ct_create(ctx, 1)
    try:
        K.ckks_hrot_hoisted(ctx, a, [], [], [])                  # nothing to do
        with pytest.raises(RuntimeError):
            K.ckks_hrot_hoisted(ctx, a, [2], [e1], [o1])         # key for another rotation
        with pytest.raises(RuntimeError):
            K.ckks_hrot_hoisted(ctx, a, [1], [e1], [a])          # output aliases the input
        with pytest.raises(RuntimeError):
            K.ckks_hrot_hoisted(ctx, a, [1, 1], [e1, e1], [o1, o1])  # shared output
        with pytest.raises(RuntimeError):
            K.ckks_hrot_hoisted(ctx, a, [1], [e1], [o2])         # capacity too small
    finally:
        for h in (a, e1, o1, o2):
            K.ckks_free(h)


# ------------------------------------------------ linear transform ---

def _rand_ext_pt(P, n_q, seed):
    return inputs.uniform_residues(seed, list(P.q[:n_q]) + list(P.p), P.n, 7)


@pytest.mark.parametrize("name,n_q,rs", [("tiny", 6, [0, 1, 2, 5]), ("tiny", 1, [3, 0]), ("toyT1", 4, [1, 7, 1]),
                                         ("toyT2", 3, [0, 2]), ("n16d3", 40, [0, 1, 2, 3, 17]),
                                         ("n16d3", 21, [5, 12345]), ("n16d3", 2, [1]), ("n16d3", 40, [0])])
def test_linear_transform_matches_oracle(K, O, name, n_q, rs):
    ctx, P = get(K, O, name)
    c = rand_ct(P, n_q, 101)
    evks = [rand_evk(P, 103 + i) if r else None for i, r in enumerate(rs)]
    pts = [_rand_ext_pt(P, n_q, 111 + i) for i in range(len(rs))]
    a = K.ckks_ct_import(ctx, c, n_q - 1, 2.0**30)
    eks = [K.ckks_evk_import(ctx, e, O.rot_k(r, P.log_n)) if r else None for e, r in zip(evks, rs)]
    dps = [K.ckks_pt_import_ext(ctx, pt, n_q - 1, 2.0**20) for pt in pts]
    out = K.ckks_ct_create(ctx, n_q - 1)
    try:
        K.ckks_linear_transform(ctx, a, rs, eks, dps, out)
        got, level, scale = K.ckks_ct_export(ctx, out, P.n)
        assert level == n_q - 1 and scale == 2.0**50
        assert np.array_equal(got, O.linear_transform(P, c, rs, evks, pts))
    finally:
        for h in [a, out] + [e for e in eks if e] + dps:
            K.ckks_free(h)


def test_linear_transform_decrypts_with_library_keys(K, O):
    """N = 2^16, top level: library encryption, keys and extended encodings;
    the decryption is the weighted sum of rotations within 1e-3."""
    ctx, P = get(K, O, "n16d3")
    lv = 39
    sk = K.ckks_keygen_secret(ctx, 7)
    u = inputs.messages(7, P.n // 2)
    rs = [0, 1, 2, 3, 4, 8]
    diags = [inputs.messages(70 + i, P.n // 2) for i in range(len(rs))]
    handles = [sk]
    try:
        pt = K.ckks_encode(ctx, u, lv, 2.0**30)
        ct = K.ckks_encrypt(ctx, sk, pt, 8)
        handles += [pt, ct]
        eks = [K.ckks_keygen_rot(ctx, sk, r, 200 + r) if r else None for r in rs]
        dps = [K.ckks_encode_ext(ctx, d, lv, 2.0**30) for d in diags]
        handles += [e for e in eks if e] + dps
        out = K.ckks_ct_create(ctx, lv)
        handles.append(out)
        K.ckks_linear_transform(ctx, ct, rs, eks, dps, out)
        res = K.ckks_ct_create(ctx, lv - 1)
        handles.append(res)
        K.ckks_rescale(ctx, out, res)
        dec = K.ckks_decrypt(ctx, sk, res)
        handles.append(dec)
        got = K.ckks_decode(ctx, dec, P.n // 2)
        want = sum(d * np.roll(u, -r) for d, r in zip(diags, rs))
        assert np.max(np.abs(got - want)) < 1e-3
    finally:
        for h in handles:
            K.ckks_free(h)


def test_linear_transform_rejects_bad_calls(K, O):
    ctx, P = get(K, O, "tiny")
    c = rand_ct(P, 4, 121)
    a = K.ckks_ct_import(ctx, c, 3, 2.0**30)
    e1 = K.ckks_evk_import(ctx, rand_evk(P, 122), O.rot_k(1, P.log_n))
    plain = K.ckks_pt_import(ctx, rand_ct(P, 4, 123)[0], 3, 1.0)
    ext = K.ckks_pt_import_ext(ctx, _rand_ext_pt(P, 4, 124), 3, 1.0)
    ext2 = K.ckks_pt_import_ext(ctx, _rand_ext_pt(P, 4, 125), 3, 2.0)
    out = K.ckks_ct_create(ctx, 3)
    try:
        with pytest.raises(RuntimeError):
            K.ckks_linear_transform(ctx, a, [1], [e1], [plain], out)       # not an extended plaintext
        with pytest.raises(RuntimeError):
            K.ckks_linear_transform(ctx, a, [2], [e1], [ext], out)         # key for another rotation
        with pytest.raises(RuntimeError):
            K.ckks_linear_transform(ctx, a, [1, 0], [e1, None], [ext, ext2], out)  # scales differ
        with pytest.raises(RuntimeError):
            K.ckks_linear_transform(ctx, a, [1], [e1], [ext], a)           # output aliases the input
        with pytest.raises(RuntimeError):
            K.ckks_linear_transform(ctx, a, [0] * 65, [None] * 65, [ext] * 65, out)  # too many terms
    finally:
        for h in (a, e1, plain, ext, ext2, out):
            K.ckks_free(h)


# --------------------------------------------- launch-shape fine-tuning ---

SHAPES = [(tc, sl, z, tp) for tc in (8, 4) for sl in (2, 4, 8) for z in (1, 2, 3, 4) for tp in (1, 2)]


def _set_all(K, ctx, level, shape):
    for kern in (K.CKKS_COL_MODUP, K.CKKS_COL_MODDOWN, K.CKKS_COL_RS_FUSED):
        K.ckks_tune_set(ctx, kern, level, *shape)


@pytest.mark.parametrize("name,n_q", [("n16d3", 40), ("n16d3", 3), ("toyT2", 4), ("tiny", 6)])
def test_every_column_shape_gives_identical_results(K, O, name, n_q):
    """Each launch shape of the three column kernels (tile width, slices,
    target split; some with idle slices at small levels) reproduces the
    oracle's HMult+rescale and HRot bit for bit."""
    ctx, P = get(K, O, name)
    c1, c2 = rand_ct(P, n_q, 71), rand_ct(P, n_q, 73)
    evk = rand_evk(P, 75)
    want_m = O.hmult(P, c1, c2, evk, rescale=n_q > 1)
    k = O.rot_k(1, P.log_n)
    want_r = O.hrot(P, c1, k, evk)
    try:
        for shape in SHAPES:
            if P.log_n == 8 and shape[0] == 4:
                # 4 columns x 4 rows per thread is half a warp per slice: refused
                with pytest.raises(RuntimeError):
                    K.ckks_tune_set(ctx, K.CKKS_COL_MODUP, n_q - 1, *shape)
                continue
            _set_all(K, ctx, n_q - 1, shape)
            got, _, _ = _run_hmult(K, ctx, P, c1, c2, evk, n_q > 1)
            assert np.array_equal(got, want_m), shape
            got, _ = _run_hrot(K, O, ctx, P, c1, evk, 1)
            assert np.array_equal(got, want_r), shape
    finally:
        _set_all(K, ctx, n_q - 1, (0, 4, 1, 1))


def test_tune_records_a_shape_and_keeps_results(K, O):
    ctx, P = get(K, O, "n16d3")
    n_q = 21
    K.ckks_tune(ctx, n_q - 1, 2)
    try:
        for kern in (K.CKKS_COL_MODUP, K.CKKS_COL_MODDOWN, K.CKKS_COL_RS_FUSED):
            tc, sl, z, tp, us = K.ckks_tune_get(ctx, kern, n_q - 1)
            assert tc in (4, 8) and sl in (2, 4, 8) and 1 <= z <= 4 and tp in (1, 2, 8, 16) and us > 0
        passes, _, _, _, us = K.ckks_tune_get(ctx, K.CKKS_ROW_PASSES, n_q - 1)
        assert passes in (2, 3, 4, 5) and us > 0
        # a clone shares the table
        import torch
        s = torch.cuda.Stream()
        lane = K.ckks_ctx_clone(ctx, s.cuda_stream)
        try:
            assert K.ckks_tune_get(lane, K.CKKS_COL_MODUP, n_q - 1) == K.ckks_tune_get(ctx, K.CKKS_COL_MODUP, n_q - 1)
        finally:
            K.ckks_ctx_destroy(lane)
        c1, c2 = rand_ct(P, n_q, 81), rand_ct(P, n_q, 83)
        evk = rand_evk(P, 85)
        got, _, _ = _run_hmult(K, ctx, P, c1, c2, evk, True)
        assert np.array_equal(got, O.hmult(P, c1, c2, evk, rescale=True))
    finally:
        _set_all(K, ctx, n_q - 1, (0, 4, 1, 1))
        K.ckks_tune_set(ctx, K.CKKS_ROW_PASSES, n_q - 1, 0, 1, 1, 1)


def test_tune_file_round_trip(K, O, tmp_path):
    """Shapes tuned on one context and written to the GPU's tune file are set
    on the next context from the file, without timing, and keep the results."""
    import torch
    from paper_2407_13055_gb300 import tune_cache
    ctx, P = get(K, O, "n16d3")
    n_q = 21
    gpu = tune_cache.gpu_identity(torch.cuda.current_device())
    assert gpu["sms"] > 0 and gpu["cc"]
    path = str(tmp_path / "tune.json")
    pkey = tune_cache.params_key(P.log_n, P.q, P.p, P.dnum)
    levels = [n_q - 1]
    try:
        first, loaded, tuned = tune_cache.tune_or_load(K, ctx, levels, pkey, tune_cache.TuneStore(path, gpu), reps=2)
        assert loaded == [] and tuned == levels
        for kid in tune_cache.kernel_names(K).values():
            K.ckks_tune_set(ctx, kid, n_q - 1, 0, 1, 1, 1)
        again, loaded, tuned = tune_cache.tune_or_load(K, ctx, levels, pkey, tune_cache.TuneStore(path, gpu), reps=2)
        assert loaded == levels and tuned == []
        for name, kid in tune_cache.kernel_names(K).items():
            assert K.ckks_tune_get(ctx, kid, n_q - 1)[:4] == first[n_q - 1][name][:4], name
        assert again[n_q - 1]["modup_cols"][4] == pytest.approx(first[n_q - 1]["modup_cols"][4], abs=1e-3)
        c1, c2 = rand_ct(P, n_q, 91), rand_ct(P, n_q, 93)
        evk = rand_evk(P, 95)
        got, _, _ = _run_hmult(K, ctx, P, c1, c2, evk, True)
        assert np.array_equal(got, O.hmult(P, c1, c2, evk, rescale=True))
    finally:
        _set_all(K, ctx, n_q - 1, (0, 4, 1, 1))
        K.ckks_tune_set(ctx, K.CKKS_ROW_PASSES, n_q - 1, 0, 1, 1, 1)


@pytest.mark.parametrize("n_q", [40, 5])
def test_row_phase_forms_give_identical_results(K, O, n_q):
    """Every form of the N = 2^16 row phase the tuner chooses between (two
    register passes of radix 2^5, three of 2^4 x 2^3 x 2^3, the three-pass
    form with its forward rows staged by bulk copies, 2 or 4 row pairs per
    block, and the three-pass form with its twiddles staged in shared memory)
    reproduces the oracle bit for bit: HMult+rescale, HMult with the merged
    ModDown + rescale, HRot and hoisted rotations."""
    ctx, P = get(K, O, "n16d3")
    c1, c2 = rand_ct(P, n_q, 91), rand_ct(P, n_q, 93)
    evk = rand_evk(P, 95)
    want_m = O.hmult(P, c1, c2, evk, rescale=True)
    want_mm = O.hmult_merged(P, c1, c2, evk)
    k = O.rot_k(1, P.log_n)
    want_r = O.hrot(P, c1, k, evk)
    a = K.ckks_ct_import(ctx, c1, n_q - 1, 2.0**30)
    ek = K.ckks_evk_import(ctx, evk, k)
    outs = [K.ckks_ct_create(ctx, n_q - 1) for _ in range(2)]
    try:
        for passes in (2, 3, 4, 5, 6):
            K.ckks_tune_set(ctx, K.CKKS_ROW_PASSES, n_q - 1, passes, 1, 1, 1)
            got, _, _ = _run_hmult(K, ctx, P, c1, c2, evk, True)
            assert np.array_equal(got, want_m), passes
            got, _, _ = _run_hmult(K, ctx, P, c1, c2, evk, True, K.CKKS_RESCALE_MERGED)
            assert np.array_equal(got, want_mm), passes
            got, _ = _run_hrot(K, O, ctx, P, c1, evk, 1)
            assert np.array_equal(got, want_r), passes
            K.ckks_hrot_hoisted(ctx, a, [1, 1], [ek, ek], outs)
            for o in outs:
                assert np.array_equal(K.ckks_ct_export(ctx, o, P.n)[0], want_r), passes
        with pytest.raises(K.CkksError):
            K.ckks_tune_set(ctx, K.CKKS_ROW_PASSES, n_q - 1, 7, 1, 1, 1)
    finally:
        K.ckks_tune_set(ctx, K.CKKS_ROW_PASSES, n_q - 1, 0, 1, 1, 1)
        for h in [a, ek] + outs:
            K.ckks_free(h)


def test_tune_rejects_bad_arguments(K, O):
    ctx, P = get(K, O, "tiny")
    with pytest.raises(RuntimeError):
        K.ckks_tune_set(ctx, 0, 0, 16, 4, 1, 1)
    with pytest.raises(RuntimeError):
        K.ckks_tune_set(ctx, 3, 0, 8, 4, 1, 1)
    with pytest.raises(RuntimeError):
        K.ckks_tune_set(ctx, 0, P.L, 8, 4, 1, 1)
    with pytest.raises(RuntimeError):
        K.ckks_tune(ctx, 0, 0)


def test_integer_multiply_probe_runs(K, O):
    """The issue-rate probe behind the integer-ALU roofline returns a plausible
    rate for each form (between 1 and 256 per SM per clock at 1-2.1 GHz)."""
    ctx, P = get(K, O, "tiny")
    for op in (K.CKKS_INTOP_MAD_LO, K.CKKS_INTOP_MAD_HI, K.CKKS_INTOP_MAD_WIDE):
        n_ops, ms = K.ckks_bench_intop(ctx, op, 64)
        assert n_ops > 0 and ms > 0
        per_sm_clk = n_ops / (ms * 1e-3) / 152 / 2.07e9
        assert 0.5 < per_sm_clk < 300
    with pytest.raises(K.CkksError):
        K.ckks_bench_intop(ctx, 7, 64)


@pytest.mark.parametrize("prime_id,rounds", [(0, 1), (1, 2), (5, 37), (39, 1000)])
def test_modmul_methods_agree_with_big_integers(K, O, prime_id, rounds):
    """Barrett, Montgomery, Shoup and signed Montgomery (Table 3) all give
    a b^rounds mod q exactly (31-bit q_0 and 30-bit q_i)."""
    ctx, P = get(K, O, "n16d3")
    q = int(P.q[prime_id])
    rng = np.random.default_rng(prime_id + rounds)
    a = rng.integers(0, q, 5000, dtype=np.int64).astype(np.uint32)
    a[:4] = [0, 1, q - 1, q // 2]
    b = int(rng.integers(1, q))
    want = np.array([(int(x) * pow(b, rounds, q)) % q for x in a], dtype=np.uint32)
    for m in (K.CKKS_MODMUL_BARRETT, K.CKKS_MODMUL_MONTGOMERY, K.CKKS_MODMUL_SHOUP, K.CKKS_MODMUL_SMR):
        got, ms = K.ckks_bench_modmul(ctx, m, prime_id, b, a, rounds)
        assert np.array_equal(got, want), m
        assert ms >= 0


def test_async_transfers_match_synchronous_ones(K, O):
    """Asynchronous upload / export on a lane give the same residues as the
    synchronous calls."""
    import torch
    ctx, P = get(K, O, "n16d3")
    n_q = 6
    c = rand_ct(P, n_q, 131)
    host = torch.empty((2, n_q, P.n), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    host[:] = c
    out = torch.empty((2, n_q, P.n), dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    s = torch.cuda.Stream()
    lane = K.ckks_ctx_clone(ctx, s.cuda_stream)
    ct = K.ckks_ct_create(ctx, n_q - 1)
    try:
        K.ckks_ct_upload_async(lane, ct, host, n_q - 1, 2.0**30)
        K.ckks_ct_export_async(lane, ct, out)
        K.ckks_sync(lane)
        assert np.array_equal(out, c)
        with pytest.raises(TypeError):
            K.ckks_ct_upload_async(lane, ct, c.astype(np.int64), n_q - 1, 1.0)
    finally:
        K.ckks_free(ct)
        K.ckks_ctx_destroy(lane)


def test_pipelined_transfers_across_lanes_match_oracle(K, O):
    """The end-to-end pattern: uploads on a transfer-only clone, HMult+rescale
    and HRot on a compute lane, exports on a second transfer-only clone, with
    CUDA events between the stages and two buffer slots per lane reused in
    flight. Every exported result equals the oracle's."""
    import torch
    ctx, P = get(K, O, "toyT1")
    n_q, nl, ns, pairs = P.L, 2, 2, 6
    pinned = lambda shape: torch.empty(shape, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    cts = [rand_ct(P, n_q, 140 + i) for i in range(pairs + 1)]
    host_in = [pinned((2, n_q, P.n)) for _ in cts]
    for h, c in zip(host_in, cts):
        h[:] = c
    evk_m, evk_r = rand_evk(P, 150), rand_evk(P, 151)
    k = O.rot_k(1, P.log_n)
    rk, gk = K.ckks_evk_import(ctx, evk_m, 0), K.ckks_evk_import(ctx, evk_r, k)
    cs = [torch.cuda.Stream() for _ in range(nl)]
    us = [torch.cuda.Stream() for _ in range(nl)]
    ds = [torch.cuda.Stream() for _ in range(nl)]
    lanes = [K.ckks_ctx_clone(ctx, x.cuda_stream) for x in cs]
    up = [K.ckks_ctx_clone(ctx, x.cuda_stream) for x in us]
    dn = [K.ckks_ctx_clone(ctx, x.cuda_stream) for x in ds]
    slot = lambda: [[K.ckks_ct_create(ctx, n_q - 1) for _ in range(ns)] for _ in range(nl)]
    da, db, dm, dr = slot(), slot(), slot(), slot()
    out_m = [pinned((2, n_q - 1, P.n)) for _ in range(pairs)]
    out_r = [pinned((2, n_q, P.n)) for _ in range(pairs)]
    ev = lambda: [[torch.cuda.Event() for _ in range(ns)] for _ in range(nl)]
    eu, ec, ed = ev(), ev(), ev()
    main = torch.cuda.current_stream()
    for l in range(nl):
        for j in range(ns):
            ec[l][j].record(main)
            ed[l][j].record(main)
    try:
        for i in range(pairs):
            l, j = i % nl, (i // nl) % ns
            us[l].wait_event(ec[l][j])
            K.ckks_ct_upload_async(up[l], da[l][j], host_in[i], n_q - 1, 2.0**30)
            K.ckks_ct_upload_async(up[l], db[l][j], host_in[i + 1], n_q - 1, 2.0**30)
            eu[l][j].record(us[l])
            cs[l].wait_event(eu[l][j])
            cs[l].wait_event(ed[l][j])
            K.ckks_hmult(lanes[l], da[l][j], db[l][j], rk, K.CKKS_RESCALE, dm[l][j])
            K.ckks_hrot(lanes[l], da[l][j], 1, gk, dr[l][j])
            ec[l][j].record(cs[l])
            ds[l].wait_event(ec[l][j])
            K.ckks_ct_export_async(dn[l], dm[l][j], out_m[i])
            K.ckks_ct_export_async(dn[l], dr[l][j], out_r[i])
            ed[l][j].record(ds[l])
        torch.cuda.synchronize()
        for i in range(pairs):
            assert np.array_equal(out_m[i], O.hmult(P, cts[i], cts[i + 1], evk_m, rescale=True)), i
            assert np.array_equal(out_r[i], O.hrot(P, cts[i], k, evk_r)), i
    finally:
        for grp in (da, db, dm, dr):
            for row in grp:
                for h in row:
                    K.ckks_free(h)
        for c in lanes + up + dn:
            K.ckks_ctx_destroy(c)
        K.ckks_free(rk)
        K.ckks_free(gk)


# ----------------------------------------- decryption after operations ---

@pytest.mark.parametrize("name", ["toyT1", "toyT2", "n16d3"])
def test_library_keys_decrypt_within_tolerance(K, O, name):
    """Keys, encryption and decoding from the library itself; decrypted slots
    within 1e-3 of the plaintext result (Sec. 2.1 semantics)."""
    ctx, P = get(K, O, name)
    scale = 2.0**28 if P.log_n == 12 else 2.0**30
    n_q = P.L if P.log_n == 12 else 6
    slots = P.n // 2
    u, v = inputs.messages(61, slots), inputs.messages(62, slots)
    sk = K.ckks_keygen_secret(ctx, 63)
    rk = K.ckks_keygen_relin(ctx, sk, 64)
    gk = K.ckks_keygen_rot(ctx, sk, 3, 65)
    ck = K.ckks_keygen_conj(ctx, sk, 66)
    hs = [sk, rk, gk, ck]
    try:
        pu, pv = K.ckks_encode(ctx, u, n_q - 1, scale), K.ckks_encode(ctx, v, n_q - 1, scale)
        cu, cv = K.ckks_encrypt(ctx, sk, pu, 67), K.ckks_encrypt(ctx, sk, pv, 68)
        out = K.ckks_ct_create(ctx, n_q - 1)
        hs += [pu, pv, cu, cv, out]

        def dec(ct):
            pt = K.ckks_decrypt(ctx, sk, ct)
            try:
                return K.ckks_decode(ctx, pt, slots)
            finally:
                K.ckks_free(pt)

        assert np.max(np.abs(dec(cu) - u)) < 1e-3
        K.ckks_hmult(ctx, cu, cv, rk, K.CKKS_RESCALE, out)
        assert np.max(np.abs(dec(out) - u * v)) < 1e-3
        K.ckks_hmult(ctx, cu, cv, rk, K.CKKS_RESCALE_MERGED, out)
        assert np.max(np.abs(dec(out) - u * v)) < 1e-3
        K.ckks_hrot(ctx, cu, 3, gk, out)
        assert np.max(np.abs(dec(out) - np.roll(u, -3))) < 1e-3
        K.ckks_hconj(ctx, cu, ck, out)
        assert np.max(np.abs(dec(out) - np.conj(u))) < 1e-3
        K.ckks_hadd(ctx, cu, cv, out)
        assert np.max(np.abs(dec(out) - (u + v))) < 1e-3
    finally:
        for h in hs:
            K.ckks_free(h)


@pytest.mark.parametrize("level", [39, 34, 33])
def test_library_decode_at_high_levels(K, O, level):
    """Encode -> encrypt -> decrypt -> decode at levels whose modulus exceeds
    the double range (more than 33 primes)."""
    ctx, P = get(K, O, "n16d3")
    u = inputs.messages(64, P.n // 2)
    sk = K.ckks_keygen_secret(ctx, 65)
    pt = K.ckks_encode(ctx, u, level, 2.0**30)
    ct = K.ckks_encrypt(ctx, sk, pt, 66)
    dec = K.ckks_decrypt(ctx, sk, ct)
    try:
        assert np.max(np.abs(K.ckks_decode(ctx, dec, P.n // 2) - u)) < 1e-3
        assert np.max(np.abs(K.ckks_decode(ctx, pt, P.n // 2) - u)) < 1e-6
    finally:
        for h in (sk, pt, ct, dec):
            K.ckks_free(h)


def test_oracle_encryptions_decrypt_after_gpu_hmult(K, O):
    """Oracle keys and encryptions, GPU HMult, oracle decryption."""
    ctx, P = get(K, O, "toyT1")
    s = inputs.ternary_secret(71, P.n, None)
    allp = P.all_primes()
    a = np.stack([inputs.uniform_residues(71, allp, P.n, 200 + j) for j in range(P.dnum)])
    e = np.stack([inputs.gaussian_error(71, P.n, 200 + j) for j in range(P.dnum)])
    evk = O.keygen_relin(P, s, a, e)
    scale = 2.0**28
    u, v = inputs.messages(72, P.n // 2), inputs.messages(73, P.n // 2)
    cts = [O.encrypt(P, s, O.encode(P, m, scale, P.L), inputs.uniform_residues(71, P.q, P.n, 300 + i),
                     inputs.gaussian_error(71, P.n, 300 + i)) for i, m in enumerate((u, v))]
    got, level, _ = _run_hmult(K, ctx, P, cts[0], cts[1], evk, True)
    dec = O.decode(P, O.decrypt(P, s, got), scale * scale / float(P.q[P.L - 1]))
    assert np.max(np.abs(dec - u * v)) < 1e-3


# ------------------------------------------------------------- errors ---

def test_error_codes(K, O):
    ctx, P = get(K, O, "tiny")
    c3 = K.ckks_ct_import(ctx, rand_ct(P, 3, 81), 2, 2.0**30)
    c4 = K.ckks_ct_import(ctx, rand_ct(P, 4, 82), 3, 2.0**30)
    c0 = K.ckks_ct_import(ctx, rand_ct(P, 1, 83), 0, 2.0**30)
    out = K.ckks_ct_create(ctx, 5)
    rk = K.ckks_evk_import(ctx, rand_evk(P, 84), O.rot_k(1, P.log_n))
    try:
        with pytest.raises(K.CkksError) as e:
            K.ckks_hadd(ctx, c3, c4, out)
        assert e.value.code == K.CKKS_ELEVEL
        with pytest.raises(K.CkksError) as e:
            K.ckks_rescale(ctx, c0, out)
        assert e.value.code == K.CKKS_ELEVEL
        with pytest.raises(K.CkksError) as e:
            K.ckks_hmult(ctx, c3, c3, rk, 0, out)     # rotation key given to HMult
        assert e.value.code == K.CKKS_ENOKEY
        with pytest.raises(K.CkksError) as e:
            K.ckks_hrot(ctx, c3, 2, rk, out)          # key is for r = 1
        assert e.value.code == K.CKKS_ENOKEY
        with pytest.raises(K.CkksError) as e:
            K.ckks_hrot(ctx, c3, 1, rk, c3)           # aliasing
        assert e.value.code == K.CKKS_EINVAL
        with pytest.raises(K.CkksError) as e:
            K.ckks_hmult(ctx, c3, c3, rk, 4, out)     # unknown flag
        assert e.value.code == K.CKKS_EINVAL
    finally:
        for h in (c3, c4, c0, out, rk):
            K.ckks_free(h)


# ------------------------------------------------- execution lanes (clones) ---

def test_lanes_give_identical_results_concurrently(K, O):
    """Operations on clone contexts (own stream and scratch) running at the
    same time give the same residues as the oracle for each input."""
    import torch
    ctx, P = get(K, O, "n16d3")
    n_q = 12
    evk = rand_evk(P, 91)
    ek = K.ckks_evk_import(ctx, evk, 0)
    streams = [torch.cuda.Stream() for _ in range(3)]
    lanes = [K.ckks_ctx_clone(ctx, s.cuda_stream) for s in streams]
    hosts = [(rand_ct(P, n_q, 92 + 2 * i), rand_ct(P, n_q, 93 + 2 * i)) for i in range(3)]
    cts = [(K.ckks_ct_import(ctx, a, n_q - 1, 2.0**30), K.ckks_ct_import(ctx, b, n_q - 1, 2.0**30)) for a, b in hosts]
    outs = [K.ckks_ct_create(ctx, n_q - 1) for _ in lanes]
    try:
        torch.cuda.synchronize()
        for _ in range(3):   # several rounds so that the lanes overlap
            for lane, (a, b), out in zip(lanes, cts, outs):
                K.ckks_hmult(lane, a, b, ek, K.CKKS_RESCALE, out)
        for lane in lanes:
            K.ckks_sync(lane)
        for (a, b), out in zip(hosts, outs):
            got = K.ckks_ct_export(ctx, out, P.n)[0]
            assert np.array_equal(got, O.hmult(P, a, b, evk, rescale=True))
    finally:
        for a, b in cts:
            K.ckks_free(a)
            K.ckks_free(b)
        for h in outs + [ek]:
            K.ckks_free(h)
        for lane in lanes:
            K.ckks_ctx_destroy(lane)


# ------------------------------------------------------------ batched form ---

def test_headline_configuration_matches_oracle(K, O):
    """The launch configuration bench.py times, on sampled operations: N = 2^16,
    40 limbs at the top level, dnum = 3, tuned column shapes, HMult+rescale and
    HRot(1) of each ciphertext issued through the batch API over four lanes and
    replayed as one CUDA graph (twice): every output equals the oracle's."""
    ctx, P = get(K, O, "n16d3")
    n_q, nl = P.L, 4
    K.ckks_tune(ctx, n_q - 1, 1)
    relin, rotk = rand_evk(P, 501), rand_evk(P, 502)
    k1 = O.rot_k(1, P.log_n)
    ek_r, ek_g = K.ckks_evk_import(ctx, relin, 0), K.ckks_evk_import(ctx, rotk, k1)
    cts = [rand_ct(P, n_q, 510 + i) for i in range(3)]
    hs = [K.ckks_ct_import(ctx, c, n_q - 1, 2.0**30) for c in cts]
    outs = [K.ckks_ct_create(ctx, n_q - 1) for _ in range(4)]
    # as in the bench: a group of ciphertexts, their HMults on lanes 0.., then their HRots
    ops = [dict(op=K.CKKS_OP_HMULT, a=hs[i], b=hs[i + 1], evk=ek_r, flags=K.CKKS_RESCALE, out=outs[i])
           for i in range(2)]
    ops += [dict(op=K.CKKS_OP_HROT, a=hs[i], r=1, evk=ek_g, out=outs[2 + i]) for i in range(2)]
    batch = K.ckks_batch_create(ctx, ops, nl, True)
    try:
        K.ckks_batch_run(ctx, batch)
        K.ckks_batch_run(ctx, batch)
        K.ckks_sync(ctx)
        for i in range(2):
            assert np.array_equal(K.ckks_ct_export(ctx, outs[i], P.n)[0],
                                  O.hmult(P, cts[i], cts[i + 1], relin, rescale=True)), i
            assert np.array_equal(K.ckks_ct_export(ctx, outs[2 + i], P.n)[0], O.hrot(P, cts[i], k1, rotk)), i
    finally:
        K.ckks_batch_destroy(batch)
        for h in hs + outs + [ek_r, ek_g]:
            K.ckks_free(h)


@pytest.mark.parametrize("lanes,use_graph", [(1, False), (3, False), (3, True)])
def test_batch_mixed_levels_matches_oracle(K, O, lanes, use_graph):
    """Independent operations at mixed levels in one batch (direct or one CUDA
    graph launch, replayed twice): every output equals the oracle's."""
    ctx, P = get(K, O, "n16d3")
    rng = np.random.default_rng(101)
    relin = rand_evk(P, 102)
    rotk = rand_evk(P, 103)
    k1 = O.rot_k(1, P.log_n)
    ek_r = K.ckks_evk_import(ctx, relin, 0)
    ek_g = K.ckks_evk_import(ctx, rotk, k1)
    kinds = ["hmult_rs", "hrot", "pmult", "rescale", "hmult", "hadd"]
    handles, ops, want = [], [], []
    for i in range(8):
        kind = kinds[i % len(kinds)]
        n_q = int(rng.integers(2, 9))
        a = rand_ct(P, n_q, 200 + i)
        ha = K.ckks_ct_import(ctx, a, n_q - 1, 2.0**30)
        out = K.ckks_ct_create(ctx, n_q - 1)
        handles += [ha, out]
        if kind in ("hmult_rs", "hmult", "hadd"):
            b = rand_ct(P, n_q, 300 + i)
            hb = K.ckks_ct_import(ctx, b, n_q - 1, 2.0**30)
            handles.append(hb)
            if kind == "hadd":
                ops.append(dict(op=K.CKKS_OP_HADD, a=ha, b=hb, out=out))
                want.append(O.hadd(a, b, P.q[:n_q]))
            else:
                rs = kind == "hmult_rs"
                ops.append(dict(op=K.CKKS_OP_HMULT, a=ha, b=hb, evk=ek_r, flags=K.CKKS_RESCALE if rs else 0, out=out))
                want.append(O.hmult(P, a, b, relin, rescale=rs))
        elif kind == "hrot":
            ops.append(dict(op=K.CKKS_OP_HROT, a=ha, r=1, evk=ek_g, out=out))
            want.append(O.hrot(P, a, k1, rotk))
        elif kind == "pmult":
            pt = rand_poly(P, P.q[:n_q], 400 + i)
            hp = K.ckks_pt_import(ctx, pt, n_q - 1, 2.0**30)
            handles.append(hp)
            ops.append(dict(op=K.CKKS_OP_PMULT, a=ha, pt=hp, out=out))
            want.append(O.pmult(a, pt, P.q[:n_q]))
        else:
            ops.append(dict(op=K.CKKS_OP_RESCALE, a=ha, out=out))
            want.append(O.rescale(a, P.q[:n_q]))
    batch = K.ckks_batch_create(ctx, ops, lanes, use_graph)
    try:
        for _ in range(2):
            K.ckks_batch_run(ctx, batch)
            K.ckks_sync(ctx)
            for o, w in zip(ops, want):
                assert np.array_equal(K.ckks_ct_export(ctx, o["out"], P.n)[0], w)
    finally:
        K.ckks_batch_destroy(batch)
        for h in handles + [ek_r, ek_g]:
            K.ckks_free(h)


def test_batch_rejects_dependent_operations(K, O):
    ctx, P = get(K, O, "tiny")
    a = K.ckks_ct_import(ctx, rand_ct(P, 3, 501), 2, 2.0**30)
    b = K.ckks_ct_import(ctx, rand_ct(P, 3, 502), 2, 2.0**30)
    out = K.ckks_ct_create(ctx, 2)
    try:
        ops = [dict(op=K.CKKS_OP_HADD, a=a, b=b, out=out), dict(op=K.CKKS_OP_HADD, a=out, b=b, out=a)]
        with pytest.raises(K.CkksError) as e:
            K.ckks_batch_create(ctx, ops, 2, True)
        assert e.value.code == K.CKKS_EINVAL
    finally:
        for h in (a, b, out):
            K.ckks_free(h)
