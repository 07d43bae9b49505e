"""Pins of the oracle's CKKS operations against big-integer CRT, closed forms,
ring identities and decryption (Sec. 2.1-2.3 of the paper)."""
from fractions import Fraction
import math

import numpy as np
import pytest

from paper_2407_13055_gb300 import inputs


def _prod(ps):
    r = 1
    for v in ps:
        r *= int(v)
    return r


def _crt(res_col, primes):
    """Centered CRT lift of one coefficient's residues (Python integers)."""
    Q = _prod(primes)
    x = 0
    for r, qi in zip(res_col, primes):
        qi = int(qi)
        qh = Q // qi
        x += int(r) * qh * pow(qh % qi, -1, qi)
    x %= Q
    return x - Q if x > Q // 2 else x


def _centered(v, m):
    v %= m
    return v - m if v > m // 2 else v


def _check_fast_conversion(x_cols, src, out_cols, dst):
    """out == X + u*Qs (mod every dst prime) for one integer u, |u| <= K/2,
    and u == round(sum_j y_j / s_j) (the fast conversion's exact error)."""
    Qs = _prod(src)
    K = len(src)
    for xc, oc in zip(x_cols, out_cols):
        X = _crt(xc, src)
        us = {_centered((int(o) - X) * pow(Qs % int(d), -1, int(d)), int(d)) for o, d in zip(oc, dst)}
        assert len(us) == 1
        u = us.pop()
        assert abs(u) <= K / 2
        s = Fraction(0)
        for r, sj in zip(xc, src):
            sj = int(sj)
            y = _centered(int(r) * pow((Qs // sj) % sj, -1, sj), sj)
            s += Fraction(y, sj)
        assert u == round(s)


def test_bconv_is_crt_plus_bounded_multiple(O):
    log_n = 6
    q, p = O.gen_primes(log_n, 9, 4)
    rng = np.random.default_rng(1)
    for src, dst in [(q[:1], p), (q[:5], np.concatenate([q[5:], p])), (p, q)]:
        x = np.stack([rng.integers(0, int(v), 1 << log_n) for v in src]).astype(np.uint32)
        out = O.bconv(x, src, dst)
        _check_fast_conversion(x.T, src, out.T, dst)
        # centered representatives make the conversion odd: BConv(-x) = -BConv(x)
        neg = ((src[:, None].astype(np.int64) - x) % src[:, None]).astype(np.uint32)
        out_neg = O.bconv(neg, src, dst)
        assert ((out.astype(np.int64) + out_neg) % dst[:, None] == 0).all()


def test_bconv_extreme_inputs(O):
    log_n = 4
    q, p = O.gen_primes(log_n, 14, 8)
    src, dst = q, p
    n = 1 << log_n
    half = ((src - 1) // 2).astype(np.int64)
    x = np.zeros((len(src), n), np.int64)
    x[:, 0] = half
    x[:, 1] = src.astype(np.int64) - half
    x[:, 2] = 0
    x[:, 3] = src.astype(np.int64) - 1
    x = x.astype(np.uint32)
    out = O.bconv(x, src, dst)
    _check_fast_conversion(x.T[:4], src, out.T[:4], dst)


def _params(O, log_n, L, dnum, alpha=None):
    return O.make_params(log_n, L, dnum, alpha)


def test_modup_digits(O):
    P = _params(O, 6, 7, 3)  # alpha = 3, digits {0,1,2}, {3,4,5}, {6}
    rng = np.random.default_rng(2)
    for n_q in (7, 5, 1):
        d = np.stack([rng.integers(0, int(v), P.n) for v in P.q[:n_q]]).astype(np.uint32)
        up = O.modup(P, d, n_q)
        ext = P.ext_primes(n_q)
        coef_in = O.intt(d, P.q[:n_q])
        for j in range(P.digits(n_q)):
            lo, hi = j * P.alpha, min(n_q, (j + 1) * P.alpha)
            assert (up[j, lo:hi] == d[lo:hi]).all()
            others = [t for t in range(n_q + P.alpha) if not lo <= t < hi]
            coef_out = O.intt(up[j][others], ext[others])
            _check_fast_conversion(coef_in[lo:hi].T, P.q[lo:hi], coef_out.T, ext[others])


def test_keymult_definition(O):
    P = _params(O, 5, 5, 2)
    rng = np.random.default_rng(3)
    n_q = 4
    ext = P.ext_primes(n_q)
    up = np.stack([np.stack([rng.integers(0, int(v), P.n) for v in ext]) for _ in range(P.digits(n_q))]).astype(np.uint32)
    evk = np.stack([np.stack([np.stack([rng.integers(0, int(v), P.n) for v in P.all_primes()]) for _ in range(2)])
                    for _ in range(P.dnum)]).astype(np.uint32)
    acc = O.keymult(P, up, n_q, evk)
    key_limbs = list(range(n_q)) + [P.L + k for k in range(P.alpha)]
    for t in range(2):
        for li, kl in enumerate(key_limbs):
            s = np.zeros(P.n, dtype=object)
            for j in range(P.digits(n_q)):
                s = s + up[j, li].astype(object) * evk[j, t, kl].astype(object)
            assert [int(v) % int(ext[li]) for v in s] == acc[t, li].tolist()


def test_moddown_exact_division(O):
    P = _params(O, 5, 6, 2)  # alpha = 3
    rng = np.random.default_rng(4)
    n_q = 5
    ext = P.ext_primes(n_q)
    acc = np.stack([np.stack([rng.integers(0, int(v), P.n) for v in ext]) for _ in range(2)]).astype(np.uint32)
    out = O.moddown(P, acc, n_q)
    Pp = _prod(P.p)
    Q = _prod(P.q[:n_q])
    for t in range(2):
        ca = O.intt(acc[t], ext)
        co = O.intt(out[t], P.q[:n_q])
        for c in range(P.n):
            A = _crt(ca[:, c], ext)
            XP = _crt(ca[n_q:, c], P.p)
            w = A - XP
            assert w % Pp == 0
            o = _crt(co[:, c], P.q[:n_q])
            u = _centered(w // Pp - o, Q)
            assert abs(u) <= P.alpha / 2


@pytest.mark.parametrize("n_q", [2, 4, 6])
def test_rescale_is_rounded_division(O, n_q):
    log_n = 6
    q, _ = O.gen_primes(log_n, 6, 1)
    q = q[:n_q]
    rng = np.random.default_rng(n_q)
    ct = np.stack([np.stack([rng.integers(0, int(v), 1 << log_n) for v in q]) for _ in range(2)]).astype(np.uint32)
    out = O.rescale(ct, q)
    ql = int(q[-1])
    for t in range(2):
        ci = O.intt(ct[t], q)
        co = O.intt(out[t], q[:-1])
        for c in range(1 << log_n):
            X = _crt(ci[:, c], q)
            want = math.floor(Fraction(X, ql) + Fraction(1, 2))
            assert _crt(co[:, c], q[:-1]) == want


def _poly_mul(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        if a[i] == 0:
            continue
        for j in range(n):
            k = i + j
            if k < n:
                out[k] = (out[k] + a[i] * b[j]) % q
            else:
                out[k - n] = (out[k - n] - a[i] * b[j]) % q
    return out


def test_automorphism_is_ring_homomorphism(O):
    log_n = 5
    n = 1 << log_n
    q = O.gen_primes(log_n, 2, 1)[0][:2]
    rng = np.random.default_rng(6)
    for k in [O.rot_k(1, log_n), O.rot_k(3, log_n), O.conj_k(log_n), 1]:
        # phi(X) = X^k
        x = np.zeros((1, n), np.uint32)
        x[0, 1] = 1
        fx = O.automorph_coeff(x, q[:1], k)[0].tolist()
        want = [0] * n
        if k % (2 * n) < n:
            want[k % (2 * n)] = 1
        else:
            want[k % (2 * n) - n] = int(q[0]) - 1
        assert fx == want
        for qi in q:
            qi = int(qi)
            a = rng.integers(0, qi, n).astype(np.uint32)
            b = rng.integers(0, qi, n).astype(np.uint32)
            ab = np.array(_poly_mul(a.tolist(), b.tolist(), qi), np.uint32)
            fa = O.automorph_coeff(a[None], [qi], k)[0]
            fb = O.automorph_coeff(b[None], [qi], k)[0]
            assert O.automorph_coeff(ab[None], [qi], k)[0].tolist() == _poly_mul(fa.tolist(), fb.tolist(), qi)
            # the NTT-domain gather is the same map
            assert (O.ntt(fa[None], [qi])[0] == O.automorph_ntt(O.ntt(a[None], [qi]), k)[0]).all()
    # composition: phi_k o phi_k' = phi_{k k'}
    a = rng.integers(0, int(q[0]), n).astype(np.uint32)[None]
    k1, k2 = O.rot_k(1, log_n), O.rot_k(2, log_n)
    assert (O.automorph_ntt(O.automorph_ntt(a, k1), k1) == O.automorph_ntt(a, k2)).all()


def test_tensor_identity(O):
    log_n = 6
    q = O.gen_primes(log_n, 3, 1)[0]
    rng = np.random.default_rng(8)
    mk = lambda: np.stack([np.stack([rng.integers(0, int(v), 1 << log_n) for v in q]) for _ in range(2)]).astype(np.uint32)
    c1, c2 = mk(), mk()
    s = np.stack([rng.integers(0, int(v), 1 << log_n) for v in q]).astype(object)
    d = O.tensor(c1, c2, q).astype(object)
    Q = q[:, None].astype(object)
    lhs = (d[0] + d[1] * s + d[2] * s * s) % Q
    rhs = ((c1[0].astype(object) + c1[1] * s) * (c2[0].astype(object) + c2[1] * s)) % Q
    assert (lhs == rhs).all()


@pytest.mark.parametrize("log_n", [3, 4, 5])
def test_encode_matches_definition(O, log_n):
    u = inputs.messages(log_n, 1 << (log_n - 1))
    assert (O.encode_coeffs(u, 2.0**20, log_n) == O.encode_coeffs_naive(u, 2.0**20, log_n)).all()


def test_decode_inverts_encode(O):
    log_n = 12
    u = inputs.messages(1, 1 << (log_n - 1))
    scale = 2.0**28
    m = O.encode_coeffs(u, scale, log_n)
    back = O.decode_coeffs(m.astype(np.float64), scale, log_n)
    # rounding error 1/2 per coefficient -> at most N/2 / scale per slot
    assert np.max(np.abs(back - u)) <= (1 << log_n) / 2 / scale


# -----------------------------------------------------------------------------
# End-to-end: decrypt after each operation (Sec. 2.1 semantics)
# -----------------------------------------------------------------------------

def _keys(O, P, seed, h=None):
    s = inputs.ternary_secret(seed, P.n, h)
    allp = P.all_primes()

    def ks_inputs(stream):
        a = np.stack([inputs.uniform_residues(seed, allp, P.n, stream * 100 + j) for j in range(P.dnum)])
        e = np.stack([inputs.gaussian_error(seed, P.n, stream * 100 + j) for j in range(P.dnum)])
        return a, e
    return s, ks_inputs


def _enc(O, P, s, u, scale, n_q, seed, stream):
    pt = O.encode(P, u, scale, n_q)
    a = inputs.uniform_residues(seed, P.q[:n_q], P.n, 1000 + stream)
    e = inputs.gaussian_error(seed, P.n, 1000 + stream)
    return O.encrypt(P, s, pt, a, e)


TOY = [
    ("T1_alpha1_dnum4", 12, 4, 4, 1),
    ("T2_dnum1_alpha4", 12, 4, 1, 4),
]


@pytest.mark.parametrize("name,log_n,L,dnum,alpha", TOY)
def test_toy_hmult_hrot_hconj_decrypt(O, name, log_n, L, dnum, alpha):
    P = O.make_params(log_n, L, dnum, alpha)
    seed = 1
    s, ks = _keys(O, P, seed, None)
    scale = 2.0**28
    u = inputs.messages(seed, P.n // 2)
    v = inputs.messages(seed + 1, P.n // 2)
    ct1 = _enc(O, P, s, u, scale, L, seed, 1)
    ct2 = _enc(O, P, s, v, scale, L, seed, 2)
    # fresh decryption
    assert np.max(np.abs(O.decode(P, O.decrypt(P, s, ct1), scale) - u)) < 1e-3
    # HMult + relinearize + rescale
    a, e = ks(1)
    evk = O.keygen_relin(P, s, a, e)
    prod = O.hmult(P, ct1, ct2, evk, rescale=True)
    new_scale = scale * scale / float(P.q[L - 1])
    err = np.max(np.abs(O.decode(P, O.decrypt(P, s, prod), new_scale) - u * v))
    assert err < 1e-3, err
    # HRot by 1 (left rotation)
    a, e = ks(2)
    k = O.rot_k(1, log_n)
    rk = O.keygen_auto(P, s, k, a, e)
    rot = O.hrot(P, ct1, k, rk)
    err = np.max(np.abs(O.decode(P, O.decrypt(P, s, rot), scale) - np.roll(u, -1)))
    assert err < 1e-3, err
    # HConj
    a, e = ks(3)
    kc = O.conj_k(log_n)
    ck = O.keygen_auto(P, s, kc, a, e)
    cj = O.hrot(P, ct1, kc, ck)
    err = np.max(np.abs(O.decode(P, O.decrypt(P, s, cj), scale) - np.conj(u)))
    assert err < 1e-3, err
    # HAdd and PMult
    add = O.hadd(ct1, ct2, P.q[:L])
    assert np.max(np.abs(O.decode(P, O.decrypt(P, s, add), scale) - (u + v))) < 1e-3
    pm = O.pmult(ct1, O.encode(P, v, scale, L), P.q[:L])
    pm = O.rescale(pm, P.q[:L])
    err = np.max(np.abs(O.decode(P, O.decrypt(P, s, pm), new_scale) - u * v))
    assert err < 1e-3, err


def test_evk_decrypts_to_gadget_times_key(O):
    P = O.make_params(8, 4, 2)
    seed = 3
    s, ks = _keys(O, P, seed, None)
    a, e = ks(1)
    evk = O.keygen_relin(P, s, a, e)
    allp = P.all_primes()
    sh = O.small_to_ntt(s, allp, P.log_n).astype(np.uint64)
    s2 = sh * sh % allp[:, None]
    Pp = _prod(P.p)
    for j in range(P.dnum):
        b, aa = evk[j, 0].astype(np.uint64), evk[j, 1].astype(np.uint64)
        g = np.array([(Pp % int(v)) if (i < P.L and i // P.alpha == j) else 0 for i, v in enumerate(allp)],
                     dtype=np.uint64)
        noise_ntt = (b + aa * sh % allp[:, None] + (allp[:, None] - g[:, None] * s2 % allp[:, None])) % allp[:, None]
        noise = O.intt(noise_ntt.astype(np.uint32), allp)
        cen = np.where(noise > allp[:, None] // 2, noise.astype(np.int64) - allp[:, None], noise.astype(np.int64))
        assert (cen == e[j][None, :]).all()


def test_hrot_automorphism_order_is_bit_identical(O):
    """The paper's HRot order (ModUp -> KeyMult -> automorphism -> ModDown)
    with the key stored as phi^-1(evk) gives the same residues as the
    automorphism-first order, because BConv on centered values is odd."""
    P = O.make_params(6, 5, 2)
    rng = np.random.default_rng(9)
    n_q = 5
    k = O.rot_k(3, P.log_n)
    kinv = pow(k, -1, 2 * P.n)
    a = np.stack([rng.integers(0, int(v), P.n) for v in P.q[:n_q]]).astype(np.uint32)
    evk = np.stack([np.stack([np.stack([rng.integers(0, int(v), P.n) for v in P.all_primes()]) for _ in range(2)])
                    for _ in range(P.dnum)]).astype(np.uint32)
    first = O.keymult(P, O.modup(P, O.automorph_ntt(a, k), n_q), n_q, evk)
    evk_inv = np.stack([np.stack([O.automorph_ntt(evk[j, t], kinv) for t in range(2)]) for j in range(P.dnum)])
    acc = O.keymult(P, O.modup(P, a, n_q), n_q, evk_inv)
    after = np.stack([O.automorph_ntt(acc[t], k) for t in range(2)])
    assert (first == after).all()


@pytest.mark.parametrize("dnum", [3])
def test_config_n16_low_level_decrypt(O, dnum):
    """N = 2^16, 40 ciphertext primes, h = 192, at level 2 (three limbs)."""
    P = O.make_params(16, 40, dnum)
    seed = 5
    s, ks = _keys(O, P, seed, 192)
    scale = 2.0**30
    n_q = 3
    u = inputs.messages(seed, P.n // 2)
    v = inputs.messages(seed + 1, P.n // 2)
    ct1 = _enc(O, P, s, u, scale, n_q, seed, 1)
    ct2 = _enc(O, P, s, v, scale, n_q, seed, 2)
    a, e = ks(1)
    evk = O.keygen_relin(P, s, a, e)
    prod = O.hmult(P, ct1, ct2, evk, rescale=True)
    new_scale = scale * scale / float(P.q[n_q - 1])
    err = np.max(np.abs(O.decode(P, O.decrypt(P, s, prod), new_scale) - u * v))
    assert err < 1e-3, err
    a, e = ks(2)
    k = O.rot_k(5, P.log_n)
    rot = O.hrot(P, ct1, k, O.keygen_auto(P, s, k, a, e))
    err = np.max(np.abs(O.decode(P, O.decrypt(P, s, rot), scale) - np.roll(u, -5)))
    assert err < 1e-3, err


@pytest.mark.parametrize("name,log_n,L,dnum,alpha", TOY)
def test_linear_transform_decrypts_to_weighted_rotation_sum(O, name, log_n, L, dnum, alpha):
    """Par. 5 with one ModDown: decrypting sum_i d_i (.) HRot_{r_i}(ct) gives
    the slot-wise sum of d_i times u rotated left by r_i."""
    P = O.make_params(log_n, L, dnum, alpha)
    seed = 5
    s, ks = _keys(O, P, seed, None)
    scale = 2.0**28
    u = inputs.messages(seed, P.n // 2)
    ct = _enc(O, P, s, u, scale, L, seed, 1)
    rots = [0, 1, 3, 1]
    diags = [inputs.messages(50 + i, P.n // 2) for i in range(len(rots))]
    pts = [O.encode_ext(P, d, scale, L) for d in diags]
    evks = []
    for i, r in enumerate(rots):
        a, e = ks(10 + i)
        evks.append(O.keygen_auto(P, s, O.rot_k(r, log_n), a, e) if r else None)
    out = O.linear_transform(P, ct, rots, evks, pts)
    want = sum(d * np.roll(u, -r) for d, r in zip(diags, rots))
    err = np.max(np.abs(O.decode(P, O.decrypt(P, s, out), scale * scale) - want))
    assert err < 1e-3, err


def test_linear_transform_single_rotation_is_pmult_of_hrot_up_to_moddown(O):
    """One rotated term: ModDown(pt (.) KeyMult) and pt (.) ModDown(KeyMult)
    are both exact divisions by P of values congruent modulo Q_l, so they
    differ by a small integer polynomial only: the coefficient-domain
    difference is bounded (here by N * max|pt| / P-scale, far below q)."""
    P = O.make_params(8, 4, 2)
    rng = np.random.default_rng(3)
    n_q = 4
    ct = np.stack([np.stack([rng.integers(0, int(v), P.n) for v in P.q[:n_q]]) for _ in range(2)]).astype(np.uint32)
    evk = np.stack([np.stack([np.stack([rng.integers(0, int(v), P.n) for v in P.all_primes()]) for _ in range(2)])
                    for _ in range(P.dnum)]).astype(np.uint32)
    k = O.rot_k(1, P.log_n)
    m = rng.integers(-3, 4, P.n)                     # small plaintext coefficients
    pt_ext = O.small_to_ntt(m, list(P.q[:n_q]) + list(P.p), P.log_n)
    got = O.linear_transform(P, ct, [1], [evk], [pt_ext])
    ref = O.pmult(O.hrot(P, ct, k, evk), pt_ext[:n_q], P.q[:n_q])
    diff = (got.astype(np.int64) - ref.astype(np.int64)) % np.array(P.q[:n_q], np.int64)[None, :, None]
    coeff = O.intt(diff.reshape(2 * n_q, P.n).astype(np.uint32), list(P.q[:n_q]) * 2).reshape(2, n_q, P.n)
    for u_ in range(2):
        big = O.crt_centered(coeff[u_], P.q[:n_q])
        # |pt (.) rounding| <= N * max|m| * (alpha + 1) / 2 per coefficient (rounding in [-K/2, K/2] per limb)
        assert max(abs(int(x)) for x in big) <= P.n * 3 * (P.alpha + 2)


def test_merged_moddown_rescale_differs_by_a_small_polynomial(O):
    """HMult with ModDown merged into the rescaling (one division by P q_l)
    and the exact ModDown-then-rescale differ per coefficient by at most a
    few units: both are (Y - X) / (P q_l) with X of bounded size."""
    P = O.make_params(8, 6, 3)
    rng = np.random.default_rng(21)
    n_q = 6
    mk = lambda: np.stack([np.stack([rng.integers(0, int(v), P.n) for v in P.q[:n_q]]) for _ in range(2)]).astype(np.uint32)
    c1, c2 = mk(), mk()
    evk = np.stack([np.stack([np.stack([rng.integers(0, int(v), P.n) for v in P.all_primes()]) for _ in range(2)])
                    for _ in range(P.dnum)]).astype(np.uint32)
    merged = O.hmult_merged(P, c1, c2, evk)
    exact = O.hmult(P, c1, c2, evk, rescale=True)
    primes = [int(v) for v in P.q[:n_q - 1]]
    for u in range(2):
        diff = (merged[u].astype(np.int64) - exact[u].astype(np.int64)) % np.array(primes, np.int64)[:, None]
        coef = O.intt(diff.astype(np.uint32), primes)
        big = O.crt_centered(coef, primes)
        assert max(abs(int(x)) for x in big) <= P.alpha + 3


def test_merged_hmult_decrypts(O):
    P = O.make_params(12, 4, 4, 1)
    seed = 4
    s, ks = _keys(O, P, seed, None)
    scale = 2.0**28
    u = inputs.messages(seed, P.n // 2)
    v = inputs.messages(seed + 1, P.n // 2)
    ct1 = _enc(O, P, s, u, scale, P.L, seed, 1)
    ct2 = _enc(O, P, s, v, scale, P.L, seed, 2)
    a, e = ks(1)
    evk = O.keygen_relin(P, s, a, e)
    prod = O.hmult_merged(P, ct1, ct2, evk)
    err = np.max(np.abs(O.decode(P, O.decrypt(P, s, prod), scale * scale / float(P.q[P.L - 1])) - u * v))
    assert err < 1e-3, err
