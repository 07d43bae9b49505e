"""The 25-30 prime system (Sec. 3.2, Table 2) and rational rescaling in the
oracle, pinned against the paper's table, big-integer arithmetic and
decryption."""
import math
import os

import numpy as np
import pytest

from paper_2407_13055_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _table2():
    """Table 2 rows from tests/golden: (n_tau, n_q, log2 Q, log2 Delta or None) per level."""
    rows = []
    with open(os.path.join(GOLDEN, "table2_prime_system_2530.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                lv, nt, nq, lq, ld = line.split()
                assert int(lv) == len(rows)
                rows.append((int(nt), int(nq), int(lq), None if ld == "-" else int(ld)))
    return rows


TABLE2 = _table2()


def _window(P, lv):
    s, n = lv
    return [int(v) for v in P.q[s:s + n]]


@pytest.mark.parametrize("log_n", [6, 12, 16])
def test_prime_system_matches_table2(O, log_n):
    P, levels = O.prime_system_2530(log_n, 5)
    m = 2 << log_n
    allp = [int(v) for v in P.q] + [int(v) for v in P.p]
    assert len(set(allp)) == len(allp)
    for v in allp:
        assert v % m == 1 and O.is_prime(v)
    taus, qs = [int(v) for v in P.q[:4]], [int(v) for v in P.q[4:]]
    # "sufficiently close to 2^k": the candidates are 2N apart (2^17 at N = 2^16)
    assert all(abs(math.log2(t) - 25) < 0.2 for t in taus)
    assert all(abs(math.log2(q) - 30) < 0.3 for q in qs)
    for lv, (nt, nq, logq, _) in zip(levels, TABLE2):
        w = _window(P, lv)
        assert sum(1 for v in w if v in taus) == nt and sum(1 for v in w if v in qs) == nq
        assert abs(sum(math.log2(v) for v in w) - logq) < 0.5
    # every level is a contiguous window; the top level holds every prime (Q_max)
    assert levels[-1] == (0, len(P.q))


def test_rescaling_cycle_keeps_scale_within_a_tenth_of_a_bit(O):
    """Sec. 3.2: with the fixed prime order, Delta stays within 2^39.9 .. 2^40.1
    through the rescaling cycle (and ~2^55 at the double-rescaling levels)."""
    P, levels = O.prime_system_2530(16, 5)
    for top in (4, 8):
        logd = float(TABLE2[top][3])
        for lv in range(top, 0 if top == 4 else 5, -1):
            old, new = set(range(*_span(levels[lv]))), set(range(*_span(levels[lv - 1])))
            drop = sum(math.log2(int(P.q[g])) for g in old - new)
            add = sum(math.log2(int(P.q[g])) for g in new - old)
            logd = 2 * logd + add - drop          # HMult squares the scale, then the rescale
            want = float(TABLE2[lv - 1][3] if TABLE2[lv - 1][3] is not None else TABLE2[lv][3])
            assert abs(logd - want) < 0.1, (lv, logd)


def _span(lv):
    return lv[0], lv[0] + lv[1]


def _crt(res, primes):
    Q = math.prod(primes)
    x = 0
    for r, q in zip(res, primes):
        qh = Q // q
        x += int(r) * qh * pow(qh % q, -1, q)
    x %= Q
    return x - Q if x > Q // 2 else x


@pytest.mark.parametrize("step", [(4, 3), (3, 2), (2, 1), (1, 0), (8, 7), (5, 4)])
def test_rational_rescale_is_division_by_t_drop_times_t_add(O, step):
    """c' = (c T_add - X) / T_drop with X = c T_add (mod T_drop) and
    |X| <= (K/2 + 1/2) T_drop (fast BConv of K dropped primes), checked per
    coefficient in big integers."""
    P, levels = O.prime_system_2530(6, 5)
    (s0, n0), (s1, n1) = levels[step[0]], levels[step[1]]
    rng = np.random.default_rng(step[0])
    old = [int(v) for v in P.q[s0:s0 + n0]]
    new = [int(v) for v in P.q[s1:s1 + n1]]
    ct = np.stack([np.stack([rng.integers(0, q, P.n) for q in old]) for _ in range(2)]).astype(np.uint32)
    out = O.rescale_rational(P, ct, s0, n0, s1, n1)
    drop = [q for g, q in zip(range(s0, s0 + n0), old) if not s1 <= g < s1 + n1]
    add = [q for g, q in zip(range(s1, s1 + n1), new) if not s0 <= g < s0 + n0]
    t_drop, t_add, K = math.prod(drop), math.prod(add), len(drop)
    for u in range(2):
        c_coef = O.intt(ct[u], old)
        o_coef = O.intt(out[u], new)
        for k in range(0, P.n, 7):
            c = _crt([c_coef[i][k] for i in range(n0)], old)
            o = _crt([o_coef[i][k] for i in range(n1)], new)
            x = c * t_add - o * t_drop
            assert (x - c * t_add) % t_drop == 0
            assert abs(x) <= (K / 2 + 0.5) * t_drop


@pytest.mark.parametrize("merged", [False, True])
def test_hmult_through_the_rescaling_cycle_decrypts(O, merged):
    """Encrypt at level 4 (Delta = 2^40), square with HMult + rational
    rescaling down to level 0 (two steps, or ModDown merged into the
    rescaling, Sec. 6): every decryption is u^(2^k) within 1e-3. HRot at a
    window level decrypts to the rotation."""
    P, levels = O.prime_system_2530(10, 5)
    seed = 11
    s = inputs.ternary_secret(seed, P.n, None)
    allp = P.all_primes()
    a = np.stack([inputs.uniform_residues(seed, allp, P.n, 100 + j) for j in range(P.dnum)])
    e = np.stack([inputs.gaussian_error(seed, P.n, 100 + j) for j in range(P.dnum)])
    rk = O.keygen_relin(P, s, a, e)
    u = 0.9 * inputs.messages(seed, P.n // 2)
    sc = 2.0 ** 40
    s4, n4 = levels[4]
    m = O.encode_coeffs(u, sc, P.log_n)
    pt = O.small_to_ntt(m, [int(v) for v in P.q[s4:s4 + n4]], P.log_n)
    ai = inputs.uniform_residues(seed, [int(v) for v in P.q[s4:s4 + n4]], P.n, 7)
    ct = _encrypt_window(O, P, s, pt, ai, inputs.gaussian_error(seed, P.n, 7), s4, n4)
    want = u.copy()
    for lv in range(4, 0, -1):
        (so, no), (sn, nn) = levels[lv], levels[lv - 1]
        if merged:
            ct = O.hmult_merged(P, ct, ct, rk, base=so, new=(sn, nn))
        else:
            prod = O.hmult(P, ct, ct, rk, rescale=False, base=so)
            ct = O.rescale_rational(P, prod, so, no, sn, nn)
        drop = [int(P.q[g]) for g in range(so, so + no) if not sn <= g < sn + nn]
        add = [int(P.q[g]) for g in range(sn, sn + nn) if not so <= g < so + no]
        sc = sc * sc * math.prod(add) / math.prod(drop)
        want = want * want
        got = _decrypt_window(O, P, s, ct, sn, nn, sc)
        assert np.max(np.abs(got - want)) < 1e-3, lv
    if merged:
        return
    # HRot by 3 at level 3 (window base 2)
    a2 = np.stack([inputs.uniform_residues(seed, allp, P.n, 200 + j) for j in range(P.dnum)])
    e2 = np.stack([inputs.gaussian_error(seed, P.n, 200 + j) for j in range(P.dnum)])
    k = O.rot_k(3, P.log_n)
    gk = O.keygen_auto(P, s, k, a2, e2)
    s3, n3 = levels[3]
    pt3 = O.small_to_ntt(O.encode_coeffs(u, 2.0 ** 40, P.log_n), [int(v) for v in P.q[s3:s3 + n3]], P.log_n)
    ai3 = inputs.uniform_residues(seed, [int(v) for v in P.q[s3:s3 + n3]], P.n, 9)
    c3 = _encrypt_window(O, P, s, pt3, ai3, inputs.gaussian_error(seed, P.n, 9), s3, n3)
    rot = O.hrot(P, c3, k, gk, base=s3)
    got = _decrypt_window(O, P, s, rot, s3, n3, 2.0 ** 40)
    assert np.max(np.abs(got - np.roll(u, -3))) < 1e-3


@pytest.mark.parametrize("step", [(4, 3), (1, 0), (8, 7), (5, 4)])
def test_merged_moddown_rescale_is_near_the_two_step_result(O, step):
    """ModDown merged into the rational rescaling (one division by P T_drop)
    and ModDown followed by the rational rescaling agree per coefficient to
    within a few units (both approximate c P^-1 T_add / T_drop, Sec. 3.2,
    Sec. 6); random ciphertexts and keys."""
    P, levels = O.prime_system_2530(6, 5)
    (s0, n0), (s1, n1) = levels[step[0]], levels[step[1]]
    rng = np.random.default_rng(40 + step[0])
    old = [int(v) for v in P.q[s0:s0 + n0]]
    new = [int(v) for v in P.q[s1:s1 + n1]]
    mk = lambda: np.stack([np.stack([rng.integers(0, q, P.n) for q in old]) for _ in range(2)]).astype(np.uint32)
    c1, c2 = mk(), mk()
    evk = np.stack([np.stack([np.stack([rng.integers(0, int(v), P.n) for v in P.all_primes()]) for _ in range(2)])
                    for _ in range(P.dnum)]).astype(np.uint32)
    merged = O.hmult_merged(P, c1, c2, evk, base=s0, new=(s1, n1))
    two = O.rescale_rational(P, O.hmult(P, c1, c2, evk, rescale=False, base=s0), s0, n0, s1, n1)
    K = sum(1 for g in range(s0, s0 + n0) if not s1 <= g < s1 + n1)
    for u in range(2):
        diff = (merged[u].astype(np.int64) - two[u].astype(np.int64)) % np.array(new, np.int64)[:, None]
        coef = O.intt(diff.astype(np.uint32), new)
        assert max(abs(int(x)) for x in O.crt_centered(coef, new)) <= P.alpha + K + 3


def _encrypt_window(O, P, s, pt, a, e, base, n):
    primes = [int(v) for v in P.q[base:base + n]]
    sh = O.small_to_ntt(s, primes, P.log_n).astype(np.uint64)
    eh = O.small_to_ntt(e, primes, P.log_n).astype(np.uint64)
    qc = np.array(primes, np.uint64)[:, None]
    a = a.astype(np.uint64)
    b = (pt.astype(np.uint64) + eh + (qc - a * sh % qc)) % qc
    return np.stack([b, a]).astype(np.uint32)


def _decrypt_window(O, P, s, ct, base, n, scale):
    primes = [int(v) for v in P.q[base:base + n]]
    sh = O.small_to_ntt(s, primes, P.log_n).astype(np.uint64)
    qc = np.array(primes, np.uint64)[:, None]
    m = (ct[0].astype(np.uint64) + ct[1].astype(np.uint64) * sh % qc) % qc
    coef = O.intt(m.astype(np.uint32), primes)
    big = O.crt_centered(coef, primes)
    return O.decode_coeffs(np.array([float(b) for b in big]), scale, P.log_n)


# ---------------------------------------------------------------------------
# Hybrid key switching on a window q[s .. s+n) that does not start at prime 0
# (the levels of the 25-30 system, Table 2). The digits are the fixed groups of
# alpha consecutive primes of the whole list (Sec. 2.3 with the level's window
# cut out of them), so a window starting inside a group opens with a partial
# digit; the evaluation key of a digit is the one of its global group. These
# pins recompute the cut from the global prime index and check each step with
# big-integer CRT arithmetic.

def _prod(ps):
    r = 1
    for v in ps:
        r *= int(v)
    return r


def _crt(res, primes):
    Q = _prod(primes)
    x = 0
    for r, qi in zip(res, primes):
        qi = int(qi)
        qh = Q // qi
        x += int(r) * qh * pow(qh % qi, -1, qi)
    x %= Q
    return x - Q if x > Q // 2 else x


def _cent(v, m):
    v %= m
    return v - m if v > m // 2 else v


def _groups(P, s, n):
    """Global digit index of each window limb, and the active digits in order."""
    g = [(s + t) // P.alpha for t in range(n)]
    return g, sorted(set(g))


# (alpha, level window): windows opening inside a group, on a group boundary,
# and with a first global digit above 0 (alpha = 2, 3, 4), so that a cut taken
# relative to the window or a key indexed by the window's digit number differs.
WINDOWS = [(5, (2, 2)), (5, (4, 7)), (5, (1, 13)), (4, (4, 3)), (3, (4, 7)), (3, (2, 11)), (2, (3, 9))]


@pytest.mark.parametrize("alpha,lv", WINDOWS)
def test_windowed_modup_cuts_digits_at_global_groups(O, alpha, lv):
    """ModUp on a window: digit j copies the window limbs of global group g_j
    and converts them (Eq. 2, centered) to every other window prime and P; the
    converted value is X + u*Q_j with |u| <= |group|/2."""
    P, _ = O.prime_system_2530(5, alpha)
    s, n = lv
    g, active = _groups(P, s, n)
    assert P.digits(n, s) == len(active)
    rng = np.random.default_rng(60 + alpha * 256 + s * 16 + n)
    win = [int(v) for v in P.q[s:s + n]]
    ext = win + [int(v) for v in P.p]
    d = np.stack([rng.integers(0, q, P.n) for q in win]).astype(np.uint32)
    up = O.modup(P, d, n, base=s)
    assert up.shape == (len(active), n + P.alpha, P.n)
    coef = O.intt(d, win)
    for j, gj in enumerate(active):
        own = [t for t in range(n) if g[t] == gj]
        assert (up[j, own] == d[own]).all()
        others = [t for t in range(n + P.alpha) if t not in own]
        src = [win[t] for t in own]
        dst = [ext[t] for t in others]
        Qs = _prod(src)
        out = O.intt(up[j][others], np.array(dst, np.uint32))
        for c in range(0, P.n, 3):
            X = _crt([int(coef[t, c]) for t in own], src)
            us = {_cent((int(out[i, c]) - X) * pow(Qs % dt, -1, dt), dt) for i, dt in enumerate(dst)}
            assert len(us) == 1
            assert abs(us.pop()) <= len(own) / 2


@pytest.mark.parametrize("alpha,lv", WINDOWS)
def test_windowed_keymult_uses_the_global_digit_key(O, alpha, lv):
    """KeyMult on a window: limb t of the window takes key limb s+t, limb k of
    P takes key limb L+k, and digit j multiplies the key of global group g_j."""
    P, _ = O.prime_system_2530(5, alpha)
    s, n = lv
    _, active = _groups(P, s, n)
    rng = np.random.default_rng(80 + alpha * 256 + s * 16 + n)
    ext = [int(v) for v in P.q[s:s + n]] + [int(v) for v in P.p]
    up = np.stack([np.stack([rng.integers(0, q, P.n) for q in ext]) for _ in active]).astype(np.uint32)
    allp = [int(v) for v in P.all_primes()]
    evk = np.stack([np.stack([np.stack([rng.integers(0, q, P.n) for q in allp]) for _ in range(2)])
                    for _ in range(P.dnum)]).astype(np.uint32)
    acc = O.keymult(P, up, n, evk, base=s)
    key = [s + t for t in range(n)] + [P.L + k for k in range(P.alpha)]
    for t in range(2):
        for li, kl in enumerate(key):
            tot = np.zeros(P.n, dtype=object)
            for j, gj in enumerate(active):
                tot = tot + up[j, li].astype(object) * evk[gj, t, kl].astype(object)
            assert [int(v) % ext[li] for v in tot] == acc[t, li].tolist()


@pytest.mark.parametrize("alpha,lv", WINDOWS)
def test_windowed_moddown_is_division_by_p(O, alpha, lv):
    """ModDown on a window: out = (A - BConv(A mod P)) / P over the window's
    primes, i.e. round(A / P) up to the conversion's |u| <= alpha/2 multiples
    of the window modulus."""
    P, _ = O.prime_system_2530(5, alpha)
    s, n = lv
    rng = np.random.default_rng(100 + alpha * 256 + s * 16 + n)
    win = [int(v) for v in P.q[s:s + n]]
    pp = [int(v) for v in P.p]
    ext = win + pp
    acc = np.stack([np.stack([rng.integers(0, q, P.n) for q in ext]) for _ in range(2)]).astype(np.uint32)
    out = O.moddown(P, acc, n, base=s)
    Pp, Q = _prod(pp), _prod(win)
    for t in range(2):
        ca = O.intt(acc[t], np.array(ext, np.uint32))
        co = O.intt(out[t], np.array(win, np.uint32))
        for c in range(0, P.n, 3):
            A = _crt([int(v) for v in ca[:, c]], ext)
            XP = _crt([int(v) for v in ca[n:, c]], pp)
            assert (A - XP) % Pp == 0
            o = _crt([int(v) for v in co[:, c]], win)
            assert abs(_cent((A - XP) // Pp - o, Q)) <= P.alpha / 2
