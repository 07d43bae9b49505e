"""Pins of the oracle's arithmetic against facts fixed outside it.

* primality against sympy; the prime-list rule (Eq. 3, q < 2^31) by scanning;
* psi (a primitive 2N-th root) by brute force;
* SMR (Alg. 2) against Python big integers, with its input/output ranges;
* the negacyclic NTT (Sec. 2.2) against schoolbook products in
  Z_q[X]/(X^N+1) and against Horner evaluation at psi^(2i+1).
"""
import os
import random

import numpy as np
import pytest

sympy = pytest.importorskip("sympy")


def test_is_prime_matches_sympy(O):
    rng = random.Random(7)
    vals = [0, 1, 2, 3, 4, 61, 97, 2**31 - 1, 2**32 - 5, 4294967291, 3215031751, 25326001]
    vals += [rng.randrange(2**32) for _ in range(3000)]
    vals += [rng.randrange(2**30, 2**31) | 1 for _ in range(3000)]
    for v in vals:
        assert O.is_prime(v) == sympy.isprime(v), v


@pytest.mark.parametrize("log_n,L,alpha", [(12, 4, 4), (16, 40, 14)])
def test_prime_rule(O, log_n, L, alpha):
    q, p = O.gen_primes(log_n, L, alpha)
    m = 2 << log_n
    allp = [int(v) for v in q] + [int(v) for v in p]
    assert len(set(allp)) == len(allp)
    for v in allp:
        assert sympy.isprime(v) and v % m == 1 and v < 2**31
    # q_0 and the auxiliary primes: the 1 + alpha largest below 2^31, in order
    top = [v for v in range((2**31 - 1) // m * m + 1, 2**30, -m) if sympy.isprime(v)][: 1 + alpha]
    assert [int(q[0])] + [int(v) for v in p] == top
    # q_1..q_{L-1}: the largest below 2^30, decreasing
    below = []
    v = (2**30 - 1) // m * m + 1
    while len(below) < L - 1:
        if sympy.isprime(v):
            below.append(v)
        v -= m
    assert [int(x) for x in q[1:]] == below


def test_psi_is_smallest_primitive_root(O):
    for log_n, q in [(3, 17), (3, 97), (4, 97), (5, 193), (12, None), (16, None)]:
        if q is None:
            q = int(O.gen_primes(log_n, 2, 1)[0][1])
        n = 1 << log_n
        psi = O.find_psi(q, log_n)
        assert pow(psi, n, q) == q - 1 and pow(psi, 2 * n, q) == 1
        for x in range(2, psi):
            assert pow(x, n, q) != q - 1


def _table3_ranges():
    """Output ranges of Table 3 (tests/golden), keyed by method."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "table3_reduction_methods.txt")
    out = {}
    with open(path) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                method, _, _, rng = line.split()
                out[method] = rng
    return out


def test_smr_definition_and_range(O):
    """Alg. 2 returns x 2^-32 mod q in the output range Table 3 prints for the
    signed Montgomery reduction, (-q, q), for every x in [-q 2^31, q 2^31)."""
    assert _table3_ranges()["signed_montgomery"] == "(-q,q)"
    rng = random.Random(11)
    qs = [int(v) for v in O.gen_primes(16, 4, 2)[0]] + [int(v) for v in O.gen_primes(16, 1, 2)[1]] + [97, 12289]
    for q in qs:
        lo, hi = -q * 2**31, q * 2**31 - 1
        xs = [lo, hi, 0, -1, 1, lo + 1, hi - 1] + [rng.randint(lo, hi) for _ in range(20000)]
        for x in xs:
            y = O.smr(x, q)
            assert -q < y < q
            assert (y * 2**32 - x) % q == 0


def _schoolbook_negacyclic(a, b, q):
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                out[k] = (out[k] + a[i] * b[j]) % q
            else:
                out[k - n] = (out[k - n] - a[i] * b[j]) % q
    return out


@pytest.mark.parametrize("log_n", [3, 4, 5, 6])
def test_ntt_convolution_matches_schoolbook(O, log_n):
    rng = np.random.default_rng(log_n)
    qs = [int(O.gen_primes(log_n, 3, 1)[0][i]) for i in range(3)]
    n = 1 << log_n
    for q in qs:
        a = rng.integers(0, q, n).astype(np.uint32)
        b = rng.integers(0, q, n).astype(np.uint32)
        fa, fb = O.ntt_naive(a, q, log_n), O.ntt_naive(b, q, log_n)
        prod = (fa.astype(np.uint64) * fb % q).astype(np.uint32)
        got = O.intt_naive(prod, q, log_n)
        assert got.tolist() == _schoolbook_negacyclic(a.tolist(), b.tolist(), q)
        # the same through the fast transform
        fa2 = O.ntt(a[None], [q])[0]
        fb2 = O.ntt(b[None], [q])[0]
        got2 = O.intt((fa2.astype(np.uint64) * fb2 % q).astype(np.uint32)[None], [q])[0]
        assert got2.tolist() == got.tolist()


@pytest.mark.parametrize("log_n", [3, 5, 8])
def test_ntt_is_evaluation_at_odd_powers_in_natural_order(O, log_n):
    rng = np.random.default_rng(100 + log_n)
    q = int(O.gen_primes(log_n, 2, 1)[0][1])
    n = 1 << log_n
    psi = O.find_psi(q, log_n)
    a = rng.integers(0, q, n).astype(np.uint32)
    got = O.ntt(a[None], [q])[0]
    for i in range(n):
        x = pow(psi, 2 * i + 1, q)
        acc = 0
        for c in reversed(a.tolist()):      # Horner
            acc = (acc * x + c) % q
        assert int(got[i]) == acc


@pytest.mark.parametrize("log_n", [4, 7, 10])
def test_fast_ntt_equals_definition(O, log_n):
    rng = np.random.default_rng(log_n)
    q, p = O.gen_primes(log_n, 3, 2)
    for pr in list(q) + list(p):
        pr = int(pr)
        a = rng.integers(0, pr, 1 << log_n).astype(np.uint32)
        assert (O.ntt(a[None], [pr])[0] == O.ntt_naive(a, pr, log_n)).all()
        assert (O.intt(a[None], [pr])[0] == O.intt_naive(a, pr, log_n)).all()


def test_ntt_roundtrip_large(O):
    q, p = O.gen_primes(16, 3, 2)
    prs = np.concatenate([q, p])
    rng = np.random.default_rng(5)
    a = np.stack([rng.integers(0, int(v), 1 << 16) for v in prs]).astype(np.uint32)
    assert (O.intt(O.ntt(a, prs), prs) == a).all()
