"""CPU oracle for the 32-bit RNS-CKKS key-switch path (Cheddar, arxiv 2407.13055).

TEST INFRASTRUCTURE ONLY. Tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it; the CUDA library never imports it.

The integer arithmetic lives in ``ckks_oracle.cpp`` (plain C++, built with g++
by :func:`build`); this module wraps it with numpy arrays and adds the
floating-point encoding (Sec. 2.1: u in C^{N/2} -> <Delta u> in R_Q) and the
big-integer CRT lift used by decoding, both written plainly in Python.

Parity unpinned: none. Every function is pinned by ``tests/test_oracle_*.py``
against schoolbook products, big-integer CRT, closed forms or brute force.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import math

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libckks_oracle.so")
_lock = threading.Lock()
_lib = None

U32P = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
I64P = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the C++ oracle into a shared library (g++, -O2, portable flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            i, u32, u64, i64 = C.c_int, C.c_uint32, C.c_uint64, C.c_int64
            sig = {
                "or_is_prime": (i, [u64]),
                "or_gen_primes": (i, [i, i, i, U32P, U32P]),
                "or_find_psi": (u32, [u32, i]),
                "or_smr": (C.c_int32, [i64, u32]),
                "or_ntt_naive": (None, [U32P, U32P, i, u32]),
                "or_intt_naive": (None, [U32P, U32P, i, u32]),
                "or_ntt": (None, [U32P, i, U32P, i]),
                "or_intt": (None, [U32P, i, U32P, i]),
                "or_bconv": (None, [U32P, i, U32P, U32P, i, U32P, i]),
                "or_automorph_ntt": (None, [U32P, U32P, i, i, u32]),
                "or_automorph_coeff": (None, [U32P, U32P, i, U32P, i, u32]),
                "or_tensor": (None, [U32P, U32P, i, U32P, i, U32P]),
                "or_modup": (None, [i, i, U32P, i, U32P, i, i, U32P, i, U32P]),
                "or_keymult": (None, [i, i, U32P, i, U32P, i, i, U32P, i, U32P, U32P]),
                "or_moddown": (None, [i, i, U32P, i, U32P, i, i, U32P, i, U32P]),
                "or_rescale_rational": (None, [U32P, i, U32P, i, i, i, i, i, U32P]),
                "or_hmult_merged": (None, [i, i, U32P, i, U32P, i, i, U32P, U32P, i, U32P, i, i, U32P]),
                "or_rescale": (None, [U32P, i, i, U32P, i, U32P]),
                "or_hmult": (None, [i, i, U32P, i, U32P, i, i, U32P, U32P, i, U32P, i, U32P]),
                "or_hrot": (None, [i, i, U32P, i, U32P, i, i, U32P, i, u32, U32P, U32P]),
                "or_hadd": (None, [U32P, U32P, i, U32P, i, U32P]),
                "or_pmult": (None, [U32P, U32P, i, U32P, i, U32P]),
                "or_small_to_ntt": (None, [I64P, i, U32P, i, U32P]),
                "or_encrypt": (None, [I64P, U32P, I64P, U32P, i, U32P, i, U32P]),
                "or_decrypt": (None, [I64P, U32P, i, U32P, i, U32P]),
                "or_keygen_ks": (None, [i, i, U32P, i, U32P, i, I64P, U32P, U32P, I64P, U32P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _i64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int64)


# ----------------------------------------------------------------------------
# Parameters
# ----------------------------------------------------------------------------

@dataclass
class Params:
    """RNS-CKKS parameters: N = 2^log_n, L ciphertext primes q, alpha auxiliary
    primes p, dnum digits of alpha primes each (Sec. 2.1, Table 1)."""
    log_n: int
    q: np.ndarray
    p: np.ndarray
    dnum: int

    @property
    def n(self) -> int:
        return 1 << self.log_n

    @property
    def L(self) -> int:
        return len(self.q)

    @property
    def alpha(self) -> int:
        return len(self.p)

    def ext_primes(self, n_q: int) -> np.ndarray:
        return np.concatenate([self.q[:n_q], self.p]).astype(np.uint32)

    def all_primes(self) -> np.ndarray:
        return self.ext_primes(self.L)

    def digits(self, n_q: int, base: int = 0) -> int:
        """Digits active in the window [base, base + n_q) of the prime list."""
        return (base + n_q - 1) // self.alpha - base // self.alpha + 1

    def args(self):
        return (self.log_n, self.L, _u32(self.q), self.alpha, _u32(self.p), self.dnum)


def gen_primes(log_n: int, n_q: int, n_p: int):
    """The prime rule (reading of Eq. 3): q_0 the largest prime = 1 mod 2N below
    2^31, q_1.. the largest below 2^30, p_0.. the next below 2^31."""
    q = np.zeros(max(n_q, 1), np.uint32)
    p = np.zeros(max(n_p, 1), np.uint32)
    if lib().or_gen_primes(log_n, n_q, n_p, q, p) != 0:
        raise ValueError("not enough NTT-friendly primes")
    return q[:n_q].copy(), p[:n_p].copy()


def make_params(log_n: int, L: int, dnum: int, alpha: int | None = None) -> Params:
    """Parameters of the prime rule (reading of Eq. 3): L ciphertext primes,
    alpha = ceil(L / dnum) auxiliary primes unless given (Sec. 2.3 gadget)."""
    if alpha is None:
        alpha = -(-L // dnum)
    q, p = gen_primes(log_n, L, alpha)
    return Params(log_n, q, p, dnum)


def is_prime(v: int) -> bool:
    """Deterministic primality of v (the prime rule of Eq. 3 needs q prime)."""
    return bool(lib().or_is_prime(int(v)))


def find_psi(q: int, log_n: int) -> int:
    """Smallest psi with psi^N = -1 mod q: the primitive 2N-th root of the
    negacyclic NTT (Eq. 3)."""
    return int(lib().or_find_psi(int(q), log_n))


def smr(x: int, q: int) -> int:
    """Signed Montgomery reduction of x (Alg. 2): x 2^-32 mod q in (-q, q)."""
    return int(lib().or_smr(int(x), int(q)))


# ----------------------------------------------------------------------------
# Polynomial operations (integer; wrappers around the C++ core)
# ----------------------------------------------------------------------------

def ntt_naive(a, q: int, log_n: int) -> np.ndarray:
    """O(N^2) negacyclic NTT, A_i = sum_k a_k psi^((2i+1)k) (Eq. 3), natural order."""
    out = np.zeros(1 << log_n, np.uint32)
    lib().or_ntt_naive(_u32(a), out, log_n, int(q))
    return out


def intt_naive(a, q: int, log_n: int) -> np.ndarray:
    """O(N^2) inverse of ntt_naive (Eq. 3)."""
    out = np.zeros(1 << log_n, np.uint32)
    lib().or_intt_naive(_u32(a), out, log_n, int(q))
    return out


def ntt(a, primes) -> np.ndarray:
    """Fast negacyclic NTT per limb (Eq. 3, natural order); limb i modulo primes[i]."""
    a = _u32(a).copy()
    primes = _u32(primes)
    log_n = int(a.shape[-1]).bit_length() - 1
    lib().or_ntt(a, len(primes), primes, log_n)
    return a


def intt(a, primes) -> np.ndarray:
    """Fast inverse negacyclic NTT per limb (Eq. 3)."""
    a = _u32(a).copy()
    primes = _u32(primes)
    log_n = int(a.shape[-1]).bit_length() - 1
    lib().or_intt(a, len(primes), primes, log_n)
    return a


def bconv(x, src, dst) -> np.ndarray:
    """Fast basis conversion (Eq. 2) with centered y_j (Sec. 4.2), coefficient domain."""
    x = _u32(x)
    src, dst = _u32(src), _u32(dst)
    log_n = int(x.shape[-1]).bit_length() - 1
    out = np.zeros((len(dst), x.shape[-1]), np.uint32)
    lib().or_bconv(x, len(src), src, out, len(dst), dst, log_n)
    return out


def automorph_ntt(a, k: int) -> np.ndarray:
    """Automorphism X -> X^k on NTT-domain limbs (Eq. 4): an index permutation."""
    a = _u32(a)
    log_n = int(a.shape[-1]).bit_length() - 1
    limbs = a.size >> log_n
    out = np.zeros_like(a)
    lib().or_automorph_ntt(a, out, limbs, log_n, int(k))
    return out


def automorph_coeff(a, primes, k: int) -> np.ndarray:
    """Automorphism X -> X^k on coefficients (Eq. 4 stated on coefficients)."""
    a = _u32(a)
    primes = _u32(primes)
    log_n = int(a.shape[-1]).bit_length() - 1
    out = np.zeros_like(a)
    lib().or_automorph_coeff(a, out, len(primes), primes, log_n, int(k))
    return out


def rot_k(r: int, log_n: int) -> int:
    """Galois element of a left rotation by r slots: 5^r mod 2N (Eq. 4)."""
    return pow(5, int(r) % (1 << (log_n - 1)), 2 << log_n)


def conj_k(log_n: int) -> int:
    """Galois element of the conjugation (Sec. 2.1): 2N - 1."""
    return (2 << log_n) - 1


def tensor(ct1, ct2, q) -> np.ndarray:
    """HMult tensor (Sec. 2.1): d0 = b1 b2, d1 = a1 b2 + a2 b1, d2 = a1 a2 (NTT domain)."""
    ct1, ct2, q = _u32(ct1), _u32(ct2), _u32(q)
    n_q, n = ct1.shape[1], ct1.shape[2]
    out = np.zeros((3, n_q, n), np.uint32)
    lib().or_tensor(ct1, ct2, n_q, q, n.bit_length() - 1, out)
    return out


def modup(P: Params, d, n_q: int, base: int = 0) -> np.ndarray:
    """ModUp (Alg. 1, Eq. 2) of the window q[base .. base + n_q); digits are the
    fixed groups of alpha consecutive primes of the whole list, cut to the window."""
    d = _u32(d)
    out = np.zeros((P.digits(n_q, base), n_q + P.alpha, P.n), np.uint32)
    lib().or_modup(*P.args(), base, d, n_q, out)
    return out


def keymult(P: Params, up, n_q: int, evk, base: int = 0) -> np.ndarray:
    """KeyMult + MAC (Sec. 2.3, Par. 1): acc_t = sum_j ModUp_j[t] evk_j[t] over the
    extended primes of the window and P."""
    out = np.zeros((2, n_q + P.alpha, P.n), np.uint32)
    lib().or_keymult(*P.args(), base, _u32(up), n_q, _u32(evk), out)
    return out


def moddown(P: Params, acc, n_q: int, base: int = 0) -> np.ndarray:
    """ModDown (Sec. 2.3): (acc_Q - BConv_{P->Q}(acc_P)) P^-1 on the window."""
    out = np.zeros((2, n_q, P.n), np.uint32)
    lib().or_moddown(*P.args(), base, _u32(acc), n_q, out)
    return out


# ----------------------------------------------------------------------------
# 25-30 prime system (Sec. 3.2, Table 2)
# ----------------------------------------------------------------------------

def _primes_near(center_bits: int, count: int, log_n: int):
    """The `count` primes q = 1 mod 2N nearest to 2^center_bits (ties: the
    smaller one first), with log2(q) - center_bits."""
    m = 2 << log_n
    c = 1 << center_bits
    up = (c // m + 1) * m + 1
    dn = (c // m) * m + 1
    if dn >= c:
        dn -= m
    found = []
    while len(found) < count:
        for v in (dn, up):
            if is_prime(v):
                found.append(v)
        up += m
        dn -= m
    found.sort(key=lambda v: (abs(v - c), v))
    return found[:count]


def prime_system_2530(log_n: int, alpha: int):
    """The exemplar 25-30 prime system of Table 2 (Delta ~ 2^40 at levels 1-4,
    double rescaling with Delta ~ 2^55 at the bootstrapping levels 5-8).

    Returns (Params, levels): the prime list in inverted-terminal order
    [tau_3, tau_2, tau_1, tau_0, q_0, ..., q_10] (Sec. 3.3), which makes every
    level a contiguous window, and levels[l] = (first index, count) of level l.
    Rescaling cycle (Sec. 3.2): 4 -> 3 drops q_4..q_6 and adds tau_1, tau_0;
    3 -> 2 drops q_1..q_3 and adds tau_3, tau_2; 2 -> 1 drops the four taus
    and adds q_1, q_2; 1 -> 0 drops q_0..q_2 and adds tau_1, tau_0; levels 5-8
    add {tau_i, q_(7+i)} by double rescaling.

    Reading of the "carefully chosen lists" (the paper gives no rule): the
    taus are the four primes = 1 mod 2N nearest to 2^25 (tau_0 nearest); with
    b_i = log2(tau_i) - 25 and a_i = log2(q_i) - 30, each q_i is the unused
    prime = 1 mod 2N near 2^30 whose a_i is nearest to the value that makes
    every rescaling of the cycle divide by exactly 2^40 (2^55 at the double
    rescalings): a_0 = -(b_2 + b_3), a_1 = a_2 = (b_0 + .. + b_3) / 2,
    a_3 = -(b_0 + b_1), a_4 = a_5 = a_6 = (b_0 + b_1) / 3, a_(7+i) = -b_i.
    The auxiliary primes are the largest 31-bit primes = 1 mod 2N."""
    t25 = _primes_near(25, 4, log_n)
    b = [math.log2(t) - 25 for t in t25]
    pool = _primes_near(30, 200, log_n)
    targets = [-(b[2] + b[3]), sum(b) / 2, sum(b) / 2, -(b[0] + b[1])] + [(b[0] + b[1]) / 3] * 3 + \
        [-b[0], -b[1], -b[2], -b[3]]
    used, q30 = set(), []
    for tgt in targets:
        best = min((v for v in pool if v not in used), key=lambda v: (abs(math.log2(v) - 30 - tgt), v))
        used.add(best)
        q30.append(best)
    g = [t25[3], t25[2], t25[1], t25[0]] + q30
    m = 2 << log_n
    p, c = [], ((1 << 31) - 1) // m * m + 1
    while len(p) < alpha:
        if is_prime(c) and c not in g:
            p.append(c)
        c -= m
    levels = [(2, 2), (4, 3), (0, 5), (2, 6), (4, 7), (3, 9), (2, 11), (1, 13), (0, 15)]
    dnum = -(-len(g) // alpha)
    return Params(log_n, np.array(g, np.uint32), np.array(p, np.uint32), dnum), levels


def rescale_rational(P: Params, ct, s_old: int, n_old: int, s_new: int, n_new: int) -> np.ndarray:
    """Rational rescaling from window [s_old, s_old + n_old) of the prime list
    to [s_new, s_new + n_new) (Sec. 3.1, Sec. 3.2, Sec. 5.1)."""
    ct = _u32(ct)
    polys = ct.shape[0]
    out = np.zeros((polys, n_new, P.n), np.uint32)
    lib().or_rescale_rational(ct, polys, _u32(P.q), s_old, n_old, s_new, n_new, P.log_n, out)
    return out


def rescale(ct, q) -> np.ndarray:
    """Rescale (Sec. 2.1): c_i = (c_i - [c_l]_centered) q_l^-1 mod q_i, i < l."""
    ct, q = _u32(ct), _u32(q)
    polys, n_q, n = ct.shape
    out = np.zeros((polys, n_q - 1, n), np.uint32)
    lib().or_rescale(ct, polys, n_q, q, n.bit_length() - 1, out)
    return out


def hmult(P: Params, ct1, ct2, evk, rescale: bool = True, base: int = 0) -> np.ndarray:
    """HMult (Sec. 2.1, Sec. 2.3): tensor, then (d0, d1) + KeySwitch(d2) with
    ModUp, KeyMult and ModDown, optionally rescaled by the top prime."""
    ct1, ct2 = _u32(ct1), _u32(ct2)
    n_q = ct1.shape[1]
    out = np.zeros((2, n_q - (1 if rescale else 0), P.n), np.uint32)
    lib().or_hmult(*P.args(), base, ct1, ct2, n_q, _u32(evk), int(bool(rescale)), out)
    return out


def hmult_merged(P: Params, ct1, ct2, evk, base: int = 0, new=None) -> np.ndarray:
    """HMult with ModDown merged into the rescaling (the MAD merge that
    Sec. 6 extends to its prime system): one conversion from P and the
    dropped primes of (KeyMult + P d) T_add, divided by P T_drop. The level's
    window starts at `base`; `new` = (start, count) of the next level's window
    (default: the usual rescaling by the top prime)."""
    ct1, ct2 = _u32(ct1), _u32(ct2)
    n_q = ct1.shape[1]
    s_new, n_new = new if new is not None else (base, n_q - 1)
    out = np.zeros((2, n_new, P.n), np.uint32)
    lib().or_hmult_merged(*P.args(), base, ct1, ct2, n_q, _u32(evk), s_new, n_new, out)
    return out


def hrot(P: Params, ct, k: int, evk, base: int = 0) -> np.ndarray:
    """HRot / HConj (Sec. 2.3, Eq. 4): (phi_k(b), 0) + KeySwitch(phi_k(a))."""
    ct = _u32(ct)
    n_q = ct.shape[1]
    out = np.zeros((2, n_q, P.n), np.uint32)
    lib().or_hrot(*P.args(), base, ct, n_q, int(k), _u32(evk), out)
    return out


def encode_ext(P: Params, u, scale: float, n_q: int) -> np.ndarray:
    """Extended plaintext (Par. 4, Par. 5): the encoding's integer coefficients reduced modulo
    q_0..q_{n_q-1} and then p_0..p_{alpha-1}, NTT domain [n_q + alpha][N]."""
    m = encode_coeffs(u, scale, P.log_n)
    return small_to_ntt(m, list(P.q[:n_q]) + list(P.p), P.log_n)


def linear_transform(P: Params, ct, rots, evks, pts_ext, base: int = 0) -> np.ndarray:
    """Linear transform sum_i pt_i (.) HRot_{r_i}(ct) with a shared ModUp and
    one ModDown (Par. 4, Par. 5; the hoisting of the cited linear-transform
    method). With M_j = ModUp_j(a) (Alg. 1) and phi_i the automorphism of r_i
    (Eq. 4), over the terms with r_i != 0:
        acc_u = sum_i pt_i (.) sum_j phi_i(M_j) (.) evk_i[j][u]   in basis Q_l P
        out_0 = ModDown(acc)_0 + sum_i pt_i (.) phi_i(b)           (all terms)
        out_1 = ModDown(acc)_1 + sum_{i: r_i = 0} pt_i (.) a
    pts_ext[i]: [n_q + alpha][N] NTT-domain residues (Q limbs, then P limbs);
    evks[i] is ignored for r_i = 0."""
    ct = _u32(ct)
    n_q = ct.shape[1]
    qcol = np.array(P.q[base:base + n_q], np.uint64)[:, None]
    ecol = np.array(list(P.q[base:base + n_q]) + list(P.p), np.uint64)[:, None]
    b, a = ct[0].astype(np.uint64), ct[1].astype(np.uint64)
    out = np.zeros((2, n_q, P.n), np.uint64)
    acc = np.zeros((2, n_q + P.alpha, P.n), np.uint64)
    up = None
    rotated = False
    for r, evk, pt in zip(rots, evks, pts_ext):
        pt = np.asarray(pt, np.uint64)
        k = rot_k(r, P.log_n)
        if k == 1:
            out[0] = (out[0] + pt[:n_q] * b) % qcol
            out[1] = (out[1] + pt[:n_q] * a) % qcol
            continue
        if up is None:
            up = modup(P, ct[1], n_q, base)
        rotated = True
        upk = np.stack([automorph_ntt(up[j], k) for j in range(up.shape[0])])
        km = keymult(P, upk, n_q, evk, base).astype(np.uint64)
        acc = (acc + km * pt[None]) % ecol[None]
        bk = automorph_ntt(ct[0], k).astype(np.uint64)
        out[0] = (out[0] + pt[:n_q] * bk) % qcol
    if rotated:
        out = (out + moddown(P, acc.astype(np.uint32), n_q, base).astype(np.uint64)) % qcol[None]
    return out.astype(np.uint32)


def hadd(x, y, q) -> np.ndarray:
    """HAdd (Sec. 2.1): limb-wise sum modulo each prime."""
    x, y = _u32(x), _u32(y)
    out = np.zeros_like(x)
    lib().or_hadd(x, y, x.shape[1], _u32(q), x.shape[2].bit_length() - 1, out)
    return out


def pmult(x, pt, q) -> np.ndarray:
    """PMult (Sec. 2.1): NTT-domain product of each ciphertext polynomial with pt."""
    x, pt = _u32(x), _u32(pt)
    out = np.zeros_like(x)
    lib().or_pmult(x, pt, x.shape[1], _u32(q), x.shape[2].bit_length() - 1, out)
    return out


def small_to_ntt(v, primes, log_n: int) -> np.ndarray:
    """Signed small integer coefficients reduced modulo each prime, then NTT (Eq. 3)."""
    primes = _u32(primes)
    out = np.zeros((len(primes), 1 << log_n), np.uint32)
    lib().or_small_to_ntt(_i64(v), len(primes), primes, log_n, out)
    return out


# ----------------------------------------------------------------------------
# Keys and encryption (Eq. 1); random inputs come from the input generators
# ----------------------------------------------------------------------------

def encrypt(P: Params, s, pt, a, e) -> np.ndarray:
    """Symmetric encryption (Eq. 1): (b, a) = (-a s + e + pt, a), NTT domain."""
    pt = _u32(pt)
    n_q = pt.shape[0]
    out = np.zeros((2, n_q, P.n), np.uint32)
    lib().or_encrypt(_i64(s), _u32(a), _i64(e), pt, n_q, _u32(P.q[:n_q]), P.log_n, out)
    return out


def decrypt(P: Params, s, ct) -> np.ndarray:
    """Decryption (Sec. 2.1): b + a s, NTT domain."""
    ct = _u32(ct)
    n_q = ct.shape[1]
    out = np.zeros((n_q, P.n), np.uint32)
    lib().or_decrypt(_i64(s), ct, n_q, _u32(P.q[:n_q]), P.log_n, out)
    return out


def keygen_ks(P: Params, s, s_from_ntt, a, e) -> np.ndarray:
    """Key-switching key (Sec. 2.3, gadget [P]_{q_i} on the digit limbs)
    [dnum][2][L+alpha][N] from s_from (NTT domain) to s."""
    out = np.zeros((P.dnum, 2, P.L + P.alpha, P.n), np.uint32)
    lib().or_keygen_ks(*P.args(), _i64(s), _u32(s_from_ntt), _u32(a), _i64(e), out)
    return out


def keygen_relin(P: Params, s, a, e) -> np.ndarray:
    """Relinearization key (Sec. 2.3): key switching from s^2 to s."""
    sh = small_to_ntt(s, P.all_primes(), P.log_n)
    s2 = ((sh.astype(np.uint64) * sh) % P.all_primes()[:, None].astype(np.uint64)).astype(np.uint32)
    return keygen_ks(P, s, s2, a, e)


def keygen_auto(P: Params, s, k: int, a, e) -> np.ndarray:
    """Key for phi_k(s) -> s (Eq. 4; rotation k = 5^r, conjugation k = 2N-1)."""
    sh = small_to_ntt(s, P.all_primes(), P.log_n)
    return keygen_ks(P, s, automorph_ntt(sh, k), a, e)


# ----------------------------------------------------------------------------
# Encoding (Sec. 2.1): slot j <-> zeta^(5^j mod 2N), zeta = exp(i pi / N)
# ----------------------------------------------------------------------------

def _slot_exponents(log_n: int) -> np.ndarray:
    n = 1 << log_n
    e = np.empty(n // 2, dtype=np.int64)
    v = 1
    for j in range(n // 2):
        e[j] = v
        v = v * 5 % (2 * n)
    return e


def encode_coeffs(u, scale: float, log_n: int) -> np.ndarray:
    """Encoding (Sec. 2.1): round(Delta * sigma^-1(u)) as int64 coefficients (half away from zero).

    sigma^-1: the real polynomial m with m(zeta^(5^j)) = u_j and
    m(zeta^(-5^j)) = conj(u_j); m_k = (1/N) sum_{o odd} z_o zeta^(-o k),
    i.e. zeta^-k (1/N) sum_j z_(2j+1) exp(-2 pi i j k / N): a length-N forward
    FFT (numpy) followed by the twist zeta^-k.
    """
    n = 1 << log_n
    e = _slot_exponents(log_n)
    z = np.zeros(2 * n, dtype=np.complex128)
    z[e] = u
    z[(2 * n - e) % (2 * n)] = np.conj(u)
    zo = z[1::2]                              # z at zeta^(2j+1)
    k = np.arange(n)
    m = np.exp(-1j * np.pi * k / n) * np.fft.fft(zo) / n
    v = np.real(m) * scale
    return (np.sign(v) * np.floor(np.abs(v) + 0.5)).astype(np.int64)


def decode_coeffs(m, scale: float, log_n: int) -> np.ndarray:
    """Decoding (Sec. 2.1): slots u_j = m(zeta^(5^j)) / Delta from real coefficients m."""
    n = 1 << log_n
    k = np.arange(n)
    tw = np.asarray(m, dtype=np.float64) * np.exp(1j * np.pi * k / n)
    zo = np.fft.ifft(tw) * n                  # z_(2j+1) = sum_k m_k zeta^((2j+1)k)
    e = _slot_exponents(log_n)
    return zo[(e - 1) // 2] / scale


def encode_coeffs_naive(u, scale: float, log_n: int) -> np.ndarray:
    """O(N^2) definition of encode_coeffs (Sec. 2.1; small N only)."""
    n = 1 << log_n
    e = _slot_exponents(log_n)
    zeta = np.exp(1j * np.pi / n)
    m = np.zeros(n)
    for k in range(n):
        s = 0j
        for j in range(n // 2):
            s += u[j] * zeta ** (-(int(e[j]) * k)) + np.conj(u[j]) * zeta ** (int(e[j]) * k)
        m[k] = (s / n).real * scale
    return (np.sign(m) * np.floor(np.abs(m) + 0.5)).astype(np.int64)


def crt_centered(res, primes) -> list:
    """Centered CRT lift (Sec. 2.1, RNS) of residues [n][N] to Python integers in (-Q/2, Q/2]."""
    primes = [int(v) for v in primes]
    Q = 1
    for v in primes:
        Q *= v
    out = [0] * res.shape[1]
    for i, qi in enumerate(primes):
        qh = Q // qi
        c = qh * pow(qh % qi, -1, qi)
        col = res[i].astype(object)
        out = [o + int(x) * c for o, x in zip(out, col)]
    half = Q // 2
    return [(o % Q) - Q if (o % Q) > half else o % Q for o in out]


def encode(P: Params, u, scale: float, n_q: int) -> np.ndarray:
    """Encoding (Sec. 2.1) to a plaintext in the NTT domain [n_q][N]."""
    m = encode_coeffs(u, scale, P.log_n)
    return small_to_ntt(m, P.q[:n_q], P.log_n)


def decode(P: Params, pt, scale: float) -> np.ndarray:
    """Decoding (Sec. 2.1) of an NTT-domain plaintext: iNTT, centered CRT lift, slots."""
    pt = _u32(pt)
    n_q = pt.shape[0]
    coef = intt(pt, P.q[:n_q])
    big = crt_centered(coef, P.q[:n_q])
    return decode_coeffs(np.array([float(b) for b in big]), scale, P.log_n)
