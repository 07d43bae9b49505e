"""Python binding of libckks_gb300.so (the C ABI in include/ckks.h).

Argument marshalling only: every step of the key-switch path runs in the
library's CUDA kernels. Importing this module loads the in-tree shared
library and raises if it has not been built (``__graft_entry__.build()``);
there is no fallback implementation.

Functions keep the C names. Handles are ``ctypes.c_void_p`` values; numpy
arrays are passed as host buffers in the canonical layout documented in the
header.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libckks_gb300.so")

CKKS_OK = 0
CKKS_EINVAL = -1
CKKS_ELEVEL = -2
CKKS_ESCALE = -3
CKKS_ENOKEY = -4
CKKS_ENOMEM = -5
CKKS_ECUDA = -6
CKKS_ETIMEOUT = -7
CKKS_EBUSY = -8
CKKS_ERANGE = -9
CKKS_RESCALE = 1
CKKS_RESCALE_MERGED = 2


class CkksError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"ckks error {code}: {msg}")
        self.code = code


class ckks_params(C.Structure):
    _fields_ = [
        ("log_n", C.c_int),
        ("n_q", C.c_int),
        ("q", C.POINTER(C.c_uint32)),
        ("n_p", C.c_int),
        ("p", C.POINTER(C.c_uint32)),
        ("dnum", C.c_int),
        ("scale", C.c_double),
        ("secret_hw", C.c_int),
        ("sigma", C.c_double),
        ("seed", C.c_uint64),
        ("n_levels", C.c_int),
        ("level_first", C.POINTER(C.c_int)),
        ("level_count", C.POINTER(C.c_int)),
    ]


class ckks_op(C.Structure):
    _fields_ = [
        ("op", C.c_int),
        ("flags", C.c_int),
        ("r", C.c_int),
        ("a", C.c_void_p),
        ("b", C.c_void_p),
        ("pt", C.c_void_p),
        ("evk", C.c_void_p),
        ("out", C.c_void_p),
    ]


CKKS_OP_HMULT, CKKS_OP_HROT, CKKS_OP_HCONJ, CKKS_OP_PMULT, CKKS_OP_RESCALE, CKKS_OP_HADD, CKKS_OP_PADD = 1, 2, 3, 4, 5, 6, 7


class ckks_request(C.Structure):
    _fields_ = [
        ("op", C.c_int),
        ("r", C.c_int),
        ("arrival_s", C.c_double),
        ("a", C.c_void_p),
        ("b", C.c_void_p),
        ("evk", C.c_void_p),
        ("out", C.c_void_p),
        ("bytes", C.c_size_t),
    ]


class ckks_request_done(C.Structure):
    _fields_ = [("start_s", C.c_double), ("end_s", C.c_double), ("lane", C.c_int)]


_ISSUE_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int, C.c_int)
_QUERY_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, C.c_int)


class ckks_serve_hooks(C.Structure):
    _fields_ = [("issue", _ISSUE_FN), ("query", _QUERY_FN), ("user", C.c_void_p)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build the CUDA library first (__graft_entry__.build())")

lib = C.CDLL(LIB_PATH)

_vp, _i, _u32, _u64, _d, _sz = C.c_void_p, C.c_int, C.c_uint32, C.c_uint64, C.c_double, C.c_size_t
_P = C.POINTER
_SIGS = {
    "ckks_gen_primes": (_i, [_i, _i, _i, _vp, _vp]),
    "ckks_gen_prime_system_2530": (_i, [_i, _i, _vp, _vp, _vp, _vp]),
    "ckks_level_limbs": (_i, [_vp, _i]),
    "ckks_ctx_create": (_i, [_P(ckks_params), _vp, _P(_vp)]),
    "ckks_ctx_destroy": (None, [_vp]),
    "ckks_ctx_clone": (_i, [_vp, _vp, _P(_vp)]),
    "ckks_last_error": (C.c_char_p, [_vp]),
    "ckks_sync": (_i, [_vp]),
    "ckks_free": (None, [_vp]),
    "ckks_ctx_device_bytes": (_sz, [_vp]),
    "ckks_set_memory_limit": (_i, [_vp, _sz]),
    "ckks_memory_in_use": (_sz, [_vp]),
    "ckks_request_bytes": (_sz, [_vp, _i, _i]),
    "ckks_pool_create": (_i, [_sz, _P(_vp)]),
    "ckks_pool_acquire": (_i, [_vp, _sz]),
    "ckks_pool_release": (_i, [_vp, _sz]),
    "ckks_pool_in_use": (_sz, [_vp]),
    "ckks_pool_destroy": (None, [_vp]),
    "ckks_keygen_secret": (_i, [_vp, _u64, _P(_vp)]),
    "ckks_sk_import": (_i, [_vp, _vp, _P(_vp)]),
    "ckks_keygen_relin": (_i, [_vp, _vp, _u64, _P(_vp)]),
    "ckks_keygen_rot": (_i, [_vp, _vp, _i, _u64, _P(_vp)]),
    "ckks_keygen_conj": (_i, [_vp, _vp, _u64, _P(_vp)]),
    "ckks_evk_import": (_i, [_vp, _vp, _u32, _P(_vp)]),
    "ckks_encode": (_i, [_vp, _vp, _i, _d, _P(_vp)]),
    "ckks_decode": (_i, [_vp, _vp, _vp]),
    "ckks_encrypt": (_i, [_vp, _vp, _vp, _u64, _P(_vp)]),
    "ckks_decrypt": (_i, [_vp, _vp, _vp, _P(_vp)]),
    "ckks_ct_create": (_i, [_vp, _i, _P(_vp)]),
    "ckks_ct_import": (_i, [_vp, _vp, _i, _d, _P(_vp)]),
    "ckks_ct_export": (_i, [_vp, _vp, _vp, _sz, _P(_i), _P(_d)]),
    "ckks_ct_upload": (_i, [_vp, _vp, _vp, _i, _d]),
    "ckks_ct_upload_async": (_i, [_vp, _vp, _vp, _i, _d]),
    "ckks_ct_export_async": (_i, [_vp, _vp, _vp, _sz]),
    "ckks_ct_wrap_device": (_i, [_vp, _vp, _i, _d, _P(_vp)]),
    "ckks_ct_info": (_i, [_vp, _P(_i), _P(_d), _P(_vp)]),
    "ckks_pt_import": (_i, [_vp, _vp, _i, _d, _P(_vp)]),
    "ckks_pt_export": (_i, [_vp, _vp, _vp, _sz, _P(_i), _P(_d)]),
    "ckks_hadd": (_i, [_vp, _vp, _vp, _vp]),
    "ckks_pmult": (_i, [_vp, _vp, _vp, _vp]),
    "ckks_padd": (_i, [_vp, _vp, _vp, _vp]),
    "ckks_hmult": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "ckks_rescale": (_i, [_vp, _vp, _vp]),
    "ckks_hrot": (_i, [_vp, _vp, _i, _vp, _vp]),
    "ckks_hconj": (_i, [_vp, _vp, _vp, _vp]),
    "ckks_hrot_hoisted": (_i, [_vp, _vp, _i, _vp, _vp, _vp]),
    "ckks_linear_transform": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "ckks_encode_ext": (_i, [_vp, _vp, _i, _d, _P(_vp)]),
    "ckks_pt_import_ext": (_i, [_vp, _vp, _i, _d, _P(_vp)]),
    "ckks_rescale_noalloc": (_i, [_vp, _vp, _i, _vp]),
    "ckks_batch_create": (_i, [_vp, _vp, _i, _i, _i, _P(_vp)]),
    "ckks_batch_run": (_i, [_vp]),
    "ckks_batch_run_admit": (_i, [_vp, _i]),
    "ckks_batch_admit": (_i, [_vp, _i]),
    "ckks_batch_destroy": (None, [_vp]),
    "ckks_serve_run": (_i, [_vp, _i, _vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "ckks_set_launch_flags": (_i, [_vp, _i]),
    "ckks_set_wait_limit": (_i, [_vp, C.c_longlong]),
    "ckks_tune": (_i, [_vp, _i, _i]),
    "ckks_tune_get": (_i, [_vp, _i, _i, _P(_i), _P(_i), _P(_i), _P(_i), _P(C.c_float)]),
    "ckks_tune_set": (_i, [_vp, _i, _i, _i, _i, _i, _i]),
    "ckks_bench_modmul": (_i, [_vp, _i, _i, _u32, _vp, _i, _i, _vp, _P(C.c_float)]),
    "ckks_bench_intop": (_i, [_vp, _i, _i, _P(C.c_double), _P(C.c_float)]),
    "ckks_profile": (_i, [_vp, _i]),
    "ckks_profile_read": (_i, [_vp, _vp, _vp]),
    "ckks_profile_name": (C.c_char_p, [_i]),
    "ckks_launch_count": (_u64, []),
    "ckks_step_smr": (_i, [_vp, _vp, _i, _i, _vp]),
    "ckks_step_ntt": (_i, [_vp, _vp, _i, _vp, _i]),
    "ckks_step_bconv": (_i, [_vp, _vp, _i, _vp, _vp, _i, _vp, _i]),
    "ckks_step_tensor": (_i, [_vp, _vp, _vp, _i, _vp]),
    "ckks_step_automorph": (_i, [_vp, _vp, _i, _u32, _vp]),
    "ckks_step_modup": (_i, [_vp, _vp, _i, _vp]),
    "ckks_step_keyswitch_acc": (_i, [_vp, _vp, _i, _vp, _vp]),
    "ckks_step_moddown": (_i, [_vp, _vp, _i, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


def check(ctx, rc: int):
    if rc != CKKS_OK:
        msg = lib.ckks_last_error(ctx).decode() if ctx else ""
        raise CkksError(rc, msg)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


# ---------------------------------------------------------------------------
# Thin wrappers (same names as the C functions)
# ---------------------------------------------------------------------------

def ckks_gen_primes(log_n: int, n_q: int, n_p: int):
    q = np.zeros(n_q, np.uint32)
    p = np.zeros(max(n_p, 1), np.uint32)
    check(None, lib.ckks_gen_primes(log_n, n_q, n_p, _ptr(q), _ptr(p)))
    return q, p[:n_p].copy()


def ckks_gen_prime_system_2530(log_n: int, n_p: int):
    """(q [15], p [n_p], levels [(first, count)] x 9) of the exemplar 25-30 system."""
    q = np.zeros(15, np.uint32)
    p = np.zeros(n_p, np.uint32)
    lf = np.zeros(9, np.int32)
    lc = np.zeros(9, np.int32)
    check(None, lib.ckks_gen_prime_system_2530(log_n, n_p, _ptr(q), _ptr(p), _ptr(lf), _ptr(lc)))
    return q, p, list(zip(lf.tolist(), lc.tolist()))


def ckks_ctx_create(log_n: int, q, p, dnum: int, scale: float = 2.0**30, secret_hw: int = 0,
                    sigma: float = 3.2, seed: int = 0, stream: int | None = None, levels=None):
    """levels: None (single rescaling) or a list of (first, count) windows of
    the prime list, one per level (rational rescaling between them)."""
    q, p = _u32(q), _u32(p)
    nl = 0 if levels is None else len(levels)
    lf = (C.c_int * max(nl, 1))(*[int(a) for a, _ in (levels or [])])
    lc = (C.c_int * max(nl, 1))(*[int(b) for _, b in (levels or [])])
    prm = ckks_params(log_n, len(q), q.ctypes.data_as(_P(C.c_uint32)), len(p), p.ctypes.data_as(_P(C.c_uint32)),
                      dnum, scale, secret_hw, sigma, seed, nl, lf, lc)
    out = _vp()
    rc = lib.ckks_ctx_create(C.byref(prm), stream, C.byref(out))
    check(None, rc)
    return out


def ckks_level_limbs(ctx, level: int) -> int:
    n = lib.ckks_level_limbs(ctx, level)
    if n < 0:
        check(ctx, n)
    return n


def ckks_ctx_destroy(ctx):
    lib.ckks_ctx_destroy(ctx)


def ckks_ctx_clone(parent, stream: int | None = None):
    out = _vp()
    check(parent, lib.ckks_ctx_clone(parent, stream, C.byref(out)))
    return out


def ckks_free(h):
    lib.ckks_free(h)


def ckks_sync(ctx):
    check(ctx, lib.ckks_sync(ctx))


def ckks_keygen_secret(ctx, seed: int):
    out = _vp()
    check(ctx, lib.ckks_keygen_secret(ctx, seed, C.byref(out)))
    return out


def ckks_sk_import(ctx, coeffs):
    c = np.ascontiguousarray(coeffs, dtype=np.int64)
    out = _vp()
    check(ctx, lib.ckks_sk_import(ctx, _ptr(c), C.byref(out)))
    return out


def ckks_keygen_relin(ctx, sk, seed: int):
    out = _vp()
    check(ctx, lib.ckks_keygen_relin(ctx, sk, seed, C.byref(out)))
    return out


def ckks_keygen_rot(ctx, sk, r: int, seed: int):
    out = _vp()
    check(ctx, lib.ckks_keygen_rot(ctx, sk, r, seed, C.byref(out)))
    return out


def ckks_keygen_conj(ctx, sk, seed: int):
    out = _vp()
    check(ctx, lib.ckks_keygen_conj(ctx, sk, seed, C.byref(out)))
    return out


def ckks_evk_import(ctx, evk, galois: int):
    e = _u32(evk)
    out = _vp()
    check(ctx, lib.ckks_evk_import(ctx, _ptr(e), galois, C.byref(out)))
    return out


def ckks_encode(ctx, u, level: int, scale: float):
    u = np.asarray(u, dtype=np.complex128)
    ri = np.ascontiguousarray(np.stack([u.real, u.imag], axis=1).reshape(-1))
    out = _vp()
    check(ctx, lib.ckks_encode(ctx, _ptr(ri), level, scale, C.byref(out)))
    return out


def ckks_encode_ext(ctx, u, level: int, scale: float):
    u = np.asarray(u, dtype=np.complex128)
    ri = np.ascontiguousarray(np.stack([u.real, u.imag], axis=1).reshape(-1))
    out = _vp()
    check(ctx, lib.ckks_encode_ext(ctx, _ptr(ri), level, scale, C.byref(out)))
    return out


def ckks_decode(ctx, pt, n_slots: int) -> np.ndarray:
    ri = np.zeros(2 * n_slots, np.float64)
    check(ctx, lib.ckks_decode(ctx, pt, _ptr(ri)))
    return ri[0::2] + 1j * ri[1::2]


def ckks_encrypt(ctx, sk, pt, seed: int):
    out = _vp()
    check(ctx, lib.ckks_encrypt(ctx, sk, pt, seed, C.byref(out)))
    return out


def ckks_decrypt(ctx, sk, ct):
    out = _vp()
    check(ctx, lib.ckks_decrypt(ctx, sk, ct, C.byref(out)))
    return out


def ckks_ct_create(ctx, capacity_level: int):
    out = _vp()
    check(ctx, lib.ckks_ct_create(ctx, capacity_level, C.byref(out)))
    return out


def ckks_ct_import(ctx, host, level: int, scale: float):
    h = _u32(host)
    out = _vp()
    check(ctx, lib.ckks_ct_import(ctx, _ptr(h), level, scale, C.byref(out)))
    return out


def ckks_ct_upload(ctx, ct, host, level: int, scale: float):
    h = _u32(host)
    check(ctx, lib.ckks_ct_upload(ctx, ct, _ptr(h), level, scale))


def _pinned_view(host) -> np.ndarray:
    """The caller's own uint32 buffer (no temporary copy may be handed to an
    asynchronous transfer)."""
    if not (isinstance(host, np.ndarray) and host.dtype == np.uint32 and host.flags["C_CONTIGUOUS"]):
        raise TypeError("asynchronous transfers need a C-contiguous uint32 array (page-locked for overlap)")
    return host


def ckks_ct_upload_async(ctx, ct, host, level: int, scale: float):
    h = _pinned_view(host)
    check(ctx, lib.ckks_ct_upload_async(ctx, ct, _ptr(h), level, scale))


def ckks_ct_export_async(ctx, ct, host):
    h = _pinned_view(host)
    check(ctx, lib.ckks_ct_export_async(ctx, ct, _ptr(h), h.size))


def ckks_ct_info(ct):
    lv, sc, dp = C.c_int(), C.c_double(), _vp()
    check(None, lib.ckks_ct_info(ct, C.byref(lv), C.byref(sc), C.byref(dp)))
    return lv.value, sc.value, dp.value


def ckks_ct_export(ctx, ct, n: int, out: np.ndarray | None = None):
    lv, sc = C.c_int(), C.c_double()
    level, _, _ = ckks_ct_info(ct)
    if out is None:
        out = np.zeros((2, ckks_level_limbs(ctx, level), n), np.uint32)
    check(ctx, lib.ckks_ct_export(ctx, ct, _ptr(out), out.size, C.byref(lv), C.byref(sc)))
    return out, lv.value, sc.value


def ckks_ct_wrap_device(ctx, dev_ptr: int, level: int, scale: float):
    out = _vp()
    check(ctx, lib.ckks_ct_wrap_device(ctx, dev_ptr, level, scale, C.byref(out)))
    return out


def ckks_pt_import(ctx, host, level: int, scale: float):
    h = _u32(host)
    out = _vp()
    check(ctx, lib.ckks_pt_import(ctx, _ptr(h), level, scale, C.byref(out)))
    return out


def ckks_pt_import_ext(ctx, host, level: int, scale: float):
    h = _u32(host)
    out = _vp()
    check(ctx, lib.ckks_pt_import_ext(ctx, _ptr(h), level, scale, C.byref(out)))
    return out


def ckks_pt_export(ctx, pt, level: int, n: int):
    out = np.zeros((ckks_level_limbs(ctx, level), n), np.uint32)
    lv, sc = C.c_int(), C.c_double()
    check(ctx, lib.ckks_pt_export(ctx, pt, _ptr(out), out.size, C.byref(lv), C.byref(sc)))
    return out, lv.value, sc.value


def ckks_hadd(ctx, a, b, out):
    check(ctx, lib.ckks_hadd(ctx, a, b, out))


def ckks_pmult(ctx, a, pt, out):
    check(ctx, lib.ckks_pmult(ctx, a, pt, out))


def ckks_hmult(ctx, a, b, evk, flags: int, out):
    check(ctx, lib.ckks_hmult(ctx, a, b, evk, flags, out))


def ckks_rescale(ctx, a, out):
    check(ctx, lib.ckks_rescale(ctx, a, out))


def ckks_hrot(ctx, a, r: int, evk, out):
    check(ctx, lib.ckks_hrot(ctx, a, r, evk, out))


def ckks_padd(ctx, a, pt, out):
    check(ctx, lib.ckks_padd(ctx, a, pt, out))


def ckks_hconj(ctx, a, evk, out):
    check(ctx, lib.ckks_hconj(ctx, a, evk, out))


def ckks_linear_transform(ctx, a, rs, evks, pts, out):
    """out = sum_i pts[i] (.) HRot(a, rs[i]) with one shared ModUp and one ModDown."""
    cnt = len(rs)
    if len(evks) != cnt or len(pts) != cnt:
        raise ValueError("rs, evks and pts must have the same length")
    r_arr = (C.c_int * max(cnt, 1))(*[int(x) for x in rs])
    e_arr = (C.c_void_p * max(cnt, 1))(*[e if e is not None else None for e in evks])
    p_arr = (C.c_void_p * max(cnt, 1))(*pts)
    check(ctx, lib.ckks_linear_transform(ctx, a, cnt, r_arr, e_arr, p_arr, out))


def ckks_hrot_hoisted(ctx, a, rs, evks, outs):
    """outs[i] = HRot(a, rs[i]) with evks[i], sharing one ModUp."""
    cnt = len(rs)
    if len(evks) != cnt or len(outs) != cnt:
        raise ValueError("rs, evks and outs must have the same length")
    r_arr = (C.c_int * max(cnt, 1))(*[int(x) for x in rs])
    e_arr = (C.c_void_p * max(cnt, 1))(*evks)
    o_arr = (C.c_void_p * max(cnt, 1))(*outs)
    check(ctx, lib.ckks_hrot_hoisted(ctx, a, cnt, r_arr, e_arr, o_arr))


CKKS_BATCH_GRAPH, CKKS_BATCH_PERSISTENT = 1, 2


def ckks_batch_create(ctx, ops, lanes: int, use_graph):
    """ops: list of dicts with keys op, flags, r, a, b, pt, evk, out (handles);
    use_graph: a bool or the mode flags CKKS_BATCH_GRAPH | CKKS_BATCH_PERSISTENT."""
    arr = (ckks_op * len(ops))()
    for i, o in enumerate(ops):
        arr[i] = ckks_op(o["op"], o.get("flags", 0), o.get("r", 0), o.get("a"), o.get("b"), o.get("pt"),
                         o.get("evk"), o["out"])
    out = _vp()
    check(ctx, lib.ckks_batch_create(ctx, arr, len(ops), lanes, int(use_graph), C.byref(out)))
    return out


def ckks_batch_run(ctx, batch):
    check(ctx, lib.ckks_batch_run(batch))


def ckks_batch_run_admit(ctx, batch, admitted: int):
    """Persistent batch: run with only the first `admitted` operations admitted."""
    check(ctx, lib.ckks_batch_run_admit(batch, admitted))


def ckks_batch_admit(ctx, batch, admitted: int):
    """Persistent batch: raise the admitted count (takes effect in the running kernel)."""
    check(ctx, lib.ckks_batch_admit(batch, admitted))


def ckks_batch_destroy(batch):
    lib.ckks_batch_destroy(batch)


CKKS_NOALLOC_SCRATCH_WORDS = 1 << 21


def ckks_rescale_noalloc(ctx, in_dev: int, level: int, out_dev: int):
    """Rescale between caller-owned device buffers with the library's fixed
    scratch; see include/ckks.h for layout, limit and ordering rules."""
    check(ctx, lib.ckks_rescale_noalloc(ctx, in_dev, level, out_dev))


CKKS_COL_MODUP, CKKS_COL_MODDOWN, CKKS_COL_RS_FUSED, CKKS_ROW_PASSES = 0, 1, 2, 3
CKKS_LAUNCH_PDL = 1
CKKS_TUNE_TENSOR = 2
CKKS_LAUNCH_UNFUSED = 4
CKKS_LAUNCH_CHECKED = 8


def ckks_set_launch_flags(ctx, flags: int):
    check(ctx, lib.ckks_set_launch_flags(ctx, flags))


def ckks_set_memory_limit(ctx, nbytes: int):
    """Limit of the device bytes the context's objects may hold together (0 = none)."""
    check(ctx, lib.ckks_set_memory_limit(ctx, nbytes))


def ckks_memory_in_use(ctx) -> int:
    return int(lib.ckks_memory_in_use(ctx))


def ckks_request_bytes(ctx, op: int, level: int) -> int:
    """Device bytes a request of kind op (CKKS_OP_*) at level holds while it runs."""
    return int(lib.ckks_request_bytes(ctx, op, level))


def ckks_serve_run(lanes, pool, reqs, lane_outs=None, hooks=None, n_lanes=None):
    """Serve `reqs` (dicts op, r, arrival (seconds), a, b, evk, out (or None:
    the lane's output from lane_outs), bytes; sorted by arrival) on the lane
    contexts `lanes`. hooks = (issue(i, lane) -> status, query(lane) -> 1 / 0 /
    negative) replaces the device work (then lanes may be None and n_lanes
    gives their count). Returns ([(start_s, end_s, lane) per request],
    [request indices in completion order])."""
    n = len(reqs)
    nl = n_lanes if n_lanes is not None else len(lanes)
    arr = (ckks_request * max(n, 1))()
    for i, q in enumerate(reqs):
        arr[i] = ckks_request(q["op"], q.get("r", 0), q["arrival"], q.get("a"), q.get("b"), q.get("evk"),
                              q.get("out"), q["bytes"])
    lanes_arr = (_vp * nl)(*lanes) if lanes is not None else None
    outs_arr = (_vp * nl)(*lane_outs) if lane_outs is not None else None
    done = (ckks_request_done * max(n, 1))()
    order = (C.c_int * max(n, 1))()
    hk = None
    if hooks is not None:
        issue_py, query_py = hooks

        def _issue(_user, i, lane):
            try:
                return int(issue_py(i, lane))
            except Exception:  # a failing hook ends the run instead of unwinding through C
                return CKKS_EINVAL

        def _query(_user, lane):
            try:
                return int(query_py(lane))
            except Exception:
                return CKKS_EINVAL

        hk = ckks_serve_hooks(_ISSUE_FN(_issue), _QUERY_FN(_query), None)
    rc = lib.ckks_serve_run(lanes_arr, nl, pool, arr, n, outs_arr, C.byref(hk) if hk is not None else None, done,
                            order)
    check(lanes[0] if lanes is not None and hooks is None else None, rc)
    return [(done[i].start_s, done[i].end_s, done[i].lane) for i in range(n)], [order[i] for i in range(n)]


def ckks_pool_create(budget: int):
    out = _vp()
    check(None, lib.ckks_pool_create(budget, C.byref(out)))
    return out


def ckks_pool_acquire(pool, nbytes: int) -> bool:
    """True when admitted; False when the budget refuses it (CKKS_EBUSY)."""
    rc = lib.ckks_pool_acquire(pool, nbytes)
    if rc == CKKS_EBUSY:
        return False
    check(None, rc)
    return True


def ckks_pool_release(pool, nbytes: int):
    check(None, lib.ckks_pool_release(pool, nbytes))


def ckks_pool_in_use(pool) -> int:
    return int(lib.ckks_pool_in_use(pool))


def ckks_pool_destroy(pool):
    lib.ckks_pool_destroy(pool)


def ckks_set_wait_limit(ctx, cycles: int):
    """Clock-cycle limit of the kernels' bounded device-side waits (see
    include/ckks.h); an expired wait surfaces as CKKS_ETIMEOUT at the next
    synchronizing call."""
    check(ctx, lib.ckks_set_wait_limit(ctx, cycles))


def ckks_tune(ctx, level: int, reps: int = 5):
    check(ctx, lib.ckks_tune(ctx, level, reps))


def ckks_tune_get(ctx, kernel: int, level: int):
    """(tc, sl, z, tp, microseconds) of the tuned shape; tc = 0 when untuned."""
    tc, sl, z, tp, us = C.c_int(), C.c_int(), C.c_int(), C.c_int(), C.c_float()
    check(ctx, lib.ckks_tune_get(ctx, kernel, level, C.byref(tc), C.byref(sl), C.byref(z), C.byref(tp),
                                 C.byref(us)))
    return tc.value, sl.value, z.value, tp.value, us.value


def ckks_tune_set(ctx, kernel: int, level: int, tc: int, sl: int = 4, z: int = 1, tp: int = 1):
    check(ctx, lib.ckks_tune_set(ctx, kernel, level, tc, sl, z, tp))


CKKS_MODMUL_BARRETT, CKKS_MODMUL_MONTGOMERY, CKKS_MODMUL_SHOUP, CKKS_MODMUL_SMR = 0, 1, 2, 3


def ckks_bench_modmul(ctx, method: int, prime_id: int, b: int, a, rounds: int):
    """(a * b^rounds mod q per element, kernel milliseconds)."""
    a = _u32(a)
    out = np.zeros_like(a)
    ms = C.c_float()
    check(ctx, lib.ckks_bench_modmul(ctx, method, prime_id, int(b), _ptr(a), a.size, rounds, _ptr(out),
                                     C.byref(ms)))
    return out, ms.value


CKKS_INTOP_MAD_LO, CKKS_INTOP_MAD_HI, CKKS_INTOP_MAD_WIDE = 0, 1, 2


def ckks_bench_intop(ctx, op: int, rounds: int = 4096):
    """(instructions executed, kernel milliseconds) of the integer-multiply
    issue-rate probe for one instruction form."""
    ops, ms = C.c_double(), C.c_float()
    check(ctx, lib.ckks_bench_intop(ctx, op, rounds, C.byref(ops), C.byref(ms)))
    return ops.value, ms.value


CKKS_PROF_KERNELS = 13


def ckks_profile(ctx, enable: bool):
    check(ctx, lib.ckks_profile(ctx, int(enable)))


def ckks_profile_read(ctx) -> dict:
    ms = np.zeros(CKKS_PROF_KERNELS, np.float64)
    cnt = np.zeros(CKKS_PROF_KERNELS, np.uint64)
    check(ctx, lib.ckks_profile_read(ctx, _ptr(ms), _ptr(cnt)))
    return {lib.ckks_profile_name(i).decode(): (float(ms[i]), int(cnt[i])) for i in range(CKKS_PROF_KERNELS)}


def ckks_launch_count() -> int:
    return int(lib.ckks_launch_count())


def ckks_step_smr(ctx, x, prime_id: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.int64)
    y = np.zeros(x.size, np.int32)
    check(ctx, lib.ckks_step_smr(ctx, _ptr(x), x.size, prime_id, _ptr(y)))
    return y


def ckks_step_ntt(ctx, data, prime_ids, inverse: bool) -> np.ndarray:
    d = _u32(data).copy()
    ids = np.ascontiguousarray(prime_ids, dtype=np.int32)
    check(ctx, lib.ckks_step_ntt(ctx, _ptr(d), len(ids), _ptr(ids), int(inverse)))
    return d


def ckks_step_bconv(ctx, x, src_ids, dst_ids, variant: int = 0) -> np.ndarray:
    x = _u32(x)
    s = np.ascontiguousarray(src_ids, dtype=np.int32)
    d = np.ascontiguousarray(dst_ids, dtype=np.int32)
    out = np.zeros((len(d), x.shape[-1]), np.uint32)
    check(ctx, lib.ckks_step_bconv(ctx, _ptr(x), len(s), _ptr(s), _ptr(out), len(d), _ptr(d), variant))
    return out


def ckks_step_tensor(ctx, ct1, ct2) -> np.ndarray:
    c1, c2 = _u32(ct1), _u32(ct2)
    out = np.zeros((3,) + c1.shape[1:], np.uint32)
    check(ctx, lib.ckks_step_tensor(ctx, _ptr(c1), _ptr(c2), c1.shape[1], _ptr(out)))
    return out


def ckks_step_automorph(ctx, x, galois: int) -> np.ndarray:
    x = _u32(x)
    out = np.zeros_like(x)
    limbs = x.size // x.shape[-1]
    check(ctx, lib.ckks_step_automorph(ctx, _ptr(x), limbs, galois, _ptr(out)))
    return out


def ckks_step_modup(ctx, d, alpha: int) -> np.ndarray:
    d = _u32(d)
    n_q, n = d.shape
    digits = -(-n_q // alpha)
    out = np.zeros((digits, n_q + alpha, n), np.uint32)
    check(ctx, lib.ckks_step_modup(ctx, _ptr(d), n_q, _ptr(out)))
    return out


def ckks_step_keyswitch_acc(ctx, d, evk, alpha: int) -> np.ndarray:
    d = _u32(d)
    n_q, n = d.shape
    out = np.zeros((2, n_q + alpha, n), np.uint32)
    check(ctx, lib.ckks_step_keyswitch_acc(ctx, _ptr(d), n_q, evk, _ptr(out)))
    return out


def ckks_step_moddown(ctx, acc, n_q: int) -> np.ndarray:
    a = _u32(acc)
    out = np.zeros((2, n_q, a.shape[-1]), np.uint32)
    check(ctx, lib.ckks_step_moddown(ctx, _ptr(a), n_q, _ptr(out)))
    return out
