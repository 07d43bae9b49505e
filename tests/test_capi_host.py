"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function declared in include/ckks.h, its prime rule
agrees with the oracle's, and it fails cleanly where a GPU is required."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def K():
    from paper_2407_13055_gb300 import build
    build.build()
    from paper_2407_13055_gb300 import ckks
    return ckks


def _declared():
    src = open(os.path.join(ROOT, "include", "ckks.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ckks_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported(K):
    names = _declared()
    assert len(names) >= 30
    for name in names:
        assert hasattr(K.lib, name), name
    assert set(names) == set(K.EXPORTED)


@pytest.mark.parametrize("log_n,n_q,n_p", [(8, 6, 2), (12, 4, 4), (16, 40, 14), (16, 40, 40)])
def test_prime_rule_matches_oracle(K, O, log_n, n_q, n_p):
    q, p = K.ckks_gen_primes(log_n, n_q, n_p)
    oq, op = O.gen_primes(log_n, n_q, n_p)
    assert np.array_equal(q, oq) and np.array_equal(p, op)


def test_ctx_create_rejects_bad_parameters(K, O):
    q, p = O.gen_primes(12, 4, 1)
    with pytest.raises(K.CkksError) as e:
        K.ckks_ctx_create(13, q, p, 4)
    assert e.value.code == K.CKKS_EINVAL
    with pytest.raises(K.CkksError) as e:
        K.ckks_ctx_create(12, q, p, 2)          # dnum must be ceil(n_q / n_p)
    assert e.value.code == K.CKKS_EINVAL
    bad = q.copy()
    bad[1] += 2                                  # not 1 mod 2N
    with pytest.raises(K.CkksError) as e:
        K.ckks_ctx_create(12, bad, p, 4)
    assert e.value.code == K.CKKS_EINVAL


def test_ctx_create_without_gpu_fails_cleanly(K, O):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    q, p = O.gen_primes(12, 4, 1)
    with pytest.raises(K.CkksError) as e:
        K.ckks_ctx_create(12, q, p, 4)
    assert e.value.code == K.CKKS_ECUDA


@pytest.mark.parametrize("log_n", [8, 12, 16])
def test_prime_system_2530_matches_oracle(K, O, log_n):
    """The library's 25-30 prime system (its own code) equals the oracle's."""
    q, p, levels = K.ckks_gen_prime_system_2530(log_n, 5)
    P, lv = O.prime_system_2530(log_n, 5)
    assert q.tolist() == [int(v) for v in P.q]
    assert p.tolist() == [int(v) for v in P.p]
    assert levels == [tuple(x) for x in lv]


def test_status_codes_and_flags_match_the_header(K):
    """The binding's error codes and launch flags are the header's."""
    src = open(os.path.join(ROOT, "include", "ckks.h")).read()
    defs = dict(re.findall(r"#define (CKKS_[A-Z0-9_]+) \(?(-?\d+)\)?", src))
    for name in ("CKKS_EINVAL", "CKKS_ETIMEOUT", "CKKS_EBUSY", "CKKS_ERANGE", "CKKS_LAUNCH_PDL", "CKKS_TUNE_TENSOR",
                 "CKKS_LAUNCH_UNFUSED", "CKKS_LAUNCH_CHECKED"):
        assert int(defs[name]) == getattr(K, name), name
    assert len({int(v) for k, v in defs.items() if k.startswith("CKKS_E")}) == \
        len([k for k in defs if k.startswith("CKKS_E")])
    assert K.lib.ckks_set_launch_flags(None, K.CKKS_LAUNCH_CHECKED) == K.CKKS_EINVAL


def test_null_handles_are_rejected_without_a_gpu(K):
    """Every operation validates its handles before touching the device:
    null context, operands or outputs give CKKS_EINVAL."""
    L = K.lib
    E = K.CKKS_EINVAL
    assert L.ckks_hmult(None, None, None, None, 0, None) == E
    assert L.ckks_hrot(None, None, 1, None, None) == E
    assert L.ckks_hconj(None, None, None, None) == E
    assert L.ckks_rescale(None, None, None) == E
    assert L.ckks_hadd(None, None, None, None) == E
    assert L.ckks_pmult(None, None, None, None) == E
    assert L.ckks_padd(None, None, None, None) == E
    assert L.ckks_tune(None, 0, 1) == E
    assert L.ckks_sync(None) == E
    assert L.ckks_batch_run(None) == E
    assert L.ckks_batch_run_admit(None, 0) == E
    assert L.ckks_batch_admit(None, 0) == E
    assert L.ckks_set_wait_limit(None, 1) == E
    assert L.ckks_rescale_noalloc(None, None, 1, None) == E
    assert L.ckks_level_limbs(None, 0) == E
    assert L.ckks_serve_run(None, 1, None, None, 0, None, None, None, None) == E   # no pool
    pool = K.ckks_pool_create(100)
    try:
        assert L.ckks_serve_run(None, 1, pool, None, 0, None, None, None, None) == E   # no lanes, no hooks
        assert L.ckks_serve_run(None, 0, pool, None, 0, None, None, None, None) == E   # no lane
        assert L.ckks_serve_run(None, 1, pool, None, 1, None, None, None, None) == E   # no requests
    finally:
        K.ckks_pool_destroy(pool)


def test_admission_pool_refuses_beyond_its_budget(K):
    """The library's admission pool (host-side): acquisitions within the
    budget succeed, one that would exceed it returns CKKS_EBUSY and takes
    nothing, releases return the bytes, over-release is refused."""
    import ctypes as C
    L = K.lib
    h = C.c_void_p()
    assert L.ckks_pool_create(1000, C.byref(h)) == K.CKKS_OK
    try:
        assert L.ckks_pool_acquire(h, 600) == K.CKKS_OK
        assert L.ckks_pool_acquire(h, 401) == K.CKKS_EBUSY
        assert L.ckks_pool_in_use(h) == 600
        assert L.ckks_pool_acquire(h, 400) == K.CKKS_OK
        assert L.ckks_pool_acquire(h, 1) == K.CKKS_EBUSY
        assert L.ckks_pool_release(h, 1001) == K.CKKS_EINVAL
        assert L.ckks_pool_release(h, 1000) == K.CKKS_OK
        assert L.ckks_pool_in_use(h) == 0
        assert L.ckks_pool_acquire(h, 1001) == K.CKKS_EBUSY
        assert L.ckks_pool_acquire(None, 1) == K.CKKS_EINVAL
        assert L.ckks_set_memory_limit(None, 1) == K.CKKS_EINVAL
        assert L.ckks_memory_in_use(None) == 0
        assert L.ckks_request_bytes(None, 1, 0) == 0
    finally:
        L.ckks_pool_destroy(h)
