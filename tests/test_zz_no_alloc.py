"""ckks_rescale_noalloc: the rescale entry point for callers that must not
allocate device memory while they run (it keeps its scratch in a fixed
device array owned by the library). Its results must equal those of
ckks_rescale, the allocating-context entry point, bit for bit, on two calls
in a row (the second call sees whatever the first left in the shared
scratch). This file sorts last so that a stop-at-first-failure run has
already run every other test."""
import numpy as np
import pytest

from paper_2407_13055_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2407_13055_gb300 import ckks
    return ckks


def _rand_ct(q, n_q, n, seed):
    return np.stack([inputs.uniform_residues(seed, q[:n_q], n, t) for t in range(2)])


def _reference(K, ctx, host, level, n):
    ct = K.ckks_ct_import(ctx, host, level, 2.0**60)
    out = K.ckks_ct_create(ctx, level - 1)
    try:
        K.ckks_rescale(ctx, ct, out)
        return K.ckks_ct_export(ctx, out, n)[0]
    finally:
        K.ckks_free(ct)
        K.ckks_free(out)


def _noalloc(K, ctx, host, level, n):
    import torch
    ct = K.ckks_ct_import(ctx, host, level, 2.0**60)
    dst = torch.empty((2, level, n), dtype=torch.int32, device="cuda")
    _, _, src_ptr = K.ckks_ct_info(ct)
    try:
        K.ckks_rescale_noalloc(ctx, src_ptr, level, dst.data_ptr())
        view = K.ckks_ct_wrap_device(ctx, dst.data_ptr(), level - 1, 2.0**60)
        try:
            return K.ckks_ct_export(ctx, view, n)[0]
        finally:
            K.ckks_free(view)
    finally:
        K.ckks_free(ct)


@pytest.mark.parametrize("log_n,L,dnum,alpha,level", [(12, 4, 4, 1, 3), (16, 40, 3, 14, 15)])
def test_noalloc_rescale_matches_rescale_twice(K, O, log_n, L, dnum, alpha, level):
    import torch
    P = O.make_params(log_n, L, dnum, alpha)
    ctx = K.ckks_ctx_create(log_n, P.q, P.p, dnum, stream=torch.cuda.current_stream().cuda_stream)
    try:
        for call, seed in enumerate((11, 12)):
            host = _rand_ct(P.q, level + 1, P.n, seed)
            want = _reference(K, ctx, host, level, P.n)
            got = _noalloc(K, ctx, host, level, P.n)
            assert np.array_equal(got, want), f"call {call}"
        # the result is also the oracle's
        assert np.array_equal(got, O.rescale(host, P.q[:level + 1]))
    finally:
        K.ckks_ctx_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_the_fixed_scratch(K, O):
    P = O.make_params(16, 40, 3, 14)
    ctx = K.ckks_ctx_create(16, P.q, P.p, 3)
    try:
        with pytest.raises(K.CkksError) as e:
            K.ckks_rescale_noalloc(ctx, 1 << 20, 16, 1 << 21)   # (2 + 32) * 2^16 > 2^21 words
        assert e.value.code == K.CKKS_EINVAL
        assert "exceed" in K.lib.ckks_last_error(ctx).decode()
    finally:
        K.ckks_ctx_destroy(ctx)
