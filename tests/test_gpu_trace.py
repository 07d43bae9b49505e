"""Bootstrap-shaped trace (linear transforms, degree-2^d polynomial by a
product tree, linear transforms) through the library: the decryption equals
the plaintext computation within 1e-3, fused and one-op-at-a-time alike."""
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


@pytest.mark.parametrize("spec_args", [dict(n1=4, n2=2, lt_levels=1, depth=3), dict()])
def test_trace_decrypts_to_plaintext_result(K, O, spec_args):
    from paper_2407_13055_gb300.trace import Trace, TraceSpec, expected
    spec = TraceSpec(**spec_args)
    log_n, L, dnum = 12, spec.levels_used() + 2, 2
    P = O.make_params(log_n, L, dnum)
    ctx = K.ckks_ctx_create(log_n, P.q, P.p, dnum, scale=2.0**30)
    handles = []
    try:
        sk = K.ckks_keygen_secret(ctx, 3)
        handles.append(sk)
        u = inputs.messages(4, P.n // 2)
        level0 = L - 1
        pt = K.ckks_encode(ctx, u, level0, 2.0**30)
        ct = K.ckks_encrypt(ctx, sk, pt, 5)
        handles += [pt, ct]
        tr = Trace(K, ctx, spec, level0, P.q, P.n // 2, sk=sk)
        try:
            want = expected(spec, u)
            got = {}
            for fused in (True, False):
                out, level = tr.run(ct, fused=fused)
                assert level == level0 - spec.levels_used()
                dec = K.ckks_decrypt(ctx, sk, out)
                got[fused] = K.ckks_decode(ctx, dec, P.n // 2)
                K.ckks_free(dec)
                assert np.max(np.abs(got[fused] - want)) < 1e-3, fused
            assert np.max(np.abs(got[True] - got[False])) < 1e-3
        finally:
            tr.close()
    finally:
        for h in handles:
            K.ckks_free(h)
        K.ckks_ctx_destroy(ctx)
