"""Host logic of the bootstrap-shaped trace (trace.py) on the CPU: the trace's
composition of linear transforms, the polynomial's factors and its product
tree, in the fused (batched) and the one-operation-at-a-time form, run
against a fake library that carries plaintext slot vectors, equals the
trace's plain definition (trace.expected), and the levels and scales follow
the rescaling bookkeeping."""
import numpy as np
import pytest

from paper_2407_13055_gb300 import trace


class H:
    """Fake handle: slot values, level, scale."""

    def __init__(self, level=0, vals=None, scale=1.0):
        self.level, self.vals, self.scale = level, vals, scale


class FakeK:
    CKKS_RESCALE = 1
    CKKS_OP_HMULT, CKKS_OP_PMULT, CKKS_OP_RESCALE, CKKS_OP_PADD = 1, 4, 5, 7

    def __init__(self, q):
        self.q = q
        self.batches = 0

    # objects
    def ckks_ct_create(self, ctx, level):
        return H(level)

    def ckks_free(self, h):
        pass

    def ckks_ct_info(self, ct):
        return ct.level, ct.scale, 0

    def ckks_keygen_rot(self, ctx, sk, r, seed):
        return ("rot", r)

    def ckks_keygen_relin(self, ctx, sk, seed):
        return ("relin",)

    def ckks_encode(self, ctx, values, level, scale):
        return H(level, np.asarray(values, np.complex128), scale)

    ckks_encode_ext = ckks_encode

    # operations (slot semantics; rotation = np.roll by -r)
    def _set(self, out, vals, level, scale):
        out.vals, out.level, out.scale = vals, level, scale

    def ckks_hadd(self, ctx, a, b, out):
        assert a.level == b.level and a.scale == pytest.approx(b.scale, rel=1e-9)
        self._set(out, a.vals + b.vals, a.level, a.scale)

    def ckks_padd(self, ctx, a, pt, out):
        assert pt.level >= a.level and pt.scale == pytest.approx(a.scale, rel=1e-9)
        self._set(out, a.vals + pt.vals, a.level, a.scale)

    def ckks_pmult(self, ctx, a, pt, out):
        self._set(out, a.vals * pt.vals, a.level, a.scale * pt.scale)

    def ckks_hrot(self, ctx, a, r, key, out):
        assert key == ("rot", r)
        self._set(out, np.roll(a.vals, -r), a.level, a.scale)

    def ckks_rescale(self, ctx, a, out):
        assert a.level >= 1
        self._set(out, a.vals, a.level - 1, a.scale / self.q[a.level])

    def ckks_hmult(self, ctx, a, b, evk, flags, out):
        assert a.level == b.level and evk == ("relin",) and flags == self.CKKS_RESCALE
        self._set(out, a.vals * b.vals, a.level - 1, a.scale * b.scale / self.q[a.level])

    def ckks_linear_transform(self, ctx, x, rs, keys, pts, out):
        acc = np.zeros_like(x.vals)
        for r, k, pt in zip(rs, keys, pts):
            assert (k is None) == (r == 0)
            acc = acc + pt.vals * np.roll(x.vals, -r)
        self._set(out, acc, x.level, x.scale * pts[0].scale)

    # batches: independent operations, run at creation and on every run
    def _run(self, ops):
        outs = [o["out"] for o in ops]
        ins = [o.get(k) for o in ops for k in ("a", "b")]
        assert len(set(map(id, outs))) == len(outs) and not set(map(id, outs)) & set(map(id, ins))
        for o in ops:
            if o["op"] == self.CKKS_OP_HMULT:
                self.ckks_hmult(None, o["a"], o["b"], o["evk"], o["flags"], o["out"])
            elif o["op"] == self.CKKS_OP_PMULT:
                self.ckks_pmult(None, o["a"], o["pt"], o["out"])
            elif o["op"] == self.CKKS_OP_RESCALE:
                self.ckks_rescale(None, o["a"], o["out"])
            else:
                self.ckks_padd(None, o["a"], o["pt"], o["out"])

    def ckks_batch_create(self, ctx, ops, lanes, use_graph):
        self.batches += 1
        self._run(ops)
        return list(ops)

    def ckks_batch_run(self, ctx, batch):
        self._run(batch)

    def ckks_batch_destroy(self, batch):
        pass


@pytest.mark.parametrize("fused", [True, False])
def test_trace_composition_matches_its_definition(fused):
    spec = trace.TraceSpec(n1=4, n2=2, lt_levels=1, depth=3, seed=7)
    slots, level0 = 32, 10
    rng = np.random.default_rng(3)
    q = [float(2**30 + 1000 * i) for i in range(level0 + 1)]
    K = FakeK(q)
    u = rng.uniform(-1, 1, slots) + 1j * rng.uniform(-1, 1, slots)
    tr = trace.Trace(K, "ctx", spec, level0, q, slots, sk="sk")
    x = H(level0, u.copy(), 2.0**40)
    want = trace.expected(spec, u)
    # scale bookkeeping: linear transforms and the factors return their input
    # scale exactly; each product-tree level squares it and divides by its prime
    s, lv = 2.0**40, level0 - spec.lt_levels - 1
    for _ in range(spec.depth):
        s, lv = s * s / q[lv], lv - 1
    for _ in range(2):  # the second run reuses the pooled ciphertexts and cached batches
        out, level = tr.run(x, fused=fused)
        assert level == level0 - spec.levels_used()
        assert out.level == level
        assert np.allclose(out.vals, want, atol=1e-9)
        assert out.scale == pytest.approx(s, rel=1e-9)
    if fused:
        assert K.batches == 3 + spec.depth  # factors (PMult, rescale, PAdd) and one per tree level
    tr.close()
