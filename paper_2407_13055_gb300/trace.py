"""Bootstrap-shaped operation trace composed from the library's operations.

The shape follows the paper's bootstrapping workload (Sec. 5.2, Par. 4-5):

* CoeffToSlot-like: `lt_levels` baby-step giant-step linear transforms, each
  y = sum_g HRot( sum_b E[g][b] (.) HRot(x, b), g n1 ) over n1 baby and n2
  giant steps (n1 n2 random plaintext diagonals), followed by a rescale;
* a degree-2^depth polynomial, prod_i (c_i x + b_i), as 2^depth PMult-by-
  constant + rescale + PAdd factors and a product tree of HMult + rescale
  (depth `depth`); siblings in the tree share their provenance, so their
  levels and scales agree exactly;
* SlotToCoeff-like: `lt_levels` more linear transforms.

`fused=True` uses the library's fused and batched forms: ckks_linear_transform
(one shared ModUp, all KeyMult + MAC in one kernel, one ModDown) and, for
the polynomial's independent operations (the factors, then each level of the
product tree), operation batches captured once into CUDA graphs over
execution lanes. `fused=False` issues the same computation one operation at a
time (separate HRot, PMult, HAdd, HMult). Plaintext scales are chosen so that every rescale returns the scale of
the input exactly: diagonals and constants are encoded at the prime that the
following rescale divides by.
"""
from __future__ import annotations

import collections
from dataclasses import dataclass, field

import numpy as np


@dataclass
class TraceSpec:
    # 32 baby x 2 giant steps: 64 diagonals per transform over 32 rotation
    # indices (1 .. 31 hoisted, 32 for the giant step)
    n1: int = 32         # baby steps
    n2: int = 2          # giant steps
    lt_levels: int = 2   # linear-transform levels on each side
    depth: int = 6       # product-tree depth: polynomial degree 2^depth
    seed: int = 1234

    def levels_used(self) -> int:
        return 2 * self.lt_levels + 1 + self.depth

    def rotations(self):
        return sorted(set(range(1, self.n1)) | {g * self.n1 for g in range(1, self.n2)})


@dataclass
class _Data:
    diags: list = field(default_factory=list)     # per LT level: [n2][n1] slot vectors
    consts: np.ndarray = None                       # c_i
    offsets: np.ndarray = None                      # b_i


def _make_data(spec: TraceSpec, slots: int) -> _Data:
    rng = np.random.default_rng(spec.seed)
    d = _Data()
    for _ in range(2 * spec.lt_levels):
        # diagonals scaled so that a transform keeps values of order one
        s = 1.0 / (spec.n1 * spec.n2) ** 0.5
        d.diags.append([[s * (rng.uniform(-1, 1, slots) + 1j * rng.uniform(-1, 1, slots)) for _ in range(spec.n1)]
                        for _ in range(spec.n2)])
    k = 1 << spec.depth
    d.consts = 0.05 * rng.uniform(-1, 1, k)
    d.offsets = 1.0 + 0.05 * rng.uniform(-1, 1, k)
    return d


def expected(spec: TraceSpec, u: np.ndarray) -> np.ndarray:
    """The trace on plaintext slots (left rotation = np.roll by -r)."""
    d = _make_data(spec, u.size)
    x = u.astype(np.complex128)

    def lt(x, diags):
        y = np.zeros_like(x)
        for g in range(spec.n2):
            inner = sum(diags[g][b] * np.roll(x, -b) for b in range(spec.n1))
            y = y + np.roll(inner, -g * spec.n1)
        return y

    for lvl in range(spec.lt_levels):
        x = lt(x, d.diags[lvl])
    p = np.ones_like(x)
    for c, b in zip(d.consts, d.offsets):
        p = p * (c * x + b)
    x = p
    for lvl in range(spec.lt_levels, 2 * spec.lt_levels):
        x = lt(x, d.diags[lvl])
    return x


class Trace:
    """Runs the trace on one ciphertext with the library binding `K`. The
    ciphertexts it creates are pooled by level and reused by later runs, so a
    warmed-up run allocates no device memory."""

    def __init__(self, K, ctx, spec: TraceSpec, level0: int, primes_q, slots: int, sk=None, keys=None,
                 relin=None, key_seed: int = 900):
        self.K, self.ctx, self.spec = K, ctx, spec
        self.level0 = level0
        self.q = [int(v) for v in primes_q]
        self.slots = slots
        self.data = _make_data(spec, slots)
        self._own = []
        if keys is None:
            keys = {r: K.ckks_keygen_rot(ctx, sk, r, key_seed + r) for r in spec.rotations()}
            self._own += list(keys.values())
        if relin is None:
            relin = K.ckks_keygen_relin(ctx, sk, key_seed - 1)
            self._own.append(relin)
        self.keys, self.relin = keys, relin
        self._pts = {}
        self._free = {}
        self._used = []
        self._batches = {}
        self.lanes = 4

    def close(self):
        self._reset()
        for b, _ in self._batches.values():
            self.K.ckks_batch_destroy(b)
        for lst in self._free.values():
            for h in lst:
                self.K.ckks_free(h)
        for h in self._own + list(self._pts.values()):
            self.K.ckks_free(h)
        self._own, self._pts, self._free, self._batches = [], {}, {}, {}

    def _reset(self):
        # first in, first out: every run after the first gets the same
        # ciphertext at the same position, so cached batches stay valid
        for level, ct in self._used:
            self._free.setdefault(level, collections.deque()).append(ct)
        self._used = []

    def _new(self, level):
        lst = self._free.get(level)
        ct = lst.popleft() if lst else self.K.ckks_ct_create(self.ctx, level)
        self._used.append((level, ct))
        return ct

    def _run_batch(self, key, ops):
        """Run independent operations as one cached graph batch."""
        sig = tuple(tuple(sorted((k, v if not hasattr(v, "value") else v.value) for k, v in o.items())) for o in ops)
        hit = self._batches.get(key)
        if hit is None or hit[1] != sig:
            if hit is not None:
                self.K.ckks_batch_destroy(hit[0])
            hit = (self.K.ckks_batch_create(self.ctx, ops, self.lanes, True), sig)
            self._batches[key] = hit
        else:
            self.K.ckks_batch_run(self.ctx, hit[0])

    # -- plaintexts (cached) ------------------------------------------------------
    def _pt(self, key, values, level, scale, ext):
        if key not in self._pts:
            enc = self.K.ckks_encode_ext if ext else self.K.ckks_encode
            self._pts[key] = enc(self.ctx, values, level, scale)
        return self._pts[key]

    def _const(self, value, level, scale, tag):
        return self._pt((tag, value, level, scale), np.full(self.slots, value, np.complex128), level, scale, False)

    # -- pieces -------------------------------------------------------------------
    def _rescaled(self, ct, level):
        out = self._new(level - 1)
        self.K.ckks_rescale(self.ctx, ct, out)
        return out

    def _lt(self, x, level, lvl_idx, fused):
        K, ctx, sp = self.K, self.ctx, self.spec
        diags = self.data.diags[lvl_idx]
        dscale = float(self.q[level])         # the rescale after the transform divides by q_level
        pts = [[self._pt(("diag", lvl_idx, g, b, level), diags[g][b], level, dscale, True) for b in range(sp.n1)]
               for g in range(sp.n2)]
        acc = None
        for g in range(sp.n2):
            inner = self._new(level)
            if fused:
                rs = list(range(sp.n1))
                K.ckks_linear_transform(ctx, x, rs, [self.keys.get(r) for r in rs], pts[g], inner)
            else:
                K.ckks_pmult(ctx, x, pts[g][0], inner)
                rot, prod = self._new(level), self._new(level)
                for b in range(1, sp.n1):
                    K.ckks_hrot(ctx, x, b, self.keys[b], rot)
                    K.ckks_pmult(ctx, rot, pts[g][b], prod)
                    K.ckks_hadd(ctx, inner, prod, inner)
            if g == 0:
                acc = inner
            else:
                rot = self._new(level)
                K.ckks_hrot(ctx, inner, g * sp.n1, self.keys[g * sp.n1], rot)
                K.ckks_hadd(ctx, acc, rot, acc)
        return self._rescaled(acc, level)

    def _poly(self, x, level, fused):
        K, ctx = self.K, self.ctx
        _, s, _ = K.ckks_ct_info(x)
        cscale = float(self.q[level])         # the rescale after PMult divides by q_level
        cs = [self._const(float(c), level, cscale, "c") for c in self.data.consts]
        bs = [self._const(float(b), level - 1, s, "b") for b in self.data.offsets]
        t = [self._new(level) for _ in cs]
        f = [self._new(level - 1) for _ in cs]
        g = [self._new(level - 1) for _ in cs]
        if fused:
            self._run_batch(("pmult", level), [dict(op=K.CKKS_OP_PMULT, a=x, pt=c, out=o) for c, o in zip(cs, t)])
            self._run_batch(("rescale", level), [dict(op=K.CKKS_OP_RESCALE, a=i, out=o) for i, o in zip(t, f)])
            self._run_batch(("padd", level), [dict(op=K.CKKS_OP_PADD, a=i, pt=b, out=o) for i, b, o in zip(f, bs, g)])
        else:
            for c, b, ti, fi, gi in zip(cs, bs, t, f, g):
                K.ckks_pmult(ctx, x, c, ti)
                K.ckks_rescale(ctx, ti, fi)
                K.ckks_padd(ctx, fi, b, gi)
        factors, lv = g, level - 1
        while len(factors) > 1:
            pairs = list(zip(factors[0::2], factors[1::2]))
            outs = [self._new(lv - 1) for _ in pairs]
            if fused:
                self._run_batch(("tree", lv), [dict(op=K.CKKS_OP_HMULT, a=a, b=b, evk=self.relin,
                                                    flags=K.CKKS_RESCALE, out=o) for (a, b), o in zip(pairs, outs)])
            else:
                for (a, b), o in zip(pairs, outs):
                    K.ckks_hmult(ctx, a, b, self.relin, K.CKKS_RESCALE, o)
            factors, lv = outs, lv - 1
        return factors[0], lv

    def run(self, ct, fused: bool = True):
        """Returns the output ciphertext (valid until the next run or close)
        and its level."""
        self._reset()
        x, level = ct, self.level0
        for lvl in range(self.spec.lt_levels):
            x = self._lt(x, level, lvl, fused)
            level -= 1
        x, level = self._poly(x, level, fused)
        for lvl in range(self.spec.lt_levels, 2 * self.spec.lt_levels):
            x = self._lt(x, level, lvl, fused)
            level -= 1
        return x, level
