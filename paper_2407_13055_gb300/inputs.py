"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only draws random numbers. It holds none of the scheme's
arithmetic: no modular reduction beyond drawing a residue below a prime, no
NTT, no encoding. Everything the CKKS scheme samples (Eq. 1 of the paper:
the uniform mask ``a``, the error ``e``, the ternary secret ``s``) is drawn
here and handed to both implementations as plain arrays, so that the two sides
can be compared bit for bit.

Distributions (the paper is silent on them; these are the usual choices):

* messages: complex slots with real and imaginary parts uniform in [-1, 1];
* secret: ternary coefficients in {-1, 0, 1}; either a fixed Hamming weight
  ``h`` (positions uniform without replacement, signs +-1 with probability
  1/2 each) or, with ``h=None``, each coefficient uniform over {-1, 0, 1};
* error: rounded Gaussian with standard deviation ``sigma`` (3.2), tail-cut
  at ``bound`` (20, about 6 sigma) by resampling;
* uniform mask: independent residues uniform in [0, q_i) for every prime.
"""
from __future__ import annotations

import numpy as np

SIGMA = 3.2
ERROR_BOUND = 20


def _rng(seed: int, *stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed), *map(int, stream)]))


def messages(seed: int, n_slots: int) -> np.ndarray:
    """Complex message vector u with Re, Im ~ U[-1, 1] (length n_slots = N/2)."""
    g = _rng(seed, 1)
    re = g.uniform(-1.0, 1.0, n_slots)
    im = g.uniform(-1.0, 1.0, n_slots)
    return re + 1j * im


def ternary_secret(seed: int, n: int, h: int | None) -> np.ndarray:
    """Ternary secret coefficients (int64, length n)."""
    g = _rng(seed, 2)
    s = np.zeros(n, dtype=np.int64)
    if h is None:
        s[:] = g.integers(-1, 2, n)
    else:
        pos = g.choice(n, size=h, replace=False)
        s[pos] = np.where(g.integers(0, 2, h) == 0, -1, 1)
    return s


def gaussian_error(seed: int, n: int, stream: int = 0,
                   sigma: float = SIGMA, bound: int = ERROR_BOUND) -> np.ndarray:
    """Rounded Gaussian error coefficients (int64, length n), |e| <= bound."""
    g = _rng(seed, 3, stream)
    e = np.rint(g.normal(0.0, sigma, n)).astype(np.int64)
    bad = np.abs(e) > bound
    while bad.any():
        e[bad] = np.rint(g.normal(0.0, sigma, int(bad.sum()))).astype(np.int64)
        bad = np.abs(e) > bound
    return e


def uniform_residues(seed: int, primes, n: int, stream: int = 0) -> np.ndarray:
    """Uniform residues: array [len(primes)][n] of uint32, row i uniform in [0, primes[i])."""
    g = _rng(seed, 4, stream)
    out = np.empty((len(primes), n), dtype=np.uint32)
    for i, q in enumerate(primes):
        out[i] = g.integers(0, int(q), n, dtype=np.uint64).astype(np.uint32)
    return out


def level_list(seed: int, count: int, top: int, low: int = 1) -> np.ndarray:
    """Levels drawn uniformly from [low, top] (batched / served workloads)."""
    return _rng(seed, 5).integers(low, top + 1, count)


def rotation_list(seed: int, count: int, n_slots: int) -> np.ndarray:
    """Rotation distances drawn uniformly from [1, n_slots)."""
    return _rng(seed, 6).integers(1, n_slots, count)
