"""The seeded input generators shared by the oracle and the CUDA path: same
seed and stream give the same draws, different streams differ, and each draw
has the stated distribution's support and moments."""
import numpy as np
import pytest

from paper_2407_13055_gb300 import inputs


def test_messages_deterministic_and_in_range():
    a, b = inputs.messages(3, 4096), inputs.messages(3, 4096)
    assert np.array_equal(a, b) and not np.array_equal(a, inputs.messages(4, 4096))
    assert np.all(np.abs(a.real) <= 1) and np.all(np.abs(a.imag) <= 1)
    assert abs(a.real.mean()) < 0.05 and a.real.var() == pytest.approx(1 / 3, rel=0.1)


@pytest.mark.parametrize("h", [192, None])
def test_ternary_secret(h):
    s = inputs.ternary_secret(5, 1 << 12, h)
    assert np.array_equal(s, inputs.ternary_secret(5, 1 << 12, h))
    assert set(np.unique(s)) <= {-1, 0, 1}
    if h is not None:
        assert int(np.count_nonzero(s)) == h
    else:
        counts = [np.count_nonzero(s == v) for v in (-1, 0, 1)]
        assert min(counts) > 0.28 * s.size


def test_gaussian_error_bound_and_spread():
    e = np.concatenate([inputs.gaussian_error(7, 1 << 14, st) for st in range(4)])
    assert np.all(np.abs(e) <= inputs.ERROR_BOUND)
    assert e.std() == pytest.approx(inputs.SIGMA, rel=0.05)
    assert not np.array_equal(inputs.gaussian_error(7, 256, 0), inputs.gaussian_error(7, 256, 1))


def test_uniform_residues_below_each_prime():
    primes = [97, 12289, 1073479681]
    r = inputs.uniform_residues(9, primes, 1 << 12, 0)
    assert r.shape == (3, 1 << 12) and r.dtype == np.uint32
    for row, q in zip(r, primes):
        assert int(row.max()) < q
        assert row.mean() == pytest.approx((q - 1) / 2, rel=0.1)
    assert np.array_equal(r, inputs.uniform_residues(9, primes, 1 << 12, 0))
