"""Host-side pieces of bench.py: the algorithmic byte model (compulsory HBM
bytes per operation), the per-stage work model and the multiply-cost model
behind the integer-ALU roofline. CPU only."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


@pytest.mark.parametrize("alpha,hm_mb,hr_mb", [(40, 104.3, 83.9), (14, 147.3, 126.9), (8, 188.2, 167.8)])
def test_algorithmic_bytes_top_level(alpha, hm_mb, hr_mb):
    """HMult+rescale moves [4n + 2d'(n+alpha) + 2(n-1)] limbs, HRot
    [2n + 2d'(n+alpha) + 2n] limbs of 2^18 bytes (n = 40 limbs)."""
    hm, hr = bench.algorithmic_bytes(40, alpha)
    assert hm / 1e6 == pytest.approx(hm_mb, abs=0.05)
    assert hr / 1e6 == pytest.approx(hr_mb, abs=0.05)


def test_kernel_models_sum_their_kinds():
    m = bench.kernel_models()
    for name, v in m.items():
        assert v["modmul"] == sum(v.get(k, 0) for k in ("shoup", "mac", "smr")), name
    # ModUp columns at dnum = 3: 122 targets, 14 products per coefficient each,
    # and the column-phase butterflies of 40 inputs + 122 targets
    N = 1 << bench.LOG_N
    assert m["modup_cols"]["mac"] == 122 * N * 14
    assert m["modup_cols"]["shoup"] == (40 + 122) * (N // 2) * 6


def test_multiply_costs_follow_the_issue_rates():
    c = bench.multiply_costs({"mad_lo": 64.0, "mad_hi": 32.0, "mad_wide": 16.0})
    assert c["shoup"] == pytest.approx(1 / 32 + 2 / 64)
    assert c["mac"] == pytest.approx(1 / 16)
    assert c["smr"] == pytest.approx(1 / 16 + 1 / 64 + 1 / 32)


def test_kernel_source_hash_covers_the_kernels_only():
    names = [os.path.basename(p) for p in bench.kernel_sources()]
    assert "k_keyswitch.cu" in names and "rows.cuh" in names and "cols.cuh" in names
    assert "host.cu" not in names and "k_ablation.cu" not in names
    assert len(bench.csrc_sha1()) == 40
