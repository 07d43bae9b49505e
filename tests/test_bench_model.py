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
    # ModUp columns at dnum = 3, n = 40: digits of 14, 14 and 12 primes, each
    # converted to the n + alpha - alpha_j = 40, 40, 42 limbs outside it, and
    # the column-phase butterflies of the 40 inputs and 122 targets
    N = 1 << bench.LOG_N
    assert bench.digit_sizes(40, 14) == [14, 14, 12]
    assert m["modup_cols"]["mac"] == (14 * 40 + 14 * 40 + 12 * 42) * N
    assert m["modup_cols"]["shoup"] == (40 + 122) * (N // 2) * 6


@pytest.mark.parametrize("n,alpha", [(40, 14), (21, 14), (2, 14), (40, 8), (40, 40), (9, 8)])
def test_modup_macs_follow_the_digit_sizes(n, alpha):
    """The ModUp BConv work is sum_j alpha_j (n + alpha - alpha_j) N products,
    written out digit by digit from the gadget (consecutive groups of alpha
    ciphertext primes, the last one partial)."""
    N = 1 << bench.LOG_N
    primes = list(range(n))
    digits = [primes[i:i + alpha] for i in range(0, n, alpha)]
    want = 0
    for dg in digits:
        others = (n + alpha) - len(dg)   # every extended limb outside the digit
        want += len(dg) * others * N
    for op in ("hmult", "hrot"):
        assert bench.stage_work(op, n, alpha)["modup_cols"]["mac"] == want


def test_moddown_stages_split_hmult_and_hrot():
    """HRot converts all 2n limbs in ModDown; HMult with the fused rescale
    converts only the top limb there (the rest in the rescale stages); the
    per-launch model of a shared stage is the mean of the two."""
    N, n, a = 1 << bench.LOG_N, 40, 14
    hm, hr = bench.stage_work("hmult", n, a), bench.stage_work("hrot", n, a)
    assert hr["moddown_cols"]["mac"] == 2 * n * N * a
    # HMult: the top limb's ModDown (P -> q_l, alpha products per coefficient
    # and polynomial) and the rescale conversion (alpha + 1 sources to the
    # n - 1 lower primes) in one column stage; no ModDown NTT rows and no
    # separate iNTT rows before the rescale columns
    assert hm["rescale_cols"]["mac"] == 2 * N * a + 2 * (n - 1) * N * (a + 1)
    assert "rescale_cols" not in hr
    assert not {"moddown_cols", "moddown_rows", "rescale_in_rows"} & set(hm)
    assert hm["moddown_in_rows"]["shoup"] > hr["moddown_in_rows"]["shoup"]
    m = bench.kernel_models(n, a)
    assert m["moddown_in_rows"]["shoup"] == (hm["moddown_in_rows"]["shoup"] + hr["moddown_in_rows"]["shoup"]) / 2
    assert m["moddown_cols"]["mac"] == hr["moddown_cols"]["mac"]
    assert m["rescale_cols"]["mac"] == hm["rescale_cols"]["mac"]
    assert m["moddown_rows"]["shoup"] == hr["moddown_rows"]["shoup"]


@pytest.mark.parametrize("alpha", [40, 14, 8])
def test_stage_bytes_add_up_to_the_operation_bytes(alpha):
    """The compulsory bytes the stages charge add up to each operation's
    algorithmic bytes (every input read once, the key stream, the output)."""
    hm_b, hr_b = bench.algorithmic_bytes(40, alpha)
    assert sum(v["bytes"] for v in bench.stage_work("hmult", 40, alpha).values()) == hm_b
    assert sum(v["bytes"] for v in bench.stage_work("hrot", 40, alpha).values()) == hr_b


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
