"""The per-GPU file of tuned launch shapes (host logic, CPU): a second process
sets the stored shapes instead of tuning, and the file is ignored or repaired
when it belongs to another GPU, other kernels, other parameters or is damaged."""
import json
import os

import pytest

from paper_2407_13055_gb300 import tune_cache


class FakeError(RuntimeError):
    pass


class FakeK:
    """The tuner calls of the binding over a dict, with the library's shape checks."""
    CkksError = FakeError
    CKKS_COL_MODUP, CKKS_COL_MODDOWN, CKKS_COL_RS_FUSED, CKKS_ROW_PASSES = 0, 1, 2, 3

    def __init__(self, levels=40):
        self.levels = levels
        self.tune_calls = []
        self.set_calls = 0

    def ckks_tune(self, ctx, level, reps):
        self.tune_calls.append(level)
        ctx[(0, level)] = ((8, 8, 1, 1) if level % 2 else (8, 4, 1, 1), 40.0 + level)
        ctx[(1, level)] = ((4, 4, 1, 1), 20.0 + level)
        if level >= 1:
            ctx[(2, level)] = ((4, 4, 1, 2), 30.0 + level)
        ctx[(3, level)] = ((3, 1, 1, 1), 25.0)

    def ckks_tune_get(self, ctx, kernel, level):
        shape, us = ctx.get((kernel, level), ((0, 0, 0, 0), 0.0))
        return tuple(shape) + (us,)

    def ckks_tune_set(self, ctx, kernel, level, tc, sl=4, z=1, tp=1):
        self.set_calls += 1
        if not 0 <= level < self.levels or kernel not in (0, 1, 2, 3):
            raise FakeError("tune: bad level or kernel")
        if tc == 0:
            ctx.pop((kernel, level), None)
            return
        if kernel == 3:
            if not 2 <= tc <= 5:
                raise FakeError("tune: row passes")
            ctx[(kernel, level)] = ((tc, 1, 1, 1), 0.0)
            return
        if tc not in (4, 8) or sl not in (2, 4, 8) or not 1 <= z <= 4 or tp not in (1, 2, 8, 16):
            raise FakeError("tune: shape")
        ctx[(kernel, level)] = ((tc, sl, z, tp), 0.0)


GPU = {"name": "NVIDIA GB300", "uuid": "GPU-1234", "sms": 152, "cc": "10.3"}
PKEY = tune_cache.params_key(16, [97, 193, 257], [353, 449], 3)
LEVELS = [39, 20, 1, 0]


def _run(path, gpu=GPU, digest="d1", levels=LEVELS, retune=False, pkey=PKEY):
    K, ctx = FakeK(), {}
    store = tune_cache.TuneStore(str(path), gpu, digest=digest)
    out, loaded, tuned = tune_cache.tune_or_load(K, ctx, levels, pkey, store, reps=2, retune=retune)
    return K, ctx, out, loaded, tuned


def test_second_process_sets_the_stored_shapes_without_tuning(tmp_path):
    f = tmp_path / "tune.json"
    K1, ctx1, out1, loaded1, tuned1 = _run(f)
    assert loaded1 == [] and tuned1 == sorted(LEVELS) and sorted(K1.tune_calls) == sorted(LEVELS)
    doc = json.loads(f.read_text())
    assert doc["format"] == 1 and doc["gpu"] == GPU
    lv39 = doc["entries"][f"{PKEY}@d1"]["39"]
    assert lv39["modup_cols"] == [8, 8, 1, 1, 79.0] and lv39["row_passes"][0] == 3
    assert "rescale_cols" not in doc["entries"][f"{PKEY}@d1"]["0"]   # untuned at level 0: no entry
    K2, ctx2, out2, loaded2, tuned2 = _run(f)
    assert K2.tune_calls == [] and tuned2 == [] and loaded2 == sorted(LEVELS)
    assert ctx2.keys() == ctx1.keys()
    for k in ctx1:
        assert ctx2[k][0] == ctx1[k][0]
    assert out2 == out1          # the stored times are reported for loaded levels


def test_new_levels_are_tuned_and_added(tmp_path):
    f = tmp_path / "tune.json"
    _run(f, levels=[39])
    K, _, _, loaded, tuned = _run(f, levels=[39, 7])
    assert loaded == [39] and tuned == [7] and K.tune_calls == [7]
    entries = json.loads(f.read_text())["entries"][f"{PKEY}@d1"]
    assert set(entries) == {"7", "39"}


def test_file_of_another_gpu_is_ignored_and_replaced(tmp_path):
    f = tmp_path / "tune.json"
    _run(f)
    other = dict(GPU, uuid="GPU-9999")
    K, _, _, loaded, tuned = _run(f, gpu=other)
    assert loaded == [] and sorted(K.tune_calls) == sorted(LEVELS)
    assert json.loads(f.read_text())["gpu"]["uuid"] == "GPU-9999"


def test_other_kernels_or_parameters_do_not_match(tmp_path):
    f = tmp_path / "tune.json"
    _run(f)
    K, _, _, loaded, _ = _run(f, digest="d2")
    assert loaded == [] and sorted(K.tune_calls) == sorted(LEVELS)
    entries = json.loads(f.read_text())["entries"]
    assert {f"{PKEY}@d1", f"{PKEY}@d2"} <= set(entries)     # the old digest's entries are kept
    other = tune_cache.params_key(16, [97, 193, 257], [353, 449], 1)
    K, _, _, loaded, _ = _run(f, pkey=other)
    assert loaded == [] and K.tune_calls


def test_damaged_entry_is_cleared_and_retuned(tmp_path):
    f = tmp_path / "tune.json"
    _run(f, levels=[39, 20])
    doc = json.loads(f.read_text())
    ent = doc["entries"][f"{PKEY}@d1"]
    ent["39"]["modup_cols"] = [6, 4, 1, 1, 10.0]      # no such shape
    ent["20"]["bogus_kernel"] = [8, 4, 1, 1, 1.0]
    f.write_text(json.dumps(doc))
    K, ctx, out, loaded, tuned = _run(f, levels=[39, 20])
    assert loaded == [] and tuned == [20, 39]
    assert out[39]["modup_cols"][:4] == (8, 8, 1, 1)
    repaired = json.loads(f.read_text())["entries"][f"{PKEY}@d1"]
    assert repaired["39"]["modup_cols"][:4] == [8, 8, 1, 1] and "bogus_kernel" not in repaired["20"]


def test_unreadable_file_and_retune(tmp_path):
    f = tmp_path / "tune.json"
    f.write_text("{not json")
    K, _, _, loaded, tuned = _run(f)
    assert loaded == [] and tuned == sorted(LEVELS)
    json.loads(f.read_text())
    K, _, _, loaded, tuned = _run(f, retune=True)
    assert loaded == [] and tuned == sorted(LEVELS)
    assert [p for p in os.listdir(tmp_path) if p.startswith(".tune-")] == []   # no temporary left


def test_without_a_store_every_level_is_tuned(tmp_path):
    K, ctx = FakeK(), {}
    out, loaded, tuned = tune_cache.tune_or_load(K, ctx, [3, 3, 2], PKEY, None)
    assert tuned == [2, 3] and K.tune_calls == [2, 3] and set(out) == {2, 3}


def test_parameter_key_separates_parameter_sets():
    q, p = [97, 193, 257], [353, 449]
    base = tune_cache.params_key(16, q, p, 3)
    assert base == tune_cache.params_key(16, list(q), tuple(p), 3)
    assert base != tune_cache.params_key(12, q, p, 3)
    assert base != tune_cache.params_key(16, q, p, 2)
    assert base != tune_cache.params_key(16, [97, 193, 449], [353, 257], 3)
    w1 = tune_cache.params_key(16, q, p, 3, [(0, 2), (0, 3)])
    assert w1 != base and w1 != tune_cache.params_key(16, q, p, 3, [(1, 2), (0, 3)])


def test_default_path(tmp_path, monkeypatch):
    monkeypatch.delenv("CKKS_TUNE_CACHE", raising=False)
    monkeypatch.setenv("XDG_CACHE_HOME", str(tmp_path))
    p = tune_cache.default_path({"name": "NVIDIA GB300 / x", "uuid": "GPU-ab:cd"})
    assert p == os.path.join(str(tmp_path), "paper_2407_13055_gb300", "tune-NVIDIA_GB300_x-GPU-ab_cd.json")
    monkeypatch.setenv("CKKS_TUNE_CACHE", str(tmp_path))
    assert tune_cache.default_path(GPU) == os.path.join(str(tmp_path), "tune-NVIDIA_GB300-GPU-1234.json")
    monkeypatch.setenv("CKKS_TUNE_CACHE", str(tmp_path / "mine.json"))
    assert tune_cache.default_path(GPU) == str(tmp_path / "mine.json")


def test_sources_digest_follows_the_sources(tmp_path):
    (tmp_path / "a.cu").write_text("x")
    (tmp_path / "notes.txt").write_text("ignored")
    d1 = tune_cache.sources_digest(str(tmp_path))
    (tmp_path / "notes.txt").write_text("changed")
    assert tune_cache.sources_digest(str(tmp_path)) == d1
    (tmp_path / "a.cu").write_text("y")
    assert tune_cache.sources_digest(str(tmp_path)) != d1
    assert len(tune_cache.sources_digest()) == 16


def test_kernel_names_match_the_binding():
    K = pytest.importorskip("paper_2407_13055_gb300.ckks")
    ids = tune_cache.kernel_names(K)
    assert sorted(ids.values()) == [0, 1, 2, 3]
