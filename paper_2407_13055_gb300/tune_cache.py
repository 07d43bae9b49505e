"""Per-GPU store of the fine-tuner's launch shapes (Sec. 4.2, "Fine-tuning"; Sec. 6).

``ckks_tune`` times every candidate launch shape of the three BConv column
kernels and the row-phase forms at one level and keeps the fastest. The choice
depends on the GPU, the parameter set and the kernels, never on the data, and
every shape computes identical values. This module writes the choices to one
JSON file per GPU and sets them again on a later context with
``ckks_tune_set``, so a process can skip the timing and two runs use the same
shapes.

File layout::

    {"format": 1,
     "gpu": {"name": ..., "uuid": ..., "sms": ..., "cc": "10.3"},
     "entries": {"<parameter key>@<kernel digest>":
                  {"<level>": {"modup_cols": [tc, sl, z, tp, us], ...}}}}

The parameter key names the ring degree, the prime counts, dnum and a digest of
the primes; the kernel digest is a hash of the library's CUDA sources, so
entries written by other kernels are ignored (and kept) and the levels are
tuned again. Writes go to a temporary file in the same folder that replaces
the old one, so a reader never sees half a file.
"""
from __future__ import annotations

import hashlib
import json
import os
import re
import tempfile

FORMAT = 1
CSRC = os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")


def kernel_names(K) -> dict:
    """Tuned kernels of the library: {name: kernel id of ckks_tune_get/set}."""
    return {"modup_cols": K.CKKS_COL_MODUP, "moddown_cols": K.CKKS_COL_MODDOWN,
            "rescale_cols": K.CKKS_COL_RS_FUSED, "row_passes": K.CKKS_ROW_PASSES}


def sources_digest(folder: str = CSRC) -> str:
    """Hash of the CUDA/C++ sources the kernels are built from (names and bytes)."""
    h = hashlib.sha256()
    for name in sorted(os.listdir(folder)):
        if name.endswith((".cu", ".cuh", ".h", ".cpp")):
            h.update(name.encode())
            with open(os.path.join(folder, name), "rb") as f:
                h.update(f.read())
    return h.hexdigest()[:16]


def params_key(log_n: int, q, p, dnum: int, levels=None) -> str:
    """Parameter set of a context: ring degree, prime counts, dnum, digest of
    the primes and of the level windows (start, count) when they are given."""
    text = ",".join(str(int(v)) for v in q) + "|" + ",".join(str(int(v)) for v in p)
    if levels is not None:
        text += "|" + ";".join(f"{int(s)}+{int(n)}" for s, n in levels)
    h = hashlib.sha256(text.encode())
    return f"logn{int(log_n)}-q{len(q)}-p{len(p)}-dnum{int(dnum)}-{h.hexdigest()[:12]}"


def gpu_identity(device: int = 0) -> dict:
    """Name, UUID, SM count and compute capability of a CUDA device."""
    import torch
    pr = torch.cuda.get_device_properties(device)
    uuid = str(getattr(pr, "uuid", "") or "")
    return {"name": pr.name, "uuid": uuid, "sms": int(pr.multi_processor_count), "cc": f"{pr.major}.{pr.minor}"}


def default_path(gpu: dict) -> str:
    """The GPU's tune file: $CKKS_TUNE_CACHE when it names a file; the GPU's own
    file in $CKKS_TUNE_CACHE when that is a folder (or ends in a separator);
    else the GPU's own file under the user's cache folder."""
    tag = re.sub(r"[^A-Za-z0-9_.-]+", "_", f"{gpu.get('name', 'gpu')}-{gpu.get('uuid') or 'nouuid'}")
    name = f"tune-{tag}.json"
    env = os.environ.get("CKKS_TUNE_CACHE")
    if env:
        if env.endswith(os.sep) or os.path.isdir(env):
            return os.path.join(env, name)
        return env
    root = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(root, "paper_2407_13055_gb300", name)


class TuneStore:
    """The tuned shapes of one GPU, read from and written to one JSON file."""

    def __init__(self, path: str, gpu: dict, digest: str | None = None):
        self.path = path
        self.gpu = dict(gpu)
        self.digest = digest if digest is not None else sources_digest()
        self.entries: dict = {}
        self.load()

    def load(self) -> bool:
        """Read the file; False (and no entries) when it is absent, unreadable,
        of another format or written for another GPU."""
        self.entries = {}
        try:
            with open(self.path) as f:
                doc = json.load(f)
        except (OSError, ValueError):
            return False
        if not isinstance(doc, dict) or doc.get("format") != FORMAT or not isinstance(doc.get("entries"), dict):
            return False
        g = doc.get("gpu") or {}
        if any(g.get(k) != self.gpu.get(k) for k in ("name", "uuid", "sms", "cc")):
            return False
        self.entries = doc["entries"]
        return True

    def _key(self, pkey: str) -> str:
        return f"{pkey}@{self.digest}"

    def lookup(self, pkey: str, level: int) -> dict | None:
        """Stored shapes {kernel name: [tc, sl, z, tp, us]} of a level, or None."""
        lv = self.entries.get(self._key(pkey), {}).get(str(int(level)))
        return lv if isinstance(lv, dict) else None

    def record(self, pkey: str, level: int, shapes: dict):
        """Keep the shapes of a level ({name: (tc, sl, z, tp, us)}; tc = 0 = no entry)."""
        clean = {}
        for name, v in shapes.items():
            tc, sl, z, tp, us = v
            if int(tc) > 0:
                clean[name] = [int(tc), int(sl), int(z), int(tp), round(float(us), 3)]
        self.entries.setdefault(self._key(pkey), {})[str(int(level))] = clean

    def save(self):
        """Write every entry (atomic replace of the file)."""
        folder = os.path.dirname(os.path.abspath(self.path))
        os.makedirs(folder, exist_ok=True)
        doc = {"format": FORMAT, "gpu": self.gpu, "entries": self.entries}
        fd, tmp = tempfile.mkstemp(prefix=".tune-", suffix=".json", dir=folder)
        try:
            with os.fdopen(fd, "w") as f:
                json.dump(doc, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)
        except BaseException:
            if os.path.exists(tmp):
                os.unlink(tmp)
            raise


def apply(K, ctx, level: int, shapes: dict) -> bool:
    """Set stored shapes on a context with ckks_tune_set. A shape the library
    refuses (CKKS_EINVAL: a damaged or foreign entry) clears the level's
    entries again and returns False, so the caller tunes it."""
    ids = kernel_names(K)
    try:
        for name, v in shapes.items():
            if name not in ids:
                raise ValueError(f"unknown tuned kernel {name!r}")
            tc, sl, z, tp = (int(x) for x in v[:4])
            K.ckks_tune_set(ctx, ids[name], level, tc, sl, z, tp)
        return True
    except (K.CkksError, ValueError, TypeError):
        for name, kid in ids.items():
            try:
                K.ckks_tune_set(ctx, kid, level, 0, 1, 1, 1)
            except K.CkksError:
                pass
        return False


def read_level(K, ctx, level: int) -> dict:
    """The context's current shapes of a level: {name: (tc, sl, z, tp, us)}."""
    return {name: K.ckks_tune_get(ctx, kid, level) for name, kid in kernel_names(K).items()}


def tune_or_load(K, ctx, levels, pkey: str, store: TuneStore | None, reps: int = 3, retune: bool = False):
    """For each level: set the stored shapes when the store has them (and
    `retune` is off), else run ckks_tune and record its choice. Saves the store
    when anything was tuned. Returns ({level: shapes}, levels loaded, levels tuned)."""
    loaded, tuned, out = [], [], {}
    for lv in sorted(set(int(x) for x in levels)):
        entry = None if (store is None or retune) else store.lookup(pkey, lv)
        if entry is not None and apply(K, ctx, lv, entry):
            loaded.append(lv)
            # ckks_tune_set records no time: report the stored one
            out[lv] = {name: (tuple(entry[name][:4]) + (float(entry[name][4]),)) if name in entry else v
                       for name, v in read_level(K, ctx, lv).items()}
            continue
        K.ckks_tune(ctx, lv, reps)
        tuned.append(lv)
        out[lv] = read_level(K, ctx, lv)
        if store is not None:
            store.record(pkey, lv, out[lv])
    if store is not None and tuned:
        store.save()
    return out, loaded, tuned
