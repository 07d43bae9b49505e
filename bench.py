#!/usr/bin/env python
"""Benchmark: HMult / HRot key-switch operations per second at N = 2^16 on GB300.

Workload (single-op key switching at N = 2^16): 40 ciphertext primes
(q_0 31-bit, q_1..q_39 30-bit), alpha = 14 auxiliary 31-bit primes, dnum = 3,
top level (40 limbs), ternary secret of Hamming weight 192, sigma = 3.2,
scale 2^30. One step = for each of B = 256 resident ciphertexts one HMult
(tensor + relinearize + rescale) and one HRot by 1 slot, so a step runs every
stage of the hot path (NTT/iNTT, tensor, ModUp BConv, KeyMult + MAC,
automorphism, ModDown, rescale). The 256 input ciphertexts (5.4 GB) and two
evaluation keys (170 MB) exceed the 129 MB L2, so consecutive operations
stream cold data (no explicit flush). Inputs are fresh encryptions of
messages uniform in [-1, 1] made by the library itself; keys are random-free
outputs of its key generation.

`--impl reference` times the CPU oracle (the only reference there is: the
paper ships no code) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2407_13055_gb300 import tune_cache  # noqa: E402  (host-side file of tuned shapes)

LOG_N, L, DNUM, ALPHA, HW, SCALE = 16, 40, 3, 14, 192, 2.0**30
LEVEL = L - 1
BATCH = 256          # distinct resident ciphertexts per timed step (5.4 GB, far above L2)
E2E_HOST = 16        # distinct pinned host ciphertexts cycled by the end-to-end leg
METRIC = "HMult/HRot key-switch ops/sec at N=2^16 (1 GB300)"
UNIT = "key-switch ops/s"
LIMB_BYTES = (1 << LOG_N) * 4


def workload_config(extra=None):
    cfg = {
        "workload": "single-op key switching, N=2^16, 40 primes (28-31 bit), dnum=3 (alpha=14), top level (40 limbs), "
                    "HMult+relin+rescale and HRot(1) per ciphertext",
        "N": 1 << LOG_N, "limbs": L, "alpha": ALPHA, "dnum": DNUM, "level": LEVEL, "secret_hw": HW,
        "batch_ciphertexts": BATCH, "ops_per_step": 2 * BATCH,
        "l2": f"inputs larger than L2 ({BATCH} ciphertexts = {BATCH * 2 * L * (1 << LOG_N) * 4 / 1e9:.2f} GB + 2 keys "
              f"= 170 MB, rotated; no flush)",
    }
    if extra:
        cfg.update(extra)
    return cfg


def algorithmic_bytes(n=L, alpha=ALPHA):
    """Compulsory HBM bytes per op (inputs + truncated evk + outputs)."""
    d = -(-n // alpha)
    hmult = (4 * n + 2 * d * (n + alpha) + 2 * (n - 1)) * LIMB_BYTES
    hrot = (2 * n + 2 * d * (n + alpha) + 2 * n) * LIMB_BYTES
    return hmult, hrot


def digit_sizes(n=L, alpha=ALPHA):
    """alpha_j of each active digit at n limbs (the last one may be partial)."""
    return [min(alpha, n - j * alpha) for j in range(-(-n // alpha))]


def stage_work(op, n=L, alpha=ALPHA):
    """Algorithmic work of each pipeline stage of one operation (op "hmult":
    HMult + relinearize + rescale; "hrot": HRot) at n limbs: compulsory HBM
    bytes (each input limb counted where it is first read, the evaluation-key
    stream, the output; scratch is meant to stay in L2) and modular
    multiplications by kind: `shoup` (NTT butterflies and products by a
    constant: one mad.hi and two mad.lo), `mac` (BConv products: one mad.wide
    each, reduced lazily) and `smr` (variable x variable: mad.wide, mad.lo,
    mad.hi; a full product mod q is two). Butterflies per limb: N/2 x 10 in
    the row phase (W = 1024), N/2 x 6 in the column phase (H = 64). BConv:
    alpha_j (n + alpha - alpha_j) products per coefficient for ModUp digit j,
    K per target for the ModDown (K = alpha) and fused-rescale (alpha + 1)
    conversions."""
    N = 1 << LOG_N
    a_j = digit_sizes(n, alpha)
    d, ext = len(a_j), n + alpha
    row, col = N // 2 * 10, N // 2 * 6
    targets = sum(ext - a for a in a_j)
    lb = LIMB_BYTES
    hm = op == "hmult"
    w = {
        # tensor a1 a2 (HMult) or phi(a) (HRot) formed while loading, iNTT rows
        "ks_in_rows": dict(bytes=(2 * n if hm else n) * lb, shoup=n * row, smr=2 * n * N if hm else 0),
        "modup_cols": dict(shoup=(n + targets) * col, mac=N * sum(a * (ext - a) for a in a_j)),
        "modup_rows": dict(shoup=targets * row),
        "keymult": dict(bytes=2 * d * ext * lb, smr=2 * d * ext * N),
    }
    if hm:
        # the iNTT rows also take E = acc_l P^-1 + d_l of the top limb (b1, b2
        # top limbs read, d0 / d1 of that limb re-formed); one column kernel
        # per tile iNTTs the P limbs and E, converts P -> q_l, forms the top
        # limb's ModDown output V = E - z P^-1 and converts the P limbs and V
        # to the n - 1 lower primes (the rescale), then their NTT columns
        w["moddown_in_rows"] = dict(bytes=2 * lb, shoup=2 * (alpha + 1) * row + 2 * N, smr=6 * N)
        w["rescale_cols"] = dict(shoup=2 * (alpha + 1) * col + 2 * N + 2 * (n - 1) * col,
                                 mac=2 * N * alpha + 2 * (n - 1) * N * (alpha + 1))
        # NTT rows + (A - w)(P q_l)^-1 + d q_l^-1 with d0 / d1 re-formed from
        # the inputs (b1, b2 read here first), output 2(n - 1) limbs
        w["rescale_rows"] = dict(bytes=4 * (n - 1) * lb, shoup=2 * (n - 1) * (row + 2 * N),
                                 smr=6 * (n - 1) * N)
    else:
        w["moddown_in_rows"] = dict(shoup=2 * alpha * row)
        w["moddown_cols"] = dict(shoup=2 * (alpha + n) * col, mac=2 * n * N * alpha)
        # NTT rows + (A - z) P^-1 + phi(b): b read, output 2n limbs
        w["moddown_rows"] = dict(bytes=3 * n * lb, shoup=2 * n * row + 2 * n * N)
    for v in w.values():
        for k in ("bytes", "shoup", "mac", "smr"):
            v.setdefault(k, 0)
        v["modmul"] = v["shoup"] + v["mac"] + v["smr"]
    return w


def kernel_models(n=L, alpha=ALPHA):
    """Per-launch work of each stage in the bench's one-lane profile, which
    alternates HMult + rescale and HRot: the mean of the two operations' work
    for the stages both run (the key-switch stages), HMult's alone for the
    rescale stages and HRot's alone for the ModDown NTT rows."""
    hm, hr = stage_work("hmult", n, alpha), stage_work("hrot", n, alpha)
    out = {}
    for k in list(hm) + [k for k in hr if k not in hm]:
        ws = [x[k] for x in (hm, hr) if k in x]
        out[k] = {kk: sum(x[kk] for x in ws) / len(ws) for kk in ("bytes", "shoup", "mac", "smr", "modmul")}
    return out


def multiply_costs(rates):
    """SM clocks per modular product of each kind at the measured issue rates
    (instructions per SM per clock of mad.lo, mad.hi, mad.wide)."""
    lo, hi, wide = 1.0 / rates["mad_lo"], 1.0 / rates["mad_hi"], 1.0 / rates["mad_wide"]
    return {"shoup": hi + 2 * lo, "mac": wide, "smr": wide + lo + hi}


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the
# one-lane pipeline's kernels from one ncu launch list with those two metrics
# (cold cache; the command is recorded with the committed profile summary;
# stages that two kernels share: the mean of the two), keyed by stage. They
# describe the kernel sources they were taken on: when the SHA-1 of those
# sources (kernel_sources) differs, the figures are stale and the bench
# reports null.
NCU_TRAFFIC = {
    "sources_sha1": "7752ec4617116707750c987e104ac7492e35ba55",
    "bytes_per_launch": {"modup_cols": 10.58e6, "keymult": 135.59e6, "modup_rows": 60.32e6,
                         "moddown_in_rows": 15.76e6, "moddown_cols": 7.40e6, "moddown_rows": 74.29e6,
                         "rescale_cols": 7.95e6, "rescale_rows": 118.13e6, "ks_in_rows": 37.31e6},
}


# Sources of the key-switch pipeline's kernels (the ones the ncu capture
# covers): the headers they include, the launch sequences and the column
# kernels' instantiations. Host code and the ablation probes are not part of it.
def kernel_sources():
    d = os.path.join(ROOT, "paper_2407_13055_gb300", "csrc")
    return [os.path.join(d, n) for n in sorted(os.listdir(d))
            if n.endswith((".cuh", ".h")) or n == "k_keyswitch.cu" or n.startswith("k_cols_")]


def csrc_sha1():
    import hashlib
    h = hashlib.sha1()
    for path in kernel_sources():
        with open(path, "rb") as f:
            h.update(os.path.basename(path).encode() + b"\0" + f.read())
    return h.hexdigest()


def ncu_traffic(stage):
    if csrc_sha1() != NCU_TRAFFIC["sources_sha1"]:
        return None
    return NCU_TRAFFIC["bytes_per_launch"].get(stage)


FORCED = {"col_shape": None, "row_passes": None}   # set from --col-shape / --row-passes
# per-GPU file of tuned shapes (tune_cache.TuneStore) and what tune_levels did with it
TUNE = {"store": None, "retune": False, "loaded": 0, "tuned": 0}


def tune_levels(K, ctx, levels, enabled, reps=3, pkey=None):
    """Set the fine-tuner's shapes at each level (outside any timed region) and
    return the chosen column shapes and row-phase passes {level: {kernel: (tc,
    sl, z, tp, us)}} (row_passes: tc = passes). Levels found in the per-GPU
    tune file under the parameter key `pkey` are set from it; the others are
    tuned and written to it. A shape or row form given on the command line
    replaces the tuner's choice for every level."""
    names = {K.CKKS_COL_MODUP: "modup_cols", K.CKKS_COL_MODDOWN: "moddown_cols", K.CKKS_COL_RS_FUSED: "rescale_cols",
             K.CKKS_ROW_PASSES: "row_passes"}
    forced = FORCED["col_shape"] is not None or FORCED["row_passes"] is not None
    if not enabled and not forced:
        return None
    levels = sorted(set(int(x) for x in levels))
    stored = {}
    if enabled:
        store = TUNE["store"] if pkey is not None else None
        stored, loaded, tuned = tune_cache.tune_or_load(K, ctx, levels, pkey, store, reps, TUNE["retune"])
        TUNE["loaded"] += len(loaded)
        TUNE["tuned"] += len(tuned)
    out = {}
    for lv in levels:
        if FORCED["col_shape"] is not None:
            for k in (K.CKKS_COL_MODUP, K.CKKS_COL_MODDOWN, K.CKKS_COL_RS_FUSED):
                if k == K.CKKS_COL_RS_FUSED and lv < 1:
                    continue
                K.ckks_tune_set(ctx, k, lv, *FORCED["col_shape"])
        if FORCED["row_passes"] is not None:
            K.ckks_tune_set(ctx, K.CKKS_ROW_PASSES, lv, FORCED["row_passes"], 1, 1, 1)
        out[lv] = {nm: K.ckks_tune_get(ctx, k, lv) for k, nm in names.items()}
        if not forced and lv in stored:
            out[lv] = stored[lv]
    return out


def open_tune_store(args, device):
    """The per-GPU file of tuned shapes (--tune-file, else $CKKS_TUNE_CACHE,
    else one file per GPU in the user's cache folder); none with --no-tune or
    --tune-file none."""
    if args.no_tune or (args.tune_file or "").lower() == "none":
        return
    gpu = tune_cache.gpu_identity(device)
    TUNE["store"] = tune_cache.TuneStore(args.tune_file or tune_cache.default_path(gpu), gpu)
    TUNE["retune"] = bool(args.retune)


def tune_file_summary():
    st = TUNE["store"]
    if st is None:
        return None
    return {"path": st.path, "levels_loaded": TUNE["loaded"], "levels_tuned": TUNE["tuned"],
            "kernels_digest": st.digest}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# reference arm / CPU baseline: the oracle on a bounded sample
# ----------------------------------------------------------------------------

def time_oracle(max_pairs: int = 1, budget_s: float = 0.0):
    """Time the CPU oracle on (HMult+rescale, HRot) pairs of the workload:
    at least one pair, more while under `budget_s` seconds and `max_pairs`.
    Returns (ops/s, seconds, pairs, description)."""
    from oracle import oracle as O
    from paper_2407_13055_gb300 import inputs
    O.build()
    P = O.make_params(LOG_N, L, DNUM, ALPHA)
    n = P.n
    allp = P.all_primes()
    evk = np.stack([np.stack([inputs.uniform_residues(5, allp, n, 10 * j + t) for t in range(2)])
                    for j in range(DNUM)])
    ct = [np.stack([inputs.uniform_residues(6, P.q, n, 2 * i + t) for t in range(2)]) for i in range(2)]
    k = O.rot_k(1, LOG_N)
    pairs, dt = 0, 0.0
    while pairs < 1 or (pairs < max_pairs and dt * (pairs + 1) / pairs < budget_s):
        t0 = time.perf_counter()
        O.hmult(P, ct[0], ct[1], evk, rescale=True)
        O.hrot(P, ct[0], k, evk)
        dt += time.perf_counter() - t0
        pairs += 1
    desc = f"{pairs} HMult+rescale and {pairs} HRot(1) of the same workload on 1 host thread"
    return 2 * pairs / dt, dt, pairs, desc


# All-core CPU baseline: independent oracle samples in a spawned process
# pool, one (HMult+rescale, HRot) pair per worker, timed by wall clock.
_OW = None


def _oracle_worker_init():
    global _OW
    from oracle import oracle as O
    from paper_2407_13055_gb300 import inputs
    P = O.make_params(LOG_N, L, DNUM, ALPHA)
    allp = P.all_primes()
    evk = np.stack([np.stack([inputs.uniform_residues(5, allp, P.n, 10 * j + t) for t in range(2)])
                    for j in range(DNUM)])
    ct = [np.stack([inputs.uniform_residues(6, P.q, P.n, 2 * i + t) for t in range(2)]) for i in range(2)]
    _OW = (O, P, evk, ct, O.rot_k(1, LOG_N))


def _oracle_worker_ready(_):
    time.sleep(0.5)
    return _OW is not None


def _oracle_worker_pair(_):
    O, P, evk, ct, k = _OW
    t0 = time.perf_counter()
    O.hmult(P, ct[0], ct[1], evk, rescale=True)
    O.hrot(P, ct[0], k, evk)
    return time.perf_counter() - t0


def _oracle_worker_op(i):
    """One key-switching operation of the workload: HMult+rescale on even
    workers, HRot(1) on odd ones."""
    O, P, evk, ct, k = _OW
    t0 = time.perf_counter()
    if i % 2 == 0:
        O.hmult(P, ct[0], ct[1], evk, rescale=True)
    else:
        O.hrot(P, ct[0], k, evk)
    return time.perf_counter() - t0


def time_oracle_all_cores(rounds: int = 1, warmup: int = 0, budget_s: float = 0.0):
    """(ops/s, wall seconds of the timed rounds, workers, description, rounds
    timed): each round is one pair per host core; `warmup` untimed rounds
    first; more than one timed round only while under `budget_s`."""
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    nw = os.cpu_count() or 1
    with mp.get_context("spawn").Pool(nw, initializer=_oracle_worker_init) as pool:
        pool.map(_oracle_worker_ready, range(nw), chunksize=1)
        for _ in range(warmup):
            pool.map(_oracle_worker_pair, range(nw), chunksize=1)
        done, wall = 0, 0.0
        while done < 1 or (done < rounds and wall * (done + 1) / done < budget_s):
            t0 = time.perf_counter()
            pool.map(_oracle_worker_pair, range(nw), chunksize=1)
            wall += time.perf_counter() - t0
            done += 1
    desc = (f"{done} x {nw} HMult+rescale and HRot(1) pairs of the same workload, one pair per worker "
            f"process per round ({nw} host cores)")
    return 2 * nw * done / wall, wall, nw, desc, done


def run_reference(args, rank, world):
    if rank != 0:
        return
    # The oracle as it stands on every host core (spawned workers). A step is
    # one key-switching operation per core, half of them HMult+rescale and half
    # HRot(1): exactly `--warmup` untimed steps, then exactly `--steps` timed
    # ones, so that the default 5 + 20 steps take about two minutes.
    import multiprocessing as mp
    from oracle import oracle as O
    O.build()
    nw = os.cpu_count() or 1
    steps, warmup = max(1, args.steps), max(0, args.warmup)
    with mp.get_context("spawn").Pool(nw, initializer=_oracle_worker_init) as pool:
        pool.map(_oracle_worker_ready, range(nw), chunksize=1)
        for _ in range(warmup):
            pool.map(_oracle_worker_op, range(nw), chunksize=1)
        t0 = time.perf_counter()
        for _ in range(steps):
            pool.map(_oracle_worker_op, range(nw), chunksize=1)
        dt = time.perf_counter() - t0
    ops_per_s = nw * steps / dt
    desc = (f"{steps} steps of {nw} key-switching operations, one per worker process per step "
            f"({(nw + 1) // 2} HMult+rescale and {nw // 2} HRot(1); {nw} host cores)")
    line = {
        "impl": "reference", "metric": METRIC, "value": ops_per_s, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warmup, "ms_per_step": 1e3 * dt / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": workload_config({"sample": desc, "step": f"one key-switching operation on each of {nw} "
                                                           "host cores"}),
        "cpu_baseline": {"value": ops_per_s, "unit": UNIT, "cores": nw, "kind": "oracle", "sample": desc},
        "e2e": {"value": ops_per_s, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# native arm
# ----------------------------------------------------------------------------

def run_native(args, rank, world, local_rank):
    import torch
    from paper_2407_13055_gb300 import ckks as K
    from paper_2407_13055_gb300 import inputs, replicas

    # CPU baseline first (rank 0 at N = 1 only), before any GPU work.
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v1, dt1, _, desc1 = time_oracle(1)
        v, dt, nw, desc, _ = time_oracle_all_cores()
        cpu = {"value": v, "unit": UNIT, "cores": nw, "kind": "oracle", "sample": desc, "seconds": dt,
               "single_thread": {"value": v1, "cores": 1, "sample": desc1, "seconds": dt1}}

    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    q, p = K.ckks_gen_primes(LOG_N, L, ALPHA)
    ctx = K.ckks_ctx_create(LOG_N, q, p, DNUM, scale=SCALE, secret_hw=HW, seed=rank,
                            stream=stream.cuda_stream)
    K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL if args.pdl == "on" else 0)
    sk = K.ckks_keygen_secret(ctx, 1000 + rank)
    rk = K.ckks_keygen_relin(ctx, sk, 2000 + rank)
    gk = K.ckks_keygen_rot(ctx, sk, 1, 3000 + rank)
    cts = []
    for i in range(BATCH):
        pt = K.ckks_encode(ctx, inputs.messages(100 + i, (1 << LOG_N) // 2), LEVEL, SCALE)
        cts.append(K.ckks_encrypt(ctx, sk, pt, 200 + i))
        K.ckks_free(pt)
    # execution lanes: lane 0 is the context itself, the others are clones
    # with their own stream and scratch; lane l takes ciphertexts i = l mod lanes
    streams = [stream] + [torch.cuda.Stream() for _ in range(args.lanes - 1)]
    lanes = [ctx] + [K.ckks_ctx_clone(ctx, s_.cuda_stream) for s_ in streams[1:]]
    outs_m = [K.ckks_ct_create(ctx, LEVEL) for _ in lanes]
    outs_r = [K.ckks_ct_create(ctx, LEVEL) for _ in lanes]
    tuned = tune_levels(K, ctx, [LEVEL], not args.no_tune, pkey=tune_cache.params_key(LOG_N, q, p, DNUM))

    def step(n_lanes):
        for i in range(BATCH):
            l = i % n_lanes
            K.ckks_hmult(lanes[l], cts[i], cts[(i + 1) % BATCH], rk, K.CKKS_RESCALE, outs_m[l])
            K.ckks_hrot(lanes[l], cts[i], 1, gk, outs_r[l])

    # the timed step through the batch API: the same 2 x BATCH independent
    # operations (own outputs), lane l taking HMult and HRot of ciphertexts
    # i = l mod lanes, issued by the library (direct) or replayed as one CUDA
    # graph per step (graph); "python" issues them one call at a time
    batch, outs_b = None, []
    if args.issue != "python":
        nl = args.lanes
        outs_b = [K.ckks_ct_create(ctx, LEVEL) for _ in range(2 * BATCH)]
        batch_ops = []
        for g0 in range(0, BATCH, nl):
            grp = range(g0, min(g0 + nl, BATCH))
            batch_ops += [dict(op=K.CKKS_OP_HMULT, a=cts[i], b=cts[(i + 1) % BATCH], evk=rk,
                               flags=K.CKKS_RESCALE, out=outs_b[2 * i]) for i in grp]
            batch_ops += [dict(op=K.CKKS_OP_HROT, a=cts[i], r=1, evk=gk, out=outs_b[2 * i + 1]) for i in grp]
        batch = K.ckks_batch_create(ctx, batch_ops, nl, args.issue == "graph")

    def barrier():
        replicas.barrier()
        torch.cuda.synchronize()

    def timed(n_steps, n_lanes, use_batch=False):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        if use_batch:
            for _ in range(n_steps):
                K.ckks_batch_run(ctx, batch)
            ev1.record(stream)
            barrier()
            return ev0.elapsed_time(ev1)
        for s_ in streams[1:n_lanes]:
            s_.wait_event(ev0)
        for _ in range(n_steps):
            step(n_lanes)
        for s_ in streams[1:n_lanes]:
            e = torch.cuda.Event()
            e.record(s_)
            stream.wait_event(e)
        ev1.record(stream)
        barrier()
        return ev0.elapsed_time(ev1)

    for _ in range(args.warmup):
        if batch is not None:
            K.ckks_batch_run(ctx, batch)
        else:
            step(args.lanes)
    barrier()
    launches0 = K.ckks_launch_count()
    with ClockSampler(local_rank) as clk:
        torch.cuda.nvtx.range_push("timed")
        ms = timed(args.steps, args.lanes, batch is not None)
        torch.cuda.nvtx.range_pop()
    launches = K.ckks_launch_count() - launches0
    ms = replicas.max_over_ranks(ms)
    ops = 2 * BATCH * args.steps * world
    value = replicas.job_throughput(2 * BATCH * args.steps, ms, world)

    # one lane, in order: per-kernel CUDA-event times on the launching stream
    seq_steps = max(3, args.steps // 4)
    K.ckks_profile(ctx, True)
    torch.cuda.nvtx.range_push("one_lane")   # profilers can scope to this phase
    ms_seq = timed(seq_steps, 1)
    torch.cuda.nvtx.range_pop()
    K.ckks_profile(ctx, False)
    prof = K.ckks_profile_read(ctx)
    seq_ops_per_s = 2 * BATCH * seq_steps / (ms_seq / 1e3)
    ks_stages = ("ks_in_rows", "modup_cols", "modup_rows", "keymult", "moddown_in_rows", "moddown_cols")
    per_launch = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in prof.items()}
    # stages both operations run are averaged over both in the profile
    hmult_us = 1e3 * sum(per_launch[k] for k in ks_stages[:5] + ("rescale_cols", "rescale_rows"))
    hrot_us = 1e3 * sum(per_launch[k] for k in ks_stages + ("moddown_rows",))

    e2e = e2e_leg(K, ctx, lanes, streams, stream, cts, rk, gk, args.lanes, args.e2e_slots, args.steps,
                  args.e2e_priority, barrier, world)

    # batched and served forms next to the headline (same context and keys;
    # levels other than the top one use the default column shapes)
    bat = batched_modes(K, ctx, sk, rk, gk, max(3, args.steps // 4), max(3, args.warmup), stream)
    srv_runs, srv_cap, srv_res = serve_runs(K, ctx, sk, rk, stream, args.requests_default, (0.8,))
    served = {"frac_of_capacity": 0.8, "capacity_ops_s": srv_cap, "resident_key_bytes": srv_res,
              "requests": args.requests_default,
              "continuous_batching_4_lanes": srv_runs["continuous_batching_4_lanes@0.8"],
              "one_op_per_launch": srv_runs["one_op_per_launch@0.8"],
              "note": "Poisson arrivals of HMult+rescale / HRot at 0.8 x the one-stream capacity, levels U{1..39}, "
                      "64 resident rotation keys; the library's native serving loop (ckks_serve_run); latency = "
                      "completion - arrival on the host's steady clock"}
    fusion = dict(fusion_ablation(K, ctx, sk, rk, gk, stream, pdl=args.pdl == "on"),
                  note="one stream, median of 15 single operations (inputs rotated over 8 fresh encryptions), "
                       "fused pipeline vs the one-step-per-launch unfused form with every intermediate in HBM")
    tc_bconv = None
    if batch is not None and args.issue == "graph":
        tc_bconv = tensor_core_leg(K, ctx, batch_ops, args.lanes, stream, max(5, args.steps // 2),
                                   max(3, args.warmup), value)
    batched = dict(bat, note="64 independent operations, levels U{1..39}, HMult+rescale / HRot / PMult / "
                             "rescale; persistent = stage-major batch with one persistent KeyMult / element-wise "
                             "kernel, replayed as a CUDA graph")

    # roofline of the dominant kernel
    peaks, peak_kind = measured_peaks()
    models = kernel_models()
    dom = max(prof, key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    avg_s = dom_ms / 1e3 / max(dom_n, 1)
    mdl = models[dom]
    hm_bytes, hr_bytes = algorithmic_bytes()
    # both resources of the dominant kernel: HBM (compulsory bytes) and the
    # integer multiply pipes; the bound reported is the one with the larger
    # fraction
    hbm_ach = mdl["bytes"] / avg_s / 1e9
    hbm = {"bound": "hbm", "kernel": dom, "achieved": hbm_ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
           "frac": hbm_ach / peaks["hbm_gbs"], "peak_source": f"{peak_kind} hbm_gbs",
           "algorithmic_bytes_per_launch": mdl["bytes"], "traffic": ncu_traffic(dom)}
    # integer-ALU peak of the dominant kernel: its own mix of modular products
    # issued back to back at this GPU's measured multiply issue rates (every
    # SM at the maximum SM clock)
    clk_hz = peaks.get("sm_max_mhz", 2070.0) * 1e6
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    rates = {}
    for op, name in ((K.CKKS_INTOP_MAD_LO, "mad_lo"), (K.CKKS_INTOP_MAD_HI, "mad_hi"),
                     (K.CKKS_INTOP_MAD_WIDE, "mad_wide")):
        n_ops, ms_op = K.ckks_bench_intop(ctx, op, 4096)
        rates[name] = n_ops / (ms_op * 1e-3) / (sms * clk_hz)
    cost = multiply_costs(rates)
    sm_clocks = sum(mdl.get(k, 0) * cost[k] for k in cost)
    alu_peak = mdl["modmul"] / (sm_clocks / (sms * clk_hz)) / 1e12
    alu_ach = mdl["modmul"] / avg_s / 1e12
    alu = {"bound": "alu", "kernel": dom, "achieved": alu_ach, "peak": alu_peak, "unit": "Tmodmul/s",
           "frac": alu_ach / alu_peak,
           "peak_source": f"derived: {sms} SM x sm_max_mhz / (the kernel's products x SM clocks per product at "
                          "the measured mad.lo / mad.hi / mad.wide issue rates)",
           "int_multiply_per_sm_clk": rates, "algorithmic_modmul_per_launch": mdl["modmul"],
           "mix": {k: mdl.get(k, 0) for k in ("shoup", "mac", "smr")}, "traffic": ncu_traffic(dom)}
    roof, other = (alu, hbm) if alu["frac"] >= hbm["frac"] else (hbm, alu)
    roof = dict(roof, other={k: other[k] for k in ("bound", "achieved", "peak", "unit", "frac")})
    stage = {k: {"ms_per_launch": (v[0] / v[1] if v[1] else None), "launches": v[1],
                 "share": v[0] / max(sum(x[0] for x in prof.values()), 1e-9)} for k, v in prof.items()}
    per_gpu_gbs = BATCH * (hm_bytes + hr_bytes) * args.steps / (ms / 1e3) / 1e9
    op_hbm = {"hmult_bytes": hm_bytes, "hrot_bytes": hr_bytes, "achieved_gbs_per_gpu": per_gpu_gbs,
              "frac_of_hbm": per_gpu_gbs / peaks["hbm_gbs"], "peak_source": f"{peak_kind} hbm_gbs",
              "frac_of_nominal_7900_gbs": per_gpu_gbs / 7900.0}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic (fresh encryptions of U[-1,1] messages)",
        "config": workload_config({"parallelism": f"replicas{world}",
                                   "lanes": f"{args.lanes} concurrent CUDA streams (context clones), "
                                            "independent ciphertexts per lane",
                                   "issue": {"graph": "ckks_batch_run: the step's operations replayed as one "
                                                      "CUDA graph",
                                             "direct": "ckks_batch_run: the library issues the step's "
                                                       "operations across the lanes",
                                             "python": "one binding call per operation"}[args.issue],
                                   "programmatic_dependent_launch": args.pdl,
                                   "column_shapes": ({k: list(v) for k, v in tuned[LEVEL].items()} if tuned
                                                     else "default rule"),
                                   "tune_file": tune_file_summary()}),
        "one_lane": {"value": seq_ops_per_s, "unit": UNIT, "hmult_rescale_us": hmult_us, "hrot_us": hrot_us,
                     "note": "same workload issued in order on one stream; stage times from its CUDA events"},
        "roofline": roof, "op_roofline": op_hbm, "stages": stage,
        "e2e": e2e, "gpu_launches": int(launches), "clocks": clk.summary(),
        "batched": batched, "serve": served, "fusion": fusion, "tensor_core_bconv": tc_bconv,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    if rank == 0:
        print(json.dumps(line), flush=True)
    if batch is not None:
        K.ckks_batch_destroy(batch)
    for h in cts + outs_m + outs_r + outs_b + [sk, rk, gk]:
        K.ckks_free(h)
    for c in lanes[1:]:
        K.ckks_ctx_destroy(c)
    K.ckks_ctx_destroy(ctx)


# ----------------------------------------------------------------------------
# batched form: independent operations at mixed levels (one op per launch vs
# lanes vs lanes captured into one CUDA graph)
# ----------------------------------------------------------------------------

def e2e_leg(K, ctx, lanes, streams, stream, cts, rk, gk, n_lanes, slots, steps, priority, barrier, world):
    """End-to-end throughput (key-switch ops/s) through the C ABI with host
    buffers: inputs uploaded from and results read back to pinned host memory
    inside the timed region, on n_lanes compute lanes (lanes / streams) with
    `slots` output slots per lane; `priority` ("high" or "normal") is the
    priority of the transfer streams."""
    import torch
    from paper_2407_13055_gb300 import replicas
    # end to end through the C ABI with host buffers. A step is e2e_pairs pairs
    # over e2e_pairs + 1 input ciphertexts (pair i: HMult(ct_i, ct_i+1) + rescale,
    # HRot(ct_i), as in the device-resident step); each input is copied once from
    # pinned host memory into a ring of device buffers, and both results of every
    # pair are read back to pinned host memory. Uploads (on transfer-only clone
    # contexts), the pairs (on the lanes) and the exports (on a second set of
    # transfer-only clones) form a pipeline ordered by CUDA events, so copies
    # overlap the computation: an upload waits for the two pairs that read its
    # buffer's previous ciphertext, a pair for its two uploads and for the export
    # of its output slot's previous results.
    n = 1 << LOG_N
    nl = n_lanes
    NS = slots
    R = NS * nl + 2                       # device input buffers (ring)
    pinned = lambda shape: torch.empty(shape, dtype=torch.int32, pin_memory=True).numpy().view(np.uint32)
    host_in = [pinned((2, L, n)) for _ in range(E2E_HOST)]
    for i in range(E2E_HOST):
        K.ckks_ct_export(ctx, cts[i], n, out=host_in[i])
    # transfer streams: with high priority their layout permutations are
    # scheduled ahead of the compute lanes' pending blocks, so the copies
    # behind them start as soon as their data is ready
    prio = -1 if priority == "high" else 0
    up_s = [torch.cuda.Stream(priority=prio) for _ in range(nl)]
    dn_s = [torch.cuda.Stream(priority=prio) for _ in range(nl)]
    up_c = [K.ckks_ctx_clone(ctx, x.cuda_stream) for x in up_s]
    dn_c = [K.ckks_ctx_clone(ctx, x.cuda_stream) for x in dn_s]
    dev_in = [K.ckks_ct_create(ctx, LEVEL) for _ in range(R)]
    slot = lambda: [[K.ckks_ct_create(ctx, LEVEL) for _ in range(NS)] for _ in range(nl)]
    dev_m, dev_r = slot(), slot()
    host_m = [[pinned((2, L - 1, n)) for _ in range(NS)] for _ in range(nl)]
    host_r = [[pinned((2, L, n)) for _ in range(NS)] for _ in range(nl)]
    ev = lambda: [[torch.cuda.Event() for _ in range(NS)] for _ in range(nl)]
    ev_comp, ev_dn = ev(), ev()
    ev_in = [torch.cuda.Event() for _ in range(R)]        # upload into the buffer done
    ev_use = [[torch.cuda.Event() for _ in range(R)] for _ in range(2)]   # read as a / as b done
    for l in range(nl):
        for k in range(NS):
            ev_dn[l][k].record(stream)
    for b in range(R):
        ev_use[0][b].record(stream)
        ev_use[1][b].record(stream)
    e2e_pairs = 4 * E2E_HOST
    uploads = [0]                          # next upload's global index

    def upload():
        u = uploads[0]
        uploads[0] += 1
        b, l = u % R, u % nl
        up_s[l].wait_event(ev_use[0][b])
        up_s[l].wait_event(ev_use[1][b])
        K.ckks_ct_upload_async(up_c[l], dev_in[b], host_in[u % E2E_HOST], LEVEL, SCALE)
        ev_in[b].record(up_s[l])
        return b

    def e2e_step():
        nxt = upload()
        for i in range(e2e_pairs):
            l, k = i % nl, (i // nl) % NS
            ba, bb = nxt, upload()
            nxt = bb
            streams[l].wait_event(ev_in[ba])
            streams[l].wait_event(ev_in[bb])
            streams[l].wait_event(ev_dn[l][k])
            K.ckks_hmult(lanes[l], dev_in[ba], dev_in[bb], rk, K.CKKS_RESCALE, dev_m[l][k])
            K.ckks_hrot(lanes[l], dev_in[ba], 1, gk, dev_r[l][k])
            ev_use[0][ba].record(streams[l])
            ev_use[1][bb].record(streams[l])
            ev_comp[l][k].record(streams[l])
            dn_s[l].wait_event(ev_comp[l][k])
            K.ckks_ct_export_async(dn_c[l], dev_m[l][k], host_m[l][k])
            K.ckks_ct_export_async(dn_c[l], dev_r[l][k], host_r[l][k])
            ev_dn[l][k].record(dn_s[l])

    e2e_step()
    barrier()
    e2e_steps = max(10, steps // 2)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    barrier()
    e2e_dt = replicas.max_over_ranks(time.perf_counter() - t0)
    ct_bytes = 2 * L * n * 4
    e2e = {"value": replicas.job_throughput(2 * e2e_pairs * e2e_steps, 1e3 * e2e_dt, world), "unit": UNIT,
           "h2d_bytes_per_step": (e2e_pairs + 1) * ct_bytes,
           "d2h_bytes_per_step": e2e_pairs * (ct_bytes * (L - 1) // L + ct_bytes),
           "ops_per_step": 2 * e2e_pairs,
           "note": f"{nl} lanes x {NS} output slots, {R} input buffers; each step's {e2e_pairs + 1} input "
                   "ciphertexts uploaded once from pinned host memory, both results of every pair read back to "
                   "pinned host memory; upload / compute / export pipelined on separate streams, wall clock"}
    for h in dev_in:
        K.ckks_free(h)
    for grp in (dev_m, dev_r):
        for row in grp:
            for h in row:
                K.ckks_free(h)
    for c in up_c + dn_c:
        K.ckks_ctx_destroy(c)

    return e2e


def tensor_core_leg(K, ctx, ops, n_lanes, stream, steps, warmup, cuda_core_ops_s, shape=(4, 8, 1, 16)):
    """The headline's operations (one CUDA graph per step over n_lanes lanes)
    with the BConv of every column kernel on the tensor cores (tcgen05, exact
    fp16 byte planes; launch shape tc, sl, z, targets per chunk) instead of
    CUDA cores, on the same context and inputs; the tuned shapes are put back
    afterwards. Returns ops/s beside the CUDA-core figure and the operations'
    HBM fraction."""
    import torch
    kernels = (K.CKKS_COL_MODUP, K.CKKS_COL_MODDOWN, K.CKKS_COL_RS_FUSED)
    saved = {k: K.ckks_tune_get(ctx, k, LEVEL) for k in kernels}
    try:
        for k in kernels:
            K.ckks_tune_set(ctx, k, LEVEL, *shape)
        b = K.ckks_batch_create(ctx, ops, n_lanes, True)
        try:
            for _ in range(warmup):
                K.ckks_batch_run(ctx, b)
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            for _ in range(steps):
                K.ckks_batch_run(ctx, b)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
        finally:
            K.ckks_batch_destroy(b)
    finally:
        for k, v in saved.items():   # tc = 0 clears an untuned entry
            K.ckks_tune_set(ctx, k, LEVEL, *v[:4])
    ops_s = len(ops) * steps / (ms / 1e3)
    mean_bytes = (algorithmic_bytes()[0] + algorithmic_bytes()[1]) / 2
    peaks, kind = measured_peaks()
    return {"ops_s": ops_s, "cuda_core_ops_s": cuda_core_ops_s, "col_shape": list(shape),
            "op_frac_of_hbm": ops_s * mean_bytes / 1e9 / peaks["hbm_gbs"],
            "cuda_core_op_frac_of_hbm": cuda_core_ops_s * mean_bytes / 1e9 / peaks["hbm_gbs"],
            "note": f"{steps} graph replays of the same {len(ops)} operations, every column kernel's BConv on "
                    f"the tensor cores (shape {shape}), against the headline's tuned CUDA-core shapes; "
                    f"HBM fraction of {kind} hbm_gbs"}


def fusion_ablation(K, ctx, sk, rk, gk, stream, levels=(L - 1, 20, 1), reps=15, pdl=True):
    """Fused pipeline vs the unfused one-step-per-launch form
    (CKKS_LAUNCH_UNFUSED) on one stream: median microseconds of HMult +
    rescale and of HRot(1) at each level (fresh encryptions, inputs rotated
    over 8 ciphertexts), with the launches per operation."""
    import torch
    from paper_2407_13055_gb300 import inputs
    base = K.CKKS_LAUNCH_PDL if pdl else 0
    out = {}
    for lv in levels:
        cts = [K.ckks_encrypt(ctx, sk, K.ckks_encode(ctx, inputs.messages(4000 + 10 * lv + i, (1 << LOG_N) // 2),
                                                      lv, SCALE), 5000 + 10 * lv + i) for i in range(8)]
        res = K.ckks_ct_create(ctx, lv)
        row = {}
        for form, flags in (("fused", base), ("unfused", base | K.CKKS_LAUNCH_UNFUSED)):
            K.ckks_set_launch_flags(ctx, flags)
            for op in ("hmult_rescale", "hrot"):
                run = ((lambda i: K.ckks_hmult(ctx, cts[i % 8], cts[(i + 1) % 8], rk, K.CKKS_RESCALE, res))
                       if op == "hmult_rescale" else (lambda i: K.ckks_hrot(ctx, cts[i % 8], 1, gk, res)))
                for i in range(3):
                    run(i)
                torch.cuda.synchronize()
                times = []
                l0 = K.ckks_launch_count()
                for i in range(reps):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    run(i)
                    e1.record(stream)
                    e1.synchronize()
                    times.append(1e3 * e0.elapsed_time(e1))
                row.setdefault(op, {})[form] = {"us": statistics.median(times),
                                                "launches": (K.ckks_launch_count() - l0) / reps}
        for op in row:
            row[op]["unfused_over_fused"] = row[op]["unfused"]["us"] / row[op]["fused"]["us"]
        out[f"level_{lv}"] = row
        K.ckks_set_launch_flags(ctx, base)
        for h in cts + [res]:
            K.ckks_free(h)
    K.ckks_set_launch_flags(ctx, base)
    return out


BATCHED_MODES = (("one_op_per_launch", 1, 0), ("lanes4_graph", 4, 1), ("lanes4_persistent_graph", 4, 3))


def batched_modes(K, ctx, sk, rk, gk, steps, warmup, stream, modes=BATCHED_MODES, count=64, seed=7):
    """The batched workload: `count` independent operations on fresh
    encryptions at levels U{1..39}, kinds uniform over HMult+rescale / HRot /
    PMult / rescale, timed as one list per step in each mode (lanes, batch
    mode flags: 1 = one CUDA graph, 2 = stage-major with the persistent
    KeyMult / element-wise kernel). Returns {mode: ops/s, ms/batch, kernel
    launches per batch}."""
    import torch
    from paper_2407_13055_gb300 import inputs
    levels = inputs.level_list(seed, count, L - 1)
    kinds = ["hmult", "hrot", "pmult", "rescale"]
    kind_ix = np.random.default_rng(seed + 1).integers(0, 4, count)
    handles, ops = [], []
    for i in range(count):
        lv, kind = int(levels[i]), kinds[int(kind_ix[i])]
        enc = lambda sd: K.ckks_encrypt(ctx, sk, K.ckks_encode(ctx, inputs.messages(sd, (1 << LOG_N) // 2), lv,
                                                                 SCALE), sd)
        a = enc(1000 + i)
        out = K.ckks_ct_create(ctx, lv)
        handles += [a, out]
        if kind == "hmult":
            b = enc(2000 + i)
            handles.append(b)
            ops.append(dict(op=K.CKKS_OP_HMULT, a=a, b=b, evk=rk, flags=K.CKKS_RESCALE, out=out))
        elif kind == "hrot":
            ops.append(dict(op=K.CKKS_OP_HROT, a=a, r=1, evk=gk, out=out))
        elif kind == "pmult":
            pt = K.ckks_encode(ctx, inputs.messages(3000 + i, (1 << LOG_N) // 2), lv, SCALE)
            handles.append(pt)
            ops.append(dict(op=K.CKKS_OP_PMULT, a=a, pt=pt, out=out))
        else:
            ops.append(dict(op=K.CKKS_OP_RESCALE, a=a, out=out))
    results = {}
    for name, lanes, flags in modes:
        batch = K.ckks_batch_create(ctx, ops, lanes, flags)
        for _ in range(warmup):
            K.ckks_batch_run(ctx, batch)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = K.ckks_launch_count()
        e0.record(stream)
        for _ in range(steps):
            K.ckks_batch_run(ctx, batch)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        results[name] = {"ops_s": count * steps / (ms / 1e3), "ms_per_batch": ms / steps,
                         "kernel_launches_per_batch": (K.ckks_launch_count() - l0) / steps}
        K.ckks_batch_destroy(batch)
    K.ckks_sync(ctx)
    for h in handles:
        K.ckks_free(h)
    return results


def run_batched(args, local_rank):
    import torch
    from paper_2407_13055_gb300 import ckks as K
    from paper_2407_13055_gb300 import inputs
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    q, p = K.ckks_gen_primes(LOG_N, L, ALPHA)
    ctx = K.ckks_ctx_create(LOG_N, q, p, DNUM, scale=SCALE, secret_hw=HW, stream=stream.cuda_stream)
    K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL if args.pdl == "on" else 0)
    sk = K.ckks_keygen_secret(ctx, 11)
    rk = K.ckks_keygen_relin(ctx, sk, 12)
    gk = K.ckks_keygen_rot(ctx, sk, 1, 13)
    tuned = tune_levels(K, ctx, inputs.level_list(7, 64, L - 1), not args.no_tune, reps=2,
                        pkey=tune_cache.params_key(LOG_N, q, p, DNUM))
    modes = BATCHED_MODES + (("lanes4_direct", 4, 0), ("lanes4_persistent_direct", 4, 2))
    results = batched_modes(K, ctx, sk, rk, gk, args.steps, args.warmup, stream, modes)
    line = {"metric": "batched mixed-level ops/sec at N=2^16 (1 GB300)", "value": results["lanes4_graph"]["ops_s"],
            "unit": "ops/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": results["lanes4_graph"]["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic (fresh encryptions)",
            "config": {"workload": "64 ciphertexts, levels U{1..39}, ops uniform over HMult+rescale / HRot / PMult / "
                                   "rescale, independent", "N": 1 << LOG_N, "limbs_top": L, "dnum": DNUM,
                       "column_shapes": "tuned per level" if tuned else "default rule"},
            "modes": results}
    print(json.dumps(line), flush=True)
    for h in (sk, rk, gk):
        K.ckks_free(h)
    K.ckks_ctx_destroy(ctx)


# ----------------------------------------------------------------------------
# single-op latency table: dnum in {1, 3, 5} x top / middle / bottom level
# ----------------------------------------------------------------------------

def run_latency(args, local_rank):
    import torch
    from paper_2407_13055_gb300 import ckks as K
    from paper_2407_13055_gb300 import inputs
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    peaks, peak_kind = measured_peaks()
    reps = max(50, args.steps)
    flush = torch.empty(2 * 129 * (1 << 20) // 4 * 2, dtype=torch.int32, device="cuda")  # 2 x L2
    rows = []
    r_rand = 12345
    for dnum in (1, 3, 5):
        alpha = -(-L // dnum)
        q, p = K.ckks_gen_primes(LOG_N, L, alpha)
        ctx = K.ckks_ctx_create(LOG_N, q, p, dnum, scale=SCALE, secret_hw=HW, stream=stream.cuda_stream)
        K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL if args.pdl == "on" else 0)
        sk = K.ckks_keygen_secret(ctx, 61)
        rk = K.ckks_keygen_relin(ctx, sk, 62)
        gks = {r: K.ckks_keygen_rot(ctx, sk, r, 63 + r % 1000) for r in (1, 5, r_rand)}
        for level in (L - 1, 20, 1):
            tune_levels(K, ctx, [level], not args.no_tune, 3, tune_cache.params_key(LOG_N, q, p, dnum))
            a = K.ckks_encrypt(ctx, sk, K.ckks_encode(ctx, inputs.messages(64, (1 << LOG_N) // 2), level, SCALE), 65)
            b = K.ckks_encrypt(ctx, sk, K.ckks_encode(ctx, inputs.messages(66, (1 << LOG_N) // 2), level, SCALE), 67)
            out = K.ckks_ct_create(ctx, level)
            ops = {"hmult_rescale": lambda: K.ckks_hmult(ctx, a, b, rk, K.CKKS_RESCALE, out),
                   "hmult": lambda: K.ckks_hmult(ctx, a, b, rk, 0, out)}
            for r in (1, 5, r_rand):
                ops[f"hrot_{r}"] = (lambda r=r: K.ckks_hrot(ctx, a, r, gks[r], out))
            n = level + 1
            hm_b, hr_b = algorithmic_bytes(n, alpha)
            for name, fn in ops.items():
                res = {}
                for mode in ("cold", "warm"):
                    ts = []
                    for _ in range(3):
                        fn()
                    for _ in range(reps):
                        if mode == "cold":
                            flush.add_(1)          # writes 2 x L2 between repetitions
                        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        fn()
                        e1.record(stream)
                        e1.synchronize()
                        ts.append(e0.elapsed_time(e1) * 1e3)
                    res[mode] = float(np.median(ts))
                alg = hr_b if name.startswith("hrot") else (hm_b if name == "hmult_rescale" else
                                                              hm_b - 2 * (n - 1) * LIMB_BYTES + 2 * n * LIMB_BYTES)
                rows.append({"dnum": dnum, "alpha": alpha, "level": level, "op": name,
                             "median_us_cold_l2": res["cold"], "median_us_warm_l2": res["warm"],
                             "algorithmic_mb": alg / 1e6,
                             "hbm_frac_cold": alg / (res["cold"] * 1e-6) / 1e9 / peaks["hbm_gbs"]})
            for h in (a, b, out):
                K.ckks_free(h)
        for h in list(gks.values()) + [sk, rk]:
            K.ckks_free(h)
        K.ckks_ctx_destroy(ctx)
    top3 = [r for r in rows if r["dnum"] == 3 and r["level"] == L - 1 and r["op"] in ("hmult_rescale", "hrot_1")]
    value = 2 / sum(r["median_us_cold_l2"] * 1e-6 for r in top3)
    line = {"metric": "single-op key-switch latency at N=2^16 (1 GB300): median of >=50, cold and warm L2",
            "value": value, "unit": "key-switch ops/s (one at a time, cold L2, dnum=3 top level)", "n_gpus": 1,
            "steps": reps, "warmup": 3, "ms_per_step": 1e3 / value, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic (fresh encryptions)",
            "config": {"workload": "HMult (with and without rescale) and HRot (r = 1, 5, 12345) at levels 39 / 20 / 1 "
                                   "for dnum = 1, 3, 5; cold L2 = a 2 x L2 buffer written between repetitions",
                       "N": 1 << LOG_N, "limbs_top": L,
                       "column_shapes": "default rule" if args.no_tune else "tuned per level"},
            "table": rows, "hbm_peak": {"value": peaks["hbm_gbs"], "source": peak_kind}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# 25-30 prime system (Table 2): per-level latency with rational rescaling
# ----------------------------------------------------------------------------

def run_rns2530(args, local_rank):
    import math
    import torch
    from paper_2407_13055_gb300 import ckks as K
    from paper_2407_13055_gb300 import inputs
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    alpha = 5
    q, p, levels = K.ckks_gen_prime_system_2530(LOG_N, alpha)
    dnum = -(-len(q) // alpha)
    ctx = K.ckks_ctx_create(LOG_N, q, p, dnum, scale=2.0**40, secret_hw=HW, stream=stream.cuda_stream,
                            levels=levels)
    K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL if args.pdl == "on" else 0)
    sk = K.ckks_keygen_secret(ctx, 81)
    rk = K.ckks_keygen_relin(ctx, sk, 82)
    gk = K.ckks_keygen_rot(ctx, sk, 1, 83)
    reps = max(50, args.steps)
    rows = []

    def median_us(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        return float(np.median(ts))

    for lv in range(len(levels)):
        tune_levels(K, ctx, [lv], not args.no_tune, 3, tune_cache.params_key(LOG_N, q, p, dnum, levels))
        delta = 2.0 ** (55 if lv >= 5 else 40)
        a = K.ckks_encrypt(ctx, sk, K.ckks_encode(ctx, inputs.messages(84, (1 << LOG_N) // 2), lv, delta), 85)
        out = K.ckks_ct_create(ctx, lv)
        s0, n0 = levels[lv]
        row = {"level": lv, "taus": sum(1 for g in range(s0, s0 + n0) if g < 4),
               "qs": sum(1 for g in range(s0, s0 + n0) if g >= 4),
               "log2_Q": sum(math.log2(int(q[g])) for g in range(s0, s0 + n0)),
               "hrot_us": median_us(lambda: K.ckks_hrot(ctx, a, 1, gk, out)),
               "hmult_us": median_us(lambda: K.ckks_hmult(ctx, a, a, rk, 0, out))}
        if lv >= 1:
            row["hmult_rational_rescale_us"] = median_us(lambda: K.ckks_hmult(ctx, a, a, rk, K.CKKS_RESCALE, out))
            row["hmult_merged_rescale_us"] = median_us(
                lambda: K.ckks_hmult(ctx, a, a, rk, K.CKKS_RESCALE_MERGED, out))
            row["rational_rescale_us"] = median_us(lambda: K.ckks_rescale(ctx, a, out))
            K.ckks_hmult(ctx, a, a, rk, K.CKKS_RESCALE, out)
            row["log2_scale_after_hmult"] = math.log2(K.ckks_ct_info(out)[1])
        rows.append(row)
        K.ckks_free(a)
        K.ckks_free(out)
    top = rows[4]
    line = {"metric": "25-30 prime system (Table 2) at N=2^16 (1 GB300): HMult+rational rescale latency",
            "value": 1e6 / top["hmult_rational_rescale_us"], "unit": "HMult+rescale/s at level 4 (one at a time)",
            "n_gpus": 1, "steps": reps, "warmup": 3, "ms_per_step": top["hmult_rational_rescale_us"] / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (fresh encryptions)",
            "config": {"workload": "levels 0-8 of the 25-30 system (15 primes, alpha=5, dnum=3, one key for all "
                                   "levels); median of >=50, warm L2",
                       "N": 1 << LOG_N, "primes": [int(v) for v in q], "levels": levels},
            "table": rows}
    print(json.dumps(line), flush=True)
    for h in (sk, rk, gk):
        K.ckks_free(h)
    K.ckks_ctx_destroy(ctx)


# ----------------------------------------------------------------------------
# ablation: Table 3 on this GPU, and sequential fusion of ModDown + rescale
# ----------------------------------------------------------------------------

def run_ablation(args, local_rank):
    import torch
    from paper_2407_13055_gb300 import ckks as K
    from paper_2407_13055_gb300 import inputs
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    q, p = K.ckks_gen_primes(LOG_N, L, ALPHA)
    ctx = K.ckks_ctx_create(LOG_N, q, p, DNUM, scale=SCALE, secret_hw=HW, stream=stream.cuda_stream)
    K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL if args.pdl == "on" else 0)
    peaks, _ = measured_peaks()
    sms = torch.cuda.get_device_properties(local_rank).multi_processor_count
    # (1) modular multiplication methods: 8 chains per thread, enough threads
    # for many waves; every method must return the same values
    n, rounds = sms * 2048 * 8, 2048
    rng = np.random.default_rng(1)
    mm = {}
    for pid, label in ((1, "30-bit q_1"), (0, "31-bit q_0")):
        qq = int(q[pid])
        a = rng.integers(0, qq, n, dtype=np.int64).astype(np.uint32)
        b = int(rng.integers(1, qq))
        ref = None
        for m, name in ((K.CKKS_MODMUL_BARRETT, "barrett64"), (K.CKKS_MODMUL_MONTGOMERY, "montgomery"),
                        (K.CKKS_MODMUL_SHOUP, "shoup"), (K.CKKS_MODMUL_SMR, "signed_montgomery")):
            out, ms = K.ckks_bench_modmul(ctx, m, pid, b, a, rounds)
            ref = out if ref is None else ref
            gmm = n * rounds / (ms * 1e-3) / 1e9
            mm.setdefault(label, {})[name] = {"gmodmul_s": gmm, "ms": ms, "agrees": bool(np.array_equal(out, ref)),
                                              "modmul_per_sm_clk": gmm * 1e9 / (sms * peaks.get("sm_max_mhz", 2070.0)
                                                                                * 1e6)}
    # integer multiply issue rates per SM per clock (the unit counts behind
    # the integer-ALU roofline)
    clk_hz = peaks.get("sm_max_mhz", 2070.0) * 1e6
    int_rates = {}
    for op, name in ((K.CKKS_INTOP_MAD_LO, "mad_lo"), (K.CKKS_INTOP_MAD_HI, "mad_hi"),
                     (K.CKKS_INTOP_MAD_WIDE, "mad_wide")):
        n_ops, ms_op = K.ckks_bench_intop(ctx, op, 4096)
        int_rates[name] = n_ops / (ms_op * 1e-3) / (sms * clk_hz)
    # (2) sequential fusion: HMult with ModDown + rescale fused vs HMult then
    # a separate rescale (top level, one stream, median of 50)
    sk = K.ckks_keygen_secret(ctx, 71)
    rk = K.ckks_keygen_relin(ctx, sk, 72)
    tune_levels(K, ctx, [LEVEL], not args.no_tune, 3, pkey=tune_cache.params_key(LOG_N, q, p, DNUM))
    a = K.ckks_encrypt(ctx, sk, K.ckks_encode(ctx, inputs.messages(73, (1 << LOG_N) // 2), LEVEL, SCALE), 74)
    b = K.ckks_encrypt(ctx, sk, K.ckks_encode(ctx, inputs.messages(75, (1 << LOG_N) // 2), LEVEL, SCALE), 76)
    mid, out = K.ckks_ct_create(ctx, LEVEL), K.ckks_ct_create(ctx, LEVEL)
    forms = {"fused_moddown_rescale": lambda: K.ckks_hmult(ctx, a, b, rk, K.CKKS_RESCALE, out),
             "merged_moddown_rescale": lambda: K.ckks_hmult(ctx, a, b, rk, K.CKKS_RESCALE_MERGED, out),
             "hmult_then_rescale": lambda: (K.ckks_hmult(ctx, a, b, rk, 0, mid), K.ckks_rescale(ctx, mid, out))}
    seq = {}
    for name, fn in forms.items():
        ts = []
        for _ in range(3):
            fn()
        for _ in range(max(50, args.steps)):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        seq[name] = float(np.median(ts))
    # precision of the exact fused form and of the merged one (Sec. 6): both
    # decrypt to u v; max slot error
    u, v = inputs.messages(73, (1 << LOG_N) // 2), inputs.messages(75, (1 << LOG_N) // 2)
    dec_err = {}
    for name, fl in (("fused_moddown_rescale", K.CKKS_RESCALE), ("merged_moddown_rescale", K.CKKS_RESCALE_MERGED)):
        K.ckks_hmult(ctx, a, b, rk, fl, out)
        pt = K.ckks_decrypt(ctx, sk, out)
        dec_err[name] = float(np.max(np.abs(K.ckks_decode(ctx, pt, u.size) - u * v)))
        K.ckks_free(pt)
    best = max(v["gmodmul_s"] for v in mm["30-bit q_1"].values())
    line = {"metric": "ablation on 1 GB300: modular multiplication methods (Table 3) and ModDown+rescale fusion",
            "value": best, "unit": "Gmodmul/s (best method, 30-bit prime)", "n_gpus": 1, "steps": 1,
            "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic",
            "config": {"workload": f"{n} elements x {rounds} dependent modular products, 8 chains per thread; "
                                   "HMult+relin at level 39 (dnum=3) with fused, merged or separate rescale"},
            "modmul": mm, "int_multiply_per_sm_clk": int_rates, "seq_fusion_us": seq,
            "seq_fusion_speedup": seq["hmult_then_rescale"] / seq["fused_moddown_rescale"],
            "merged_speedup_over_fused": seq["fused_moddown_rescale"] / seq["merged_moddown_rescale"],
            "decrypt_max_err": dec_err}
    print(json.dumps(line), flush=True)
    for h in (a, b, mid, out, sk, rk):
        K.ckks_free(h)
    K.ckks_ctx_destroy(ctx)


# ----------------------------------------------------------------------------
# hoisted rotations: one ModUp shared by many rotations of one ciphertext
# ----------------------------------------------------------------------------

def run_hoisted(args, local_rank):
    import torch
    from paper_2407_13055_gb300 import ckks as K
    from paper_2407_13055_gb300 import inputs
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    q, p = K.ckks_gen_primes(LOG_N, L, ALPHA)
    ctx = K.ckks_ctx_create(LOG_N, q, p, DNUM, scale=SCALE, secret_hw=HW, stream=stream.cuda_stream)
    K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL if args.pdl == "on" else 0)
    sk = K.ckks_keygen_secret(ctx, 41)
    rots = list(range(1, 33))
    gks = [K.ckks_keygen_rot(ctx, sk, r, 500 + r) for r in rots]
    cts = [K.ckks_encrypt(ctx, sk, K.ckks_encode(ctx, inputs.messages(600 + i, (1 << LOG_N) // 2), LEVEL, SCALE),
                          700 + i) for i in range(4)]
    outs = [K.ckks_ct_create(ctx, LEVEL) for _ in rots]
    tuned = tune_levels(K, ctx, [LEVEL], not args.no_tune, pkey=tune_cache.params_key(LOG_N, q, p, DNUM))
    # linear transform sum_{r=0..32} d_r (.) HRot(ct, r): extended diagonals
    lt_rots = [0] + rots
    lt_keys = [None] + gks
    diags = [K.ckks_encode_ext(ctx, inputs.messages(800 + i, (1 << LOG_N) // 2), LEVEL, SCALE)
             for i in range(len(lt_rots))]
    acc = K.ckks_ct_create(ctx, LEVEL)
    tmp = K.ckks_ct_create(ctx, LEVEL)

    def hoisted(c):
        K.ckks_hrot_hoisted(ctx, c, rots, gks, outs)

    def separate(c):
        for r, g, o in zip(rots, gks, outs):
            K.ckks_hrot(ctx, c, r, g, o)

    def lt_fused(c):
        K.ckks_linear_transform(ctx, c, lt_rots, lt_keys, diags, acc)

    def lt_composed(c):
        # the same sum from hoisted rotations, PMult and HAdd (one ModDown per rotation)
        K.ckks_hrot_hoisted(ctx, c, rots, gks, outs)
        K.ckks_pmult(ctx, c, diags[0], acc)
        for o, d in zip(outs, diags[1:]):
            K.ckks_pmult(ctx, o, d, tmp)
            K.ckks_hadd(ctx, acc, tmp, acc)

    res = {}
    for name, fn in (("separate_hrot", separate), ("hoisted", hoisted), ("lt_composed", lt_composed),
                     ("lt_fused", lt_fused)):
        for _ in range(args.warmup):
            fn(cts[0])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = K.ckks_launch_count()
        e0.record(stream)
        for i in range(args.steps):
            fn(cts[i % len(cts)])
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[name] = {"rotations_s": len(rots) * args.steps / (ms / 1e3), "us_per_rotation": 1e3 * ms / args.steps /
                     len(rots), "launches_per_step": (K.ckks_launch_count() - l0) / args.steps}
    line = {"metric": "hoisted HRot throughput at N=2^16 (1 GB300): 32 rotations of one ciphertext",
            "value": res["hoisted"]["rotations_s"], "unit": "rotations/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": len(rots) * res["hoisted"]["us_per_rotation"] / 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic (fresh encryptions)",
            "config": {"workload": "32 rotations (r = 1..32) of one top-level ciphertext per step, one shared ModUp",
                       "N": 1 << LOG_N, "limbs": L, "dnum": DNUM,
                       "column_shapes": "tuned" if tuned else "default rule"},
            "modes": res, "speedup_vs_separate": res["hoisted"]["rotations_s"] / res["separate_hrot"]["rotations_s"],
            "linear_transform": {"terms": len(lt_rots), "fused_ms": 32e-3 * res["lt_fused"]["us_per_rotation"],
                                 "composed_ms": 32e-3 * res["lt_composed"]["us_per_rotation"],
                                 "speedup": res["lt_fused"]["rotations_s"] / res["lt_composed"]["rotations_s"]}}
    print(json.dumps(line), flush=True)
    for h in outs + cts + gks + diags + [sk, acc, tmp]:
        K.ckks_free(h)
    K.ckks_ctx_destroy(ctx)


# ----------------------------------------------------------------------------
# bootstrap-shaped trace: linear transforms, polynomial, linear transforms
# ----------------------------------------------------------------------------

def run_bootstrap(args, local_rank):
    import torch
    from paper_2407_13055_gb300 import ckks as K
    from paper_2407_13055_gb300 import inputs
    from paper_2407_13055_gb300.trace import Trace, TraceSpec, expected
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    q, p = K.ckks_gen_primes(LOG_N, L, ALPHA)
    ctx = K.ckks_ctx_create(LOG_N, q, p, DNUM, scale=SCALE, secret_hw=HW, stream=stream.cuda_stream)
    K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL if args.pdl == "on" else 0)
    sk = K.ckks_keygen_secret(ctx, 51)
    spec = TraceSpec()
    slots = (1 << LOG_N) // 2
    u = inputs.messages(52, slots)
    pt = K.ckks_encode(ctx, u, LEVEL, SCALE)
    ct = K.ckks_encrypt(ctx, sk, pt, 53)
    tuned = tune_levels(K, ctx, range(LEVEL - spec.levels_used(), LEVEL + 1), not args.no_tune, reps=2,
                         pkey=tune_cache.params_key(LOG_N, q, p, DNUM))
    tr = Trace(K, ctx, spec, LEVEL, q, slots, sk=sk)
    want = expected(spec, u)
    res = {}
    for name, fused in (("one_op_at_a_time", False), ("fused", True)):
        out, level = tr.run(ct, fused)           # first run: plaintexts, pooled ciphertexts
        dec = K.ckks_decrypt(ctx, sk, out)
        err = float(np.max(np.abs(K.ckks_decode(ctx, dec, slots) - want)))
        K.ckks_free(dec)
        for _ in range(args.warmup):
            tr.run(ct, fused)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        l0 = K.ckks_launch_count()
        e0.record(stream)
        for _ in range(args.steps):
            tr.run(ct, fused)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[name] = {"ms_per_trace": ms, "traces_s": 1e3 / ms, "max_abs_error": err, "final_level": level,
                     "launches_per_trace": (K.ckks_launch_count() - l0) / args.steps}
    tr.close()
    line = {"metric": "bootstrap-shaped trace at N=2^16 (1 GB300)", "value": res["fused"]["traces_s"],
            "unit": "traces/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": res["fused"]["ms_per_trace"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic (fresh encryption of U[-1,1] slots)",
            "config": {"workload": f"CoeffToSlot-like {spec.lt_levels} BSGS linear transforms ({spec.n1} baby x "
                                   f"{spec.n2} giant steps, random diagonals), degree-{1 << spec.depth} polynomial "
                                   f"(product tree of HMult+rescale, depth {spec.depth}), SlotToCoeff-like "
                                   f"{spec.lt_levels} transforms; start level {LEVEL}",
                       "N": 1 << LOG_N, "limbs": L, "dnum": DNUM,
                       "column_shapes": "tuned per level" if tuned else "default rule"},
            "modes": res, "speedup_vs_one_op": res["one_op_at_a_time"]["ms_per_trace"] / res["fused"]["ms_per_trace"]}
    print(json.dumps(line), flush=True)
    for h in (pt, ct, sk):
        K.ckks_free(h)
    K.ckks_ctx_destroy(ctx)


# ----------------------------------------------------------------------------
# served form: Poisson arrivals, continuous batching over lanes
# ----------------------------------------------------------------------------

def serve_runs(K, ctx, sk, rk, stream, count, fracs, n_keys=64, seed=21):
    """The served workload: `count` Poisson arrivals of single HMult+rescale /
    HRot requests (50:50, levels U{1..39}, rotations over `n_keys` resident
    keys) at each rate frac x the one-stream capacity, served one operation
    at a time and by continuous batching on 4 lanes (admission by request
    footprint next to the resident keys, in a budget of keys + 4 GB). Returns
    ({run: latency stats}, capacity ops/s, resident key bytes)."""
    import torch
    from paper_2407_13055_gb300 import inputs
    from paper_2407_13055_gb300.serve import Request, Server, latency_stats, poisson_arrivals
    rots = sorted(set(int(r) for r in inputs.rotation_list(seed + 2, 4 * n_keys, (1 << LOG_N) // 2)))[:n_keys]
    gks = {r: K.ckks_keygen_rot(ctx, sk, r, 100 + r) for r in rots}
    pool = {}
    for lv in range(1, L):
        pool[lv] = [K.ckks_encrypt(ctx, sk, K.ckks_encode(ctx, inputs.messages(500 + 2 * lv + t, (1 << LOG_N) // 2),
                                                           lv, SCALE), 900 + 2 * lv + t) for t in range(2)]
    rng = np.random.default_rng(seed + 10)
    levels = inputs.level_list(seed + 11, count, L - 1)
    ops = ["hmult" if v < 0.5 else "hrot" for v in rng.random(count)]
    rot_ix = rng.integers(0, len(rots), count)
    reqs = [Request(i, ops[i], int(levels[i]), rots[int(rot_ix[i])] if ops[i] == "hrot" else 0) for i in range(count)]
    lane_outs = [K.ckks_ct_create(ctx, L - 1) for _ in range(4)]   # one output per lane, reused

    inputs_for = lambda r: (pool[r.level][0], pool[r.level][1])
    key_for = lambda r: rk if r.op == "hmult" else gks[r.rot]
    # capacity: the whole request list back to back on one stream
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for r in reqs:
        a, b = inputs_for(r)
        if r.op == "hmult":
            K.ckks_hmult(ctx, a, b, rk, K.CKKS_RESCALE, lane_outs[0])
        else:
            K.ckks_hrot(ctx, a, r.rot, gks[r.rot], lane_outs[0])
    e1.record(stream)
    torch.cuda.synchronize()
    capacity = count / (e0.elapsed_time(e1) / 1e3)
    resident = (len(gks) + 1) * DNUM * 2 * (L + ALPHA) * (1 << LOG_N) * 4
    budget = resident + (4 << 30)
    results = {}
    for frac in fracs:
        arr = poisson_arrivals(np.random.default_rng(int(frac * 100)), count, frac * capacity)
        for r, t in zip(reqs, arr):
            r.arrival = t
        for name, lanes in (("one_op_per_launch", 1), ("continuous_batching_4_lanes", 4)):
            srv = Server(K, ctx, lanes, budget, 1 << LOG_N, resident_bytes=resident)
            try:
                done = srv.run(reqs, inputs_for, key_for, lane_outs=lane_outs[:lanes])
            finally:
                srv.close()
            results[f"{name}@{frac}"] = latency_stats(done)
    K.ckks_sync(ctx)
    for h in lane_outs + [c for v in pool.values() for c in v] + list(gks.values()):
        K.ckks_free(h)
    return results, capacity, resident


def run_serve(args, local_rank):
    import torch
    from paper_2407_13055_gb300 import ckks as K
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    q, p = K.ckks_gen_primes(LOG_N, L, ALPHA)
    ctx = K.ckks_ctx_create(LOG_N, q, p, DNUM, scale=SCALE, secret_hw=HW, stream=stream.cuda_stream)
    K.ckks_set_launch_flags(ctx, K.CKKS_LAUNCH_PDL if args.pdl == "on" else 0)
    sk = K.ckks_keygen_secret(ctx, 21)
    rk = K.ckks_keygen_relin(ctx, sk, 22)
    tuned = tune_levels(K, ctx, range(1, L), not args.no_tune, reps=2,
                        pkey=tune_cache.params_key(LOG_N, q, p, DNUM))
    count = args.requests
    results, capacity, resident = serve_runs(K, ctx, sk, rk, stream, count, (0.5, 0.8, 0.95))
    best = results["continuous_batching_4_lanes@0.95"]
    line = {"metric": "served HMult/HRot requests at N=2^16 (1 GB300): throughput and p50/p99 latency",
            "value": best["throughput_ops_s"], "unit": "requests/s", "n_gpus": 1, "steps": count, "warmup": 0,
            "ms_per_step": best["mean_ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u32", "data": "synthetic (fresh encryptions)",
            "config": {"workload": f"{count} Poisson requests, HMult+rescale / HRot 50:50, levels U{{1..39}}, "
                                   "64 resident rotation keys, arrival rate = 0.5/0.8/0.95 x one-stream "
                                   "capacity", "capacity_ops_s": capacity, "resident_key_bytes": resident,
                       "admission_budget_bytes": resident + (4 << 30),
                       "column_shapes": "tuned per level" if tuned else "default rule"},
            "runs": results}
    print(json.dumps(line), flush=True)
    for h in (sk, rk):
        K.ckks_free(h)
    K.ckks_ctx_destroy(ctx)


def main():
    global BATCH
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lanes", type=int, default=4, help="concurrent execution lanes (streams)")
    ap.add_argument("--workload", choices=["single", "batched", "serve", "hoisted", "bootstrap", "latency", "ablation", "rns2530"], default="single")
    ap.add_argument("--requests", type=int, default=2000, help="requests per served run (--workload serve)")
    ap.add_argument("--requests-default", type=int, default=1000,
                    help="requests of the served run reported in the default line")
    ap.add_argument("--no-tune", action="store_true", help="use the default column-kernel launch shapes")
    ap.add_argument("--tune-file", default=None,
                    help="JSON file of tuned launch shapes for this GPU (default: $CKKS_TUNE_CACHE, else one file "
                         "per GPU under ~/.cache/paper_2407_13055_gb300; 'none': tune every run, keep nothing)")
    ap.add_argument("--retune", action="store_true",
                    help="tune every level again and overwrite its entries in the tune file")
    ap.add_argument("--issue", choices=["graph", "direct", "python"], default="graph",
                    help="single workload: how the timed step's operations are issued")
    ap.add_argument("--batch", type=int, default=BATCH,
                    help="resident ciphertexts per step of the single-op workload (smaller only for profiling)")
    ap.add_argument("--col-shape", default=None,
                    help="tc,sl,z,tp: use this launch shape for the three column kernels at every level instead "
                         "of the tuner's (tp 8/16: tensor-core BConv)")
    ap.add_argument("--row-passes", type=int, default=None, choices=[2, 3, 4, 5, 6],
                    help="N=2^16 row-phase form instead of the tuner's (4, 5: forward rows staged by bulk copies; "
                         "6: twiddles in shared memory)")
    ap.add_argument("--e2e-slots", type=int, default=2,
                    help="buffer slots per lane of the end-to-end upload / compute / export pipeline")
    ap.add_argument("--e2e-priority", choices=["high", "normal"], default="high",
                    help="priority of the end-to-end leg's transfer streams")
    ap.add_argument("--pdl", choices=["on", "off"], default="on",
                    help="programmatic dependent launch for the key-switch kernels")
    args = ap.parse_args()
    BATCH = args.batch
    if args.col_shape:
        FORCED["col_shape"] = tuple(int(x) for x in args.col_shape.split(","))
    FORCED["row_passes"] = args.row_passes
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    open_tune_store(args, local_rank)
    if args.workload == "batched":
        run_batched(args, local_rank)
        return
    if args.workload == "serve":
        run_serve(args, local_rank)
        return
    if args.workload == "hoisted":
        run_hoisted(args, local_rank)
        return
    if args.workload == "bootstrap":
        run_bootstrap(args, local_rank)
        return
    if args.workload == "latency":
        run_latency(args, local_rank)
        return
    if args.workload == "ablation":
        run_ablation(args, local_rank)
        return
    if args.workload == "rns2530":
        run_rns2530(args, local_rank)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run_native(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
