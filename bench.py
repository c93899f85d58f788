#!/usr/bin/env python
"""Benchmark of the ZSMILES codec hot path on GB300.

Workload (N=1): the batched configuration - 64 shards of seeded synthetic SMILES lines (line counts log-uniform
in 1k-5M, per-shard mean length 25-70; about 49M lines, 2.47 GB), the frozen default dictionary.

One step = the whole hot path over those shards, through the C ABI on device-resident data:
    zs_plan_run of the compression plan (pre-processing + shortest-output parse + line index, all 64 shards in
    one persistent launch replayed from a CUDA graph, geometry autotuned)
    -> zs_plan_run of the decompression plan over the 64 compressed streams
    -> zs_decompress_lines of 100,000 random line ids of the largest shard (random access).
value = uncompressed bytes per second of step (GB/s, 1e9); the line also gives each direction on its own
(input GB/s and the fraction of HBM bandwidth its kernel reaches) and the random-access p99. Inputs are larger
than the 129 MB L2, so no flush is needed between steps. Extra keys: the batched form against one launch per
shard, config 1 (one 10M-line stream), config 3 (100M long-tail lines), the serving sweep (config 4), the
CPU oracle.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own replica of the 64 shards on its own line ranges (weak scaling,
no collective on the data path); timing is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "compress/decompress input GB/s (frac. of HBM peak); random-access p99 latency"
RA_IDS = 100_000
REF_BUDGET_S = 120.0  # CPU seconds the reference arm's warm-up and timed steps aim to take in all
HBM_FALLBACK_GBS = 6800.0
HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e, nominal (context only; fractions are taken of the measured peak)


def metric_name() -> str:
    return METRIC


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def kernel_traffic(kernel: str):
    """DRAM bytes per launch for `kernel` from the committed ncu summary, if the kernel source is unchanged
    since the counters were taken (the summary records the sha256 of its source file); else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        text = open(path).read()
    except OSError:
        return None
    for line in text.splitlines():
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel:
            src, sha, traffic = parts[1], parts[2], float(parts[3])
            cur = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()
            return traffic if cur == sha else None
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, begin: bool):
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for t, line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 10:
                continue
            try:
                rows.append((t, float(f[2]), float(f[3]), f[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if self.t0 is not None and self.t0 - 0.15 <= r[0] <= (self.t1 or r[0]) + 0.15]
        use = inside or rows
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in use for k in range(4) if r[3][k].lower().startswith("active")})
        return {"sm_mhz": float(np.median([r[1] for r in use])), "sm_max_mhz": max(r[2] for r in use),
                "reasons": reasons, "samples": len(use), "in_region": bool(inside)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_first_line(rank: int, lines: int) -> int:
    """First line of a rank's replica: ranks take consecutive, disjoint line ranges of one synthetic stream."""
    return rank * lines


def reduce_over_ranks(maxes, sums, device):
    """Max over ranks of the timing values and sum of the work values (identity with one process)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return [float(x) for x in maxes], [float(x) for x in sums]
    a = torch.tensor(list(maxes), dtype=torch.float64, device=device)
    b = torch.tensor(list(sums), dtype=torch.float64, device=device)
    dist.all_reduce(a, op=dist.ReduceOp.MAX)
    dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return a.tolist(), b.tolist()


def workload_desc_cfg2(n_shards: int, lines: int, nbytes: int) -> str:
    return (f"batched: {n_shards} shards, {lines:,} synthetic SMILES lines ({nbytes / 1e9:.2f} GB), line counts "
            "log-uniform 1k-5M, per-shard mean length 25-70; one persistent launch per direction (CUDA graph)")


def workload_desc(lines: int, nbytes: int) -> str:
    return (f"plain codec, large single stream: {lines:,} synthetic drug-like SMILES lines "
            f"({nbytes / 1e6:.1f} MB, mean {nbytes / max(1, lines):.1f} B/line incl. newline), one shard per launch")


# ---------------------------------------------------------------------------------------------------------
# CPU oracle (the reported baseline; also the reference arm)
# ---------------------------------------------------------------------------------------------------------

def oracle_round_trip(raw: np.ndarray, threads: int):
    import oracle
    d = oracle.Dict(open(os.path.join(ROOT, "paper_2404_19391_gb300", "data", "zs_default.zsd"), "rb").read())
    t0 = time.perf_counter()
    comp, idx = oracle.compress_stream_parallel(d, raw, oracle.PREPROCESS, threads=threads)
    t1 = time.perf_counter()
    oracle.decompress_stream_parallel(d, comp, threads=threads)
    t2 = time.perf_counter()
    rng = np.random.default_rng(1)
    ids = rng.integers(0, idx.size - 1, size=min(RA_IDS, idx.size - 1)).astype(np.uint64)
    oracle.decompress_lines(d, comp, idx, ids)
    t3 = time.perf_counter()
    return t1 - t0, t2 - t1, t3 - t2


def cpu_baseline(sample_lines: int, shape, threads: int | None = None, stream: str = "the same stream"):
    threads = threads or (os.cpu_count() or 1)
    raw = synth.generate(shape, 0, sample_lines)
    tc, td, tr = oracle_round_trip(raw, threads)
    total = tc + td + tr
    n_ids = min(RA_IDS, sample_lines)
    return {"value": raw.size / total / 1e9, "unit": "GB/s", "cores": threads, "kind": "oracle",
            "sample": f"first {sample_lines:,} lines ({raw.size / 1e6:.1f} MB) of {stream}; compress + "
                      f"decompress line-partitioned over {threads} thread(s), then {n_ids:,}-id random access "
                      f"(single thread)",
            "seconds": round(total, 3), "compress_s": round(tc, 3), "decompress_s": round(td, 3),
            "random_access_s": round(tr, 3)}


def cfg2_sample(sample_bytes: int):
    """A bounded sample of the batched workload: the first lines of every shard, the same fraction of each,
    about sample_bytes in all (one stream; lines are independent)."""
    specs = synth.batched_shards()
    total = sum(synth.lines_size(sh, 0, c) for sh, c in specs)
    f = min(1.0, sample_bytes / max(1, total))
    parts = [synth.generate(sh, 0, max(1, int(c * f))) for sh, c in specs]
    return np.concatenate(parts), f


def cpu_baseline_cfg2(sample_bytes: int, threads: int | None = None):
    threads = threads or (os.cpu_count() or 1)
    raw, f = cfg2_sample(sample_bytes)
    tc, td, tr = oracle_round_trip(raw, threads)
    total = tc + td + tr
    return {"value": raw.size / total / 1e9, "unit": "GB/s", "cores": threads, "kind": "oracle",
            "sample": f"the first {f * 100:.1f}% of the lines of each of the 64 shards ({raw.size / 1e6:.1f} MB); "
                      f"compress + decompress line-partitioned over {threads} thread(s), then {RA_IDS:,}-id "
                      "random access (single thread)",
            "seconds": round(total, 3), "compress_s": round(tc, 3), "decompress_s": round(td, 3),
            "random_access_s": round(tr, 3)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    # each step is a bounded sample of the workload (the first lines of every shard), sized from a timed probe
    # so that the warm-up and timed steps together take about REF_BUDGET_S of CPU work whatever --steps and
    # --warmup are
    probe, _ = cfg2_sample(5_000_000)
    t_probe = sum(oracle_round_trip(probe, threads))
    bytes_per_s = probe.size / max(t_probe, 1e-6)
    fit = int(bytes_per_s * REF_BUDGET_S / max(1, args.steps + args.warmup))
    raw, f = cfg2_sample(max(2_000_000, min(args.ref_sample_bytes, fit)))
    for _ in range(args.warmup):
        oracle_round_trip(raw, threads)
    times = []
    for _ in range(args.steps):
        tc, td, tr = oracle_round_trip(raw, threads)
        times.append(tc + td + tr)
    t = float(np.mean(times))
    value = raw.size / t / 1e9
    specs = synth.batched_shards()
    total = sum(synth.lines_size(sh, 0, c) for sh, c in specs)
    line = {"impl": "reference", "metric": metric_name(), "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": workload_desc_cfg2(len(specs), sum(c for _, c in specs), total),
                       "step": "CPU oracle round trip (compress + decompress + random access) over a bounded "
                               "sample of the workload"},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle",
                             "sample": f"the first {f * 100:.2f}% of the lines of each of the 64 shards "
                                       f"({raw.size / 1e6:.1f} MB) per step"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------------------
# GPU path
# ---------------------------------------------------------------------------------------------------------

def _aligned_shards(zs, specs, dev, first_of=lambda c: 0):
    """Generates [(shape, count)] (lines [first_of(count), + count) of each shard's stream) into one pinned
    buffer, each shard 16-byte aligned, copies it to the device; returns (device slices, sizes, line counts)."""
    import torch
    sizes = [synth.lines_size(sh, first_of(c), c) for sh, c in specs]
    spans = [(n + 15) & ~15 for n in sizes]
    host = torch.empty(max(16, sum(spans)), dtype=torch.uint8, pin_memory=True)
    at = 0
    for (sh, c), n, sp in zip(specs, sizes, spans):
        synth.generate_into(sh, first_of(c), c, host.data_ptr() + at, n)
        at += sp
    big = host.to(dev)
    ins, at = [], 0
    for n, sp in zip(sizes, spans):
        ins.append(big[at:at + n])
        at += sp
    return ins, sizes, [c for _, c in specs]


def _time_ms(stream, fn, reps):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def bench_serving(zs, d, dev, lines: int, n_req: int, rates):
    """Open-loop Poisson request streams (1-100,000 random ids per request, log-uniform) against a
    resident store of `lines` lines: the continuous-batching server vs one launch per request. The request
    sizes and ids are drawn once; each rate scales the arrival times (Poisson arrivals at rate r are those at
    rate 1 divided by r)."""
    import torch
    nbytes = synth.lines_size(synth.CFG4, 0, lines)
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    synth.generate_into(synth.CFG4, 0, lines, host.data_ptr(), nbytes)
    x = host.to(dev)
    del host
    comp, idx, _ = zs.compress(d, x)
    comp, idx = comp.clone(), idx.clone()
    del x
    base = synth.requests(n_req, 7, lines, rate=1.0)
    nid = sum(len(i) for _, i in base)
    srv = zs.Server(d, comp, idx, arena_bytes=2 << 30, max_inflight=4)
    rows = []
    for rate in rates:
        reqs = [(t / float(rate), ids) for t, ids in base]
        b0 = srv.stats()["batches"]
        lat, mk = srv.replay(reqs)
        nb = srv.stats()["batches"] - b0
        lat2, mk2 = zs.zs_serial_replay(d, comp, idx, reqs)
        rows.append({"rate_req_s": rate, "requests": n_req, "ids": nid,
                     "server": {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                                "lines_per_s": nid / mk, "launches": nb, "requests_per_launch": n_req / max(1, nb)},
                     "per_request": {"p50_ms": float(np.percentile(lat2, 50)),
                                     "p99_ms": float(np.percentile(lat2, 99)), "lines_per_s": nid / mk2}})
    st = srv.stats()
    srv.close()
    return {"workload": f"resident store of {lines:,} synthetic lines ({nbytes / 1e9:.2f} GB raw, "
                        f"{comp.numel() / 1e9:.2f} GB compressed + {idx.numel() * 8 / 1e9:.2f} GB index); "
                        f"{n_req:,} requests per rate, 1-100,000 ids each (log-uniform), ids uniform without "
                        "replacement",
            "rates": rows, "mean_requests_per_launch": st["mean_batch_requests"],
            "max_inflight": st["max_inflight"],
            "how": "zs_server_replay (continuous batching, 4 launches in flight, memory admission) vs "
                   "zs_serial_replay (one random-access launch + wait + copy per request, arrival order); "
                   "latency from scheduled arrival to result bytes in host memory"}


ABLATION = [  # (dictionary file, what it varies), the paper's sweeps (Sec. V-C) on the synthetic stream
    ("zs_default.zsd", "L_max 8, SMILES alphabet pre-populated, trained on pre-processed lines (default)"),
    ("zs_lmax5.zsd", "L_max 5"),
    ("zs_lmax15.zsd", "L_max 15"),
    ("zs_no_alphabet.zsd", "no pre-populated alphabet"),
    ("zs_raw_train.zsd", "trained on lines without ring-ID renumbering"),
    ("zs_outer_train.zsd", "trained on lines renumbered in opening order (the other reading of Sec. IV-A)"),
    ("zs_printable.zsd", "every printable byte pre-populated (Table I 'Printable'; 95 learned patterns)"),
    ("zs_printable_raw.zsd", "printable pre-population, trained on lines without ring-ID renumbering"),
    ("zs_no_alphabet_raw.zsd", "no pre-populated alphabet, trained on lines without ring-ID renumbering"),
]


def run_ablation(args):
    """Compression ratio and kernel times of each ablation dictionary on the benchmark stream, with
    pre-processing in either reading of Sec. IV-A (closing order, the default; opening order) and without
    (one JSON line)."""
    import torch
    from paper_2404_19391_gb300 import zsmiles as zs
    zs.load_library()
    lines = args.lines
    nbytes = synth.lines_size(synth.CFG1, 0, lines)
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    synth.generate_into(synth.CFG1, 0, lines, host.data_ptr(), nbytes)
    x = host.cuda()
    out = torch.empty(zs.zs_compress_bound(nbytes), dtype=torch.uint8, device="cuda")
    idx = torch.empty(lines + 2, dtype=torch.int64, device="cuda")
    rows = []
    for fname, what in ABLATION:
        d = zs.Dictionary(path=os.path.join(ROOT, "paper_2404_19391_gb300", "data", fname))
        dec = torch.empty(d.decompress_bound(zs.zs_compress_bound(nbytes)) // 4 + nbytes, dtype=torch.uint8,
                          device="cuda")
        for flags in (zs.PREPROCESS, zs.PREPROCESS | zs.PREPROCESS_OUTER, 0):
            for _ in range(2):
                r = zs.zs_compress(d, x, flags, out, idx)
            kc = []
            for _ in range(5):
                r = zs.zs_compress(d, x, flags, out, idx)
                kc.append(zs.zs_last_kernel_ms())
            comp = out[: r.out_len]
            kd = []
            for _ in range(3):
                rd = zs.zs_decompress(d, comp, dec)
                kd.append(zs.zs_last_kernel_ms())
            reading = None if not flags else ("opening" if flags & zs.PREPROCESS_OUTER else "closing")
            rows.append({"dictionary": fname, "varies": what, "preprocess": bool(flags), "reading": reading,
                         "lmax": d.lmax,
                         "transducer": d.uses_transducer, "ratio": r.out_len / nbytes,
                         "compress_ms": float(np.median(kc)), "compress_gbps_in": nbytes / np.median(kc) / 1e6,
                         "decompress_ms": float(np.median(kd)), "decoded_bytes": rd.out_len})
        d.close()
    print(json.dumps({"ablation": rows, "workload": workload_desc(lines, nbytes)}), flush=True)


def _concat_host(specs, first_of):
    """The shards' lines back to back in one pinned host buffer (lines are independent, so the shards'
    concatenation is one valid stream whose coding is the shards' codings back to back)."""
    import torch
    sizes = [synth.lines_size(sh, first_of(c), c) for sh, c in specs]
    host = torch.empty(max(1, sum(sizes)), dtype=torch.uint8, pin_memory=True)
    at = 0
    for (sh, c), n in zip(specs, sizes):
        synth.generate_into(sh, first_of(c), c, host.data_ptr() + at, n)
        at += n
    return host[:at], sizes


def bench_stream(zs, d, dev, shape, lines: int, peak: float, reps: int, first: int = 0, index: bool = True,
                 line_index: bool = False, plan: bool = False):
    """One stream through zs_compress and zs_decompress (one launch each), or (plan) through an autotuned
    plan each way (the geometry timed on the stream itself): kernel times (median of reps, CUDA events),
    GB/s, HBM fractions of the algorithmic bytes."""
    import torch
    nbytes = synth.lines_size(shape, first, lines)
    host = np.empty(nbytes, dtype=np.uint8)
    synth.generate_into(shape, first, lines, host.ctypes.data, nbytes)
    x = torch.from_numpy(host).to(dev)
    del host
    comp = torch.empty(zs.zs_compress_bound(nbytes), dtype=torch.uint8, device=dev)
    idx = torch.empty(lines + 2, dtype=torch.int64, device=dev) if index else None
    kc, kd = [], []
    variants = {}
    dec = torch.empty(nbytes + nbytes // 8 + 64, dtype=torch.uint8, device=dev)  # decoded <= input + %nn growth
    if plan:
        pc = zs.Plan(d, zs.OP_COMPRESS, [(x, comp, idx)], flags=zs.PREPROCESS, variant=-1, tune_reps=2)
        for k in range(reps + 1):
            r = pc.run()[0]
            if k:
                kc.append(pc.last_ms)
        variants["compress"] = zs.zs_kernel_variant_name(zs.OP_COMPRESS, pc.variant)
        pc.close()
        c = comp[: r.out_len]
        pd = zs.Plan(d, zs.OP_DECOMPRESS, [(c, dec, None)], variant=-1, tune_reps=2)
        for k in range(reps + 1):
            rd = pd.run()[0]
            if k:
                kd.append(pd.last_ms)
        variants["decompress"] = zs.zs_kernel_variant_name(zs.OP_DECOMPRESS, pd.variant)
        pd.close()
    else:
        for k in range(reps + 1):
            r = zs.zs_compress(d, x, zs.PREPROCESS, comp, idx)
            if k:
                kc.append(zs.zs_last_kernel_ms())
        c = comp[: r.out_len]
        for k in range(reps + 1):
            rd = zs.zs_decompress(d, c, dec)
            if k:
                kd.append(zs.zs_last_kernel_ms())
    assert r.n_lines == lines, (r.n_lines, lines)
    assert rd.n_lines == lines
    kc, kd = float(np.median(kc)), float(np.median(kd))
    ca = nbytes + r.out_len + (8 * (lines + 1) if index else 0)
    da = r.out_len + rd.out_len
    out = {"lines": lines, "bytes": nbytes, "ratio": r.out_len / nbytes,
           "compress": {"kernel_ms": kc, "gbps_in": nbytes / kc / 1e6, "lines_per_s": lines / (kc * 1e-3),
                        "hbm_gbps": ca / kc / 1e6, "hbm_frac": ca / kc / 1e6 / peak,
                        "algorithmic_bytes": ca},
           "decompress": {"kernel_ms": kd, "gbps_in": r.out_len / kd / 1e6, "gbps_out": rd.out_len / kd / 1e6,
                          "hbm_gbps": da / kd / 1e6, "hbm_frac": da / kd / 1e6 / peak, "algorithmic_bytes": da},
           "decoded_bytes": rd.out_len}
    if variants:
        out["variants"] = variants
    if line_index and index:  # the index rebuilt from the compressed stream alone, against the compressor's
        idx2 = torch.empty(lines + 2, dtype=torch.int64, device=dev)
        li = []
        for k in range(reps + 1):
            n_li = zs.zs_build_line_index(c, idx2)
            if k:
                li.append(zs.zs_last_kernel_ms())
        lk = float(np.median(li))
        la = r.out_len + 8 * (lines + 1)
        out["line_index"] = {"kernel_ms": lk, "gbps_in": r.out_len / lk / 1e6, "hbm_gbps": la / lk / 1e6,
                             "hbm_frac": la / lk / 1e6 / peak,
                             "identical_to_compress_index": bool(n_li == lines and torch.equal(idx2[: lines + 1],
                                                                                                 idx[: lines + 1]))}
        del idx2
    del x, comp, idx, dec
    torch.cuda.empty_cache()
    return out


def long_line_stream(base: np.ndarray, count: int = 50, lo: int = 4096, hi: int = 8192, seed: int = 3) -> np.ndarray:
    """base with `count` lines of lo..hi bytes spliced in at seeded line boundaries; each long line is made of
    long-tail lines (ring labels, bracket atoms, %nn) joined without separators, so it stays one valid line."""
    rng = np.random.default_rng(seed)
    frag = [l for l in bytes(synth.generate(synth.CFG3, 0, 20000)).split(b"\n")[:-1] if len(l) > 150]
    longs = []
    for _ in range(count):
        target, cur = int(rng.integers(lo, hi + 1)), b""
        while len(cur) < target:
            cur += frag[int(rng.integers(0, len(frag)))]
        longs.append(cur + b"\n")
    nl = np.flatnonzero(base == 10)
    at = np.sort(rng.choice(nl.size, count, replace=False))
    parts, prev = [], 0
    for k, i in enumerate(at):
        cut = int(nl[i]) + 1
        parts.append(base[prev:cut])
        parts.append(np.frombuffer(longs[k], dtype=np.uint8))
        prev = cut
    parts.append(base[prev:])
    return np.concatenate(parts)


def bench_long_lines(zs, d, dev, lines: int, reps: int = 3):
    """Compression of the drug-like stream with and without 50 lines of 4-8 KB (longer than any tile's stage),
    each through an autotuned plan: kernel time of both, and their ratio."""
    import torch
    nbytes = synth.lines_size(synth.CFG1, 0, lines)
    base = np.empty(nbytes, dtype=np.uint8)
    synth.generate_into(synth.CFG1, 0, lines, base.ctypes.data, nbytes)
    mixed = long_line_stream(base)
    out = {}
    for name, host in (("base", base), ("with_long_lines", mixed)):
        x = torch.from_numpy(host).to(dev)
        comp = torch.empty(zs.zs_compress_bound(host.size), dtype=torch.uint8, device=dev)
        idx = torch.empty(int(np.count_nonzero(host == 10)) + 2, dtype=torch.int64, device=dev)
        pc = zs.Plan(d, zs.OP_COMPRESS, [(x, comp, idx)], flags=zs.PREPROCESS, variant=-1, tune_reps=2)
        ts = []
        for k in range(reps + 1):
            pc.run()
            if k:
                ts.append(pc.last_ms)
        out[name] = {"bytes": int(host.size), "kernel_ms": float(np.median(ts)),
                     "variant": zs.zs_kernel_variant_name(zs.OP_COMPRESS, pc.variant)}
        pc.close()
        del x, comp, idx
        torch.cuda.empty_cache()
    out["ratio"] = out["with_long_lines"]["kernel_ms"] / out["base"]["kernel_ms"]
    out["workload"] = (f"{lines:,} drug-like lines, then the same with 50 lines of 4-8 KB (long-tail lines joined, "
                       "longer than any tile and its halo) spliced in at seeded line boundaries; autotuned plan each")
    return out


def _read_into(path: str, arr: np.ndarray) -> int:
    """Reads the file into arr (a host buffer), looping over partial reads (one read() stops near 2 GB)."""
    mv, got = memoryview(arr).cast("B"), 0
    with open(path, "rb", buffering=0) as f:
        while got < mv.nbytes:
            n = f.readinto(mv[got:])
            if not n:
                break
            got += n
    return got


def _write_from(path: str, arr: np.ndarray) -> int:
    """Writes arr (a host buffer) to the file, looping over partial writes."""
    mv, put = memoryview(arr).cast("B"), 0
    with open(path, "wb", buffering=0) as f:
        while put < mv.nbytes:
            put += f.write(mv[put:])
    return put


def _storage_dir(need: int):
    """A scratch directory with `need` bytes free: /dev/shm (memory) if it has room, else the system temporary
    directory; None if neither does."""
    import shutil
    import tempfile
    for base in ("/dev/shm", tempfile.gettempdir()):
        try:
            if os.path.isdir(base) and shutil.disk_usage(base).free > need:
                return tempfile.mkdtemp(prefix="zs_storage_", dir=base)
        except OSError:
            pass
    return None


def run_gpu(args):
    import torch
    from paper_2404_19391_gb300 import zsmiles as zs

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    zs.load_library()
    d = zs.Dictionary()
    peak, peak_kind = hbm_peak()
    stream = torch.cuda.current_stream(dev)

    # ---- the workload: config 2, 64 shards in one batched plan each way. Rank r takes the lines
    # [r * count, (r + 1) * count) of every shard's seeded stream (weak scaling, no collective) ----
    specs = synth.batched_shards()
    first_of = (lambda c: rank * c)
    ins, sizes, counts = _aligned_shards(zs, specs, dev, first_of)
    nbytes, nlines = sum(sizes), sum(counts)
    outs = [torch.empty(zs.zs_compress_bound(n), dtype=torch.uint8, device=dev) for n in sizes]
    idxs = [torch.empty(c + 2, dtype=torch.int64, device=dev) for c in counts]
    shards = list(zip(ins, outs, idxs))
    t0 = time.time()
    plan_c = zs.Plan(d, zs.OP_COMPRESS, shards, flags=zs.PREPROCESS, variant=-1, tune_reps=2)
    tune_c = time.time() - t0
    res_c = plan_c.run()
    assert [r.n_lines for r in res_c] == counts
    comps = [o[: r.out_len] for o, r in zip(outs, res_c)]
    cbytes = sum(r.out_len for r in res_c)
    douts = [torch.empty(n + n // 8 + 64, dtype=torch.uint8, device=dev) for n in sizes]
    dsh = [(c, o, None) for c, o in zip(comps, douts)]
    t0 = time.time()
    plan_d = zs.Plan(d, zs.OP_DECOMPRESS, dsh, variant=-1, tune_reps=2)
    tune_d = time.time() - t0
    res_d = plan_d.run()
    dbytes = sum(r.out_len for r in res_d)
    assert [r.n_lines for r in res_d] == counts
    big = int(np.argmax(counts))  # random access reads the largest shard's stream and index
    store, store_idx = comps[big], idxs[big][: counts[big] + 1]
    rng = np.random.default_rng(1000 + rank)
    ids_host = torch.from_numpy(rng.integers(0, counts[big], size=RA_IDS).astype(np.int64)).pin_memory()
    ids = ids_host.to(dev)
    ra_out = torch.empty(RA_IDS * 256, dtype=torch.uint8, device=dev)
    ra_off = torch.empty(RA_IDS + 1, dtype=torch.int64, device=dev)
    kms = {"compress": [], "decompress": [], "lines": []}

    def step(record=True):
        plan_c.run()
        kc = plan_c.last_ms
        plan_d.run()
        kd = plan_d.last_ms
        zs.zs_decompress_lines(d, store, store_idx, ids, ra_out, ra_off)
        kl = zs.zs_last_kernel_ms()
        if record:
            kms["compress"].append(kc)
            kms["decompress"].append(kd)
            kms["lines"].append(kl)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        step(record=False)
    visible = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")
    smi_index = int(visible[local]) if len(visible) > local and visible[local].strip().isdigit() else local
    clocks = ClockSampler(smi_index)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize(dev)
    clocks.mark(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark(False)
    barrier()
    ms_total = e0.elapsed_time(e1)

    # ---- end to end through the host-buffer API: the 64 shards back to back in pinned host memory (one
    # stream), zs_compress_host to pinned host stream + index, zs_decompress_host of that to pinned host
    # text, and the 100,000-id request from host ids into host memory against the device-resident store ----
    host_in, _ = _concat_host(specs, first_of)
    host_comp = torch.empty(cbytes + 64, dtype=torch.uint8, pin_memory=True)
    host_idx = torch.empty(nlines + 2, dtype=torch.int64, pin_memory=True)
    host_dec = torch.empty(dbytes + 64, dtype=torch.uint8, pin_memory=True)
    host_ra = torch.empty(ra_out.numel(), dtype=torch.uint8, pin_memory=True)
    host_off = torch.empty(ra_off.numel(), dtype=torch.int64, pin_memory=True)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    io = {}

    def e2e_step():
        r = zs.zs_compress_host(d, host_in, zs.PREPROCESS, host_comp, host_idx)
        rd = zs.zs_decompress_host(d, host_comp[: r.out_len], host_dec)
        ids.copy_(ids_host, non_blocking=True)
        rl = zs.zs_decompress_lines(d, store, store_idx, ids, ra_out, ra_off)
        host_ra[: rl.out_len].copy_(ra_out[: rl.out_len], non_blocking=True)
        host_off.copy_(ra_off, non_blocking=True)
        torch.cuda.synchronize(dev)
        io.update(h2d=host_in.numel() + r.out_len + ids_host.numel() * 8,
                  d2h=r.out_len + (r.n_lines + 1) * 8 + rd.out_len + rl.out_len + ra_off.numel() * 8,
                  same=(r.out_len == cbytes and r.n_lines == nlines and rd.out_len == dbytes))

    e2e_step()
    torch.cuda.synchronize(dev)
    barrier()
    w0 = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize(dev)
    e2e_ms = (time.perf_counter() - w0) * 1e3 / e2e_steps
    barrier()
    clocks.stop()

    # ---- storage leg: the step's compression and decompression from and to files. The 64 shards as one text
    # file (written once, untimed); each timed step reads it into pinned memory, compresses it through the host
    # pipeline, writes the compressed file and its line index, reads the compressed file back, decompresses it
    # and writes the decoded text file. The files sit in the box's page cache (or /dev/shm): this measures the
    # host file path around the GPU, not a storage device ----
    storage = None
    sdir = _storage_dir(3 * nbytes + 2 * cbytes + 16 * nlines + (1 << 30))
    if sdir is not None:
        import shutil
        fin, fz, fx, fo = (os.path.join(sdir, f"{k}_{rank}") for k in ("in.smi", "out.zs", "out.idx", "out.smi"))
        hin_np, hcomp_np, hidx_np, hdec_np = host_in.numpy(), host_comp.numpy(), host_idx.numpy(), host_dec.numpy()
        _write_from(fin, hin_np)
        sio = {}

        def storage_step():
            got = _read_into(fin, hin_np)
            r = zs.zs_compress_host(d, host_in, zs.PREPROCESS, host_comp, host_idx)
            w1 = _write_from(fz, hcomp_np[: r.out_len]) + _write_from(fx, hidx_np[: r.n_lines + 1])
            got2 = _read_into(fz, hcomp_np[: r.out_len])
            rd = zs.zs_decompress_host(d, host_comp[: r.out_len], host_dec)
            w2 = _write_from(fo, hdec_np[: rd.out_len])
            sio.update(read=got + got2, written=w1 + w2,
                       same=(got == nbytes and r.out_len == cbytes and r.n_lines == nlines and rd.out_len == dbytes))

        storage_step()
        st_steps = max(1, min(3, e2e_steps))
        barrier()
        w0 = time.perf_counter()
        for _ in range(st_steps):
            storage_step()
        st_ms = (time.perf_counter() - w0) * 1e3 / st_steps
        barrier()
        shutil.rmtree(sdir, ignore_errors=True)
        storage = {"value": nbytes / (st_ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": st_ms, "steps": st_steps,
                   "read_bytes_per_step": sio["read"], "written_bytes_per_step": sio["written"],
                   "same_sizes_as_device_step": sio["same"], "directory": os.path.dirname(sdir),
                   "leg": "text file -> pinned -> H2D -> compress -> D2H -> compressed + index files; compressed "
                          "file -> pinned -> H2D -> decompress -> D2H -> text file (page cache or /dev/shm)"}
    del host_in, host_comp, host_idx, host_dec

    (ms_step, e2e_ms), (total_bytes,) = reduce_over_ranks([ms_total / args.steps, e2e_ms], [nbytes], dev)
    value = total_bytes / (ms_step * 1e-3) / 1e9
    kc = float(np.mean(kms["compress"]))
    kd = float(np.mean(kms["decompress"]))
    kl = float(np.mean(kms["lines"]))
    c_alg = nbytes + cbytes + 8 * (nlines + len(counts))  # read the text, write the streams and the indexes
    d_alg = cbytes + dbytes                                # read the streams, write the text
    achieved_c, achieved_d = c_alg / kc / 1e6, d_alg / kd / 1e6
    cvar = zs.zs_kernel_variant_name(zs.OP_COMPRESS, plan_c.variant)
    dvar = zs.zs_kernel_variant_name(zs.OP_DECOMPRESS, plan_d.variant)
    ckernel = "compress_span_kernel" if "span" in cvar else "compress_warp_kernel"
    traffic = kernel_traffic(ckernel)
    if traffic is not None:
        traffic *= nbytes  # the committed figure is per input byte

    if rank == 0:
        # ---- the same shards one launch per shard (zs_compress / zs_decompress per shard, as a caller without
        # the batched form would), identical output; wall time and the shards' kernel times summed ----
        ref_c = [o[: r.out_len].clone() for o, r in zip(outs, res_c)]
        ref_d = [o[: r.out_len].clone() for o, r in zip(douts, res_d)]

        def per_shard(op):
            ks = []
            for (x, o, i), c, dd in zip(shards, comps, douts):
                if op == "c":
                    zs.zs_compress(d, x, zs.PREPROCESS, o, i)
                else:
                    zs.zs_decompress(d, c, dd)
                ks.append(zs.zs_last_kernel_ms())
            return sum(ks)

        per = {}
        for op in ("c", "d"):
            per_shard(op)
            ks = []
            w0 = torch.cuda.Event(enable_timing=True)
            w1 = torch.cuda.Event(enable_timing=True)
            w0.record(stream)
            for _ in range(3):
                ks.append(per_shard(op))
            w1.record(stream)
            torch.cuda.synchronize(dev)
            per[op] = (w0.elapsed_time(w1) / 3, float(np.mean(ks)))
        same_c = all(torch.equal(o[: r.out_len], c) for o, r, c in zip(outs, res_c, ref_c))
        same_d = all(torch.equal(o[: r.out_len], c) for o, r, c in zip(douts, res_d, ref_d))
        del ref_c, ref_d
        batched = {
            "compress": {"batched_kernel_ms": kc, "batched_step_ms": None, "per_shard_wall_ms": per["c"][0],
                         "per_shard_kernel_ms_sum": per["c"][1], "speedup_wall": per["c"][0] / kc,
                         "speedup_kernel": per["c"][1] / kc, "identical_output": bool(same_c),
                         "variant": cvar, "autotune_s": tune_c,
                         "tuned_ms": {zs.zs_kernel_variant_name(0, v): plan_c.tuned_ms(v)
                                      for v in range(zs.zs_kernel_variants(0))}},
            "decompress": {"batched_kernel_ms": kd, "per_shard_wall_ms": per["d"][0],
                           "per_shard_kernel_ms_sum": per["d"][1], "speedup_wall": per["d"][0] / kd,
                           "speedup_kernel": per["d"][1] / kd, "identical_output": bool(same_d),
                           "variant": dvar, "autotune_s": tune_d,
                           "tuned_ms": {zs.zs_kernel_variant_name(1, v): plan_d.tuned_ms(v)
                                        for v in range(zs.zs_kernel_variants(1))}},
            "how": "batched = zs_plan_run of an autotuned plan replaying one CUDA graph (clear, one persistent "
                   "launch over all shards, result copy), kernel time from events captured around the launch; "
                   "per shard = one zs_compress / zs_decompress call per shard (wall, mean of 3 passes; and the "
                   "shards' own kernel times summed)"}
    plan_c.close()
    plan_d.close()
    del ins, outs, idxs, shards, comps, douts, dsh, ra_out, store, store_idx
    torch.cuda.empty_cache()

    if rank == 0:
        # ---- the other configurations: config 1 (one 10M-line stream, one launch each way, plus the line index
        # rebuilt from its compressed stream) and config 3 (the long-tail mix at its full 100M lines) ----
        cfg1 = bench_stream(zs, d, dev, synth.CFG1, args.lines, peak, reps=5, line_index=True)
        cfg1["workload"] = workload_desc(args.lines, cfg1["bytes"])
        cfg3 = None
        if args.cfg3_lines > 0:
            cfg3 = bench_stream(zs, d, dev, synth.CFG3, args.cfg3_lines, peak, reps=3, plan=True)
            cfg3["workload"] = (f"batched long tail: {args.cfg3_lines:,} synthetic lines ({cfg3['bytes'] / 1e9:.2f} "
                                "GB), 90% drug-like, 10% of 150-400 chars with bracket atoms, stereo bonds and "
                                "%nn ring labels; one stream, one autotuned plan (CUDA graph) each way")
        long_lines = bench_long_lines(zs, d, dev, args.lines) if args.cfg3_lines > 0 else None
        line = {
            "metric": metric_name(), "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": workload_desc_cfg2(len(specs), nlines, nbytes), "shards": len(specs),
                       "lines_per_rank": nlines, "bytes_per_rank": nbytes,
                       "dictionary": "frozen default (Algorithm 1, seed-1 100k-line training set, L_max 8, T 146)",
                       "dictionary_sha256": hashlib.sha256(open(zs.DEFAULT_DICTIONARY, "rb").read()).hexdigest(),
                       "step": "zs_plan_run of the compression plan (64 shards, one launch) + zs_plan_run of the "
                               f"decompression plan + zs_decompress_lines({RA_IDS:,} random ids of the largest shard)",
                       "value": "uncompressed bytes of the 64 shards per second of step",
                       "l2": "inputs (and outputs) larger than the 129 MB L2; no flush",
                       "parallelism": f"{world} independent replica(s)"},
            "clocks": clocks.summary(),
            "compress_gbps_in": nbytes / kc / 1e6, "compress_hbm_frac": achieved_c / peak,
            "decompress_gbps_in": cbytes / kd / 1e6, "decompress_hbm_frac": achieved_d / peak,
            "random_access_p99_ms": float(np.percentile(kms["lines"], 99)),
            "e2e": {"value": total_bytes / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": io["h2d"],
                    "d2h_bytes_per_step": io["d2h"], "ms_per_step": e2e_ms, "same_sizes_as_device_step": io["same"],
                    "how": "wall clock per step of zs_compress_host (the 64 shards back to back in pinned host "
                           "memory, to a pinned host stream and index) + zs_decompress_host (that stream to pinned "
                           f"host text) + {RA_IDS:,} random ids H2D, zs_decompress_lines on the device-resident "
                           "largest shard, lines and offsets D2H"},
            # per step: compress (span geometries: a probe for lines longer than the stage, the span kernel and
            # the patch kernel that writes such lines), decompress, random access
            "gpu_launches": ((3 if "span" in cvar else 1) + 2) * args.steps,
            "e2e_storage": storage if storage is not None else {"unavailable": "no scratch directory with room"},
            "roofline": {"bound": "hbm", "achieved": achieved_c, "peak": peak, "unit": "GB/s",
                         "frac": achieved_c / peak, "traffic": traffic, "kernel": ckernel,
                         "peak_kind": f"{peak_kind} (copy, MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                         else "fallback 6.8 TB/s",
                         "algorithmic_bytes_per_launch": c_alg, "kernel_ms": kc},
            "compress": {"kernel_ms": kc, "gbps_in": nbytes / kc / 1e6, "lines_per_s": nlines / (kc * 1e-3),
                         "hbm_gbps": achieved_c, "hbm_frac": achieved_c / peak,
                         "hbm_frac_nominal": achieved_c / HBM_NOMINAL_GBS, "ratio": cbytes / nbytes,
                         "algorithmic_bytes": c_alg, "variant": cvar},
            "decompress": {"kernel_ms": kd, "gbps_in": cbytes / kd / 1e6, "gbps_out": dbytes / kd / 1e6,
                           "hbm_gbps": achieved_d, "hbm_frac": achieved_d / peak,
                           "hbm_frac_nominal": achieved_d / HBM_NOMINAL_GBS, "algorithmic_bytes": d_alg,
                           "variant": dvar},
            "random_access": {"ids": RA_IDS, "kernel_ms": kl, "lines_per_s": RA_IDS / (kl * 1e-3),
                              "p50_ms": float(np.percentile(kms["lines"], 50)),
                              "p99_ms": float(np.percentile(kms["lines"], 99))},
            "batched": batched,
            "config1": cfg1,
        }
        if cfg3 is not None:
            line["config3"] = cfg3
        if long_lines is not None:
            line["long_lines"] = long_lines
        if world == 1 and not args.no_serving:
            line["serving"] = bench_serving(zs, d, dev, args.serve_lines, args.serve_requests,
                                            [int(r) for r in args.serve_rates.split(",")])
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_cfg2(args.cpu_sample_bytes)
            line["cpu_oracle_cfg0"] = {t: cpu_baseline(synth.CFG0_LINES, synth.CFG0, threads=n,
                                                       stream="the 10,000-line config-0 stream")
                                       for t, n in (("single_thread", 1), ("all_threads", None))}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_profile_stream(args):
    """A small case of the two kernels the headline step runs (for a profiler): one drug-like and one long-tail
    stream of args.profile_stream lines, each compressed and decompressed 4 times by the single-call API."""
    import torch
    from paper_2404_19391_gb300 import zsmiles as zs
    zs.load_library()
    d = zs.Dictionary()
    peak, _ = hbm_peak()
    out = {}
    for name, shape in (("drug_like", synth.CFG1), ("long_tail", synth.CFG3)):
        out[name] = bench_stream(zs, d, torch.device("cuda", 0), shape, args.profile_stream, peak, reps=3)
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lines", type=int, default=synth.CFG1_LINES, help="lines of the config-1 stream")
    ap.add_argument("--cfg3-lines", type=int, default=synth.CFG3_LINES,
                    help="lines of the config-3 long-tail stream (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--cpu-sample-bytes", type=int, default=1_000_000_000,
                    help="bytes of the batched workload the CPU oracle codes for the cpu_baseline key")
    ap.add_argument("--ref-sample-bytes", type=int, default=20_000_000,
                    help="largest per-step sample of the reference arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-stream", type=int, default=0,
                    help="only time one drug-like and one long-tail stream of this many lines through the "
                         "single-call API (a small case for a profiler capture)")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-form request replay")
    ap.add_argument("--serve-lines", type=int, default=synth.CFG4_LINES)
    ap.add_argument("--serve-requests", type=int, default=20_000)
    ap.add_argument("--serve-rates", default="1000,3000,10000,30000,100000")
    ap.add_argument("--ablation", action="store_true",
                    help="instead of the benchmark line: ratio and kernel times of the ablation dictionaries")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.profile_stream:
        run_profile_stream(args)
    elif args.ablation:
        run_ablation(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
