#!/usr/bin/env python
"""Benchmark of the ZSMILES codec hot path on GB300.

Workload (N=1): the large single-stream configuration - 10,000,000 seeded synthetic SMILES lines
(drug-like, mean ~49 bytes, ~490 MB), one shard per launch, the frozen default dictionary.

One step = the whole hot path over that stream, through the C ABI on device-resident data:
    zs_compress (pre-processing + shortest-output parse + line index)
    -> zs_decompress of the result
    -> zs_decompress_lines of 100,000 random line ids (random access).
value = uncompressed bytes per second of step (GB/s, 1e9). Inputs (490 MB) are larger than the 129 MB L2,
so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--lines L]

Under torchrun (N > 1) every rank runs its own replica on its own 10M-line range (weak scaling, no
collective on the data path); timing is the max over ranks.
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


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    shape = synth.CFG1
    # each step is a bounded sample of the workload, sized from a timed probe so that the warm-up and timed
    # steps together take about REF_BUDGET_S of CPU work whatever --steps and --warmup are
    probe = synth.generate(shape, 0, 100_000)
    t_probe = sum(oracle_round_trip(probe, threads))
    lines_per_s = 100_000 / max(t_probe, 1e-6)
    fit = int(lines_per_s * REF_BUDGET_S / max(1, args.steps + args.warmup))
    sample = max(10_000, min(args.ref_sample_lines, fit))
    raw = synth.generate(shape, 0, sample)
    for _ in range(args.warmup):
        oracle_round_trip(raw, threads)
    times = []
    for _ in range(args.steps):
        tc, td, tr = oracle_round_trip(raw, threads)
        times.append(tc + td + tr)
    t = float(np.mean(times))
    value = raw.size / t / 1e9
    line = {"impl": "reference", "metric": metric_name(), "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": {"workload": workload_desc(args.lines, synth.lines_size(shape, 0, args.lines)),
                       "step": "CPU oracle round trip (compress + decompress + random access) over a bounded "
                               "sample of the workload"},
            "cpu_baseline": {"value": value, "unit": "GB/s", "cores": threads, "kind": "oracle",
                             "sample": f"first {sample:,} lines ({raw.size / 1e6:.1f} MB) per step"},
            "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------------------
# GPU path
# ---------------------------------------------------------------------------------------------------------

def _aligned_shards(zs, specs, dev):
    """Generates [(shape, count)] into one pinned buffer (each shard 16-byte aligned), copies it to the
    device; returns (device slices, sizes, line counts)."""
    import torch
    sizes = [synth.lines_size(sh, 0, c) for sh, c in specs]
    spans = [(n + 15) & ~15 for n in sizes]
    host = torch.empty(max(16, sum(spans)), dtype=torch.uint8, pin_memory=True)
    at = 0
    for (sh, c), n, sp in zip(specs, sizes, spans):
        synth.generate_into(sh, 0, c, host.data_ptr() + at, n)
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


def bench_batched(zs, d, dev, reps: int, peak: float):
    """64 shards (log-uniform 1k-5M lines, per-shard mean length 25-70) through one autotuned,
    graph-captured plan, against one zs_compress / zs_decompress launch per shard, same buffers."""
    import torch
    specs = synth.batched_shards()
    ins, sizes, counts = _aligned_shards(zs, specs, dev)
    outs = [torch.empty(zs.zs_compress_bound(n), dtype=torch.uint8, device=dev) for n in sizes]
    idxs = [torch.empty(c + 2, dtype=torch.int64, device=dev) for c in counts]
    shards = list(zip(ins, outs, idxs))
    stream = torch.cuda.current_stream(dev)
    t0 = time.time()
    plan = zs.Plan(d, zs.OP_COMPRESS, shards, flags=zs.PREPROCESS, variant=-1, tune_reps=2)
    tune_s = time.time() - t0
    res = plan.run()
    for _ in range(2):
        plan.run()
    ms_b = _time_ms(stream, plan.run, reps)
    kern_b = plan.last_ms
    ref = [o[: r.out_len].clone() for o, r in zip(outs, res)]

    def per_shard_c():
        for x, o, i in shards:
            zs.zs_compress(d, x, zs.PREPROCESS, o, i)
    per_shard_c()
    ms_p = _time_ms(stream, per_shard_c, reps)
    same_c = all(torch.equal(o[: r.out_len], c) for o, r, c in zip(outs, res, ref))
    del ref
    comps = [o[: r.out_len] for o, r in zip(outs, res)]
    douts = [torch.empty(d.decompress_bound(c.numel()) // 2 + n + 64, dtype=torch.uint8, device=dev)
             for c, n in zip(comps, sizes)]
    dsh = [(c, o, None) for c, o in zip(comps, douts)]
    dplan = zs.Plan(d, zs.OP_DECOMPRESS, dsh, variant=-1, tune_reps=2)
    dres = dplan.run()
    ms_db = _time_ms(stream, dplan.run, reps)
    kern_db = dplan.last_ms
    dref = [o[: r.out_len].clone() for o, r in zip(douts, dres)]

    def per_shard_d():
        for c, o, _ in dsh:
            zs.zs_decompress(d, c, o)
    per_shard_d()
    ms_dp = _time_ms(stream, per_shard_d, reps)
    same_d = all(torch.equal(o[: r.out_len], x) for o, r, x in zip(douts, dres, dref))
    nbytes, cbytes = sum(sizes), sum(c.numel() for c in comps)
    # algorithmic bytes: compress reads the text and writes the stream and the index (n_lines + 1 entries a
    # shard); decompress reads the stream and writes the text
    c_alg = nbytes + cbytes + 8 * (sum(counts) + len(counts))
    d_alg = cbytes + nbytes
    out = {
        "workload": f"{len(specs)} shards, {sum(counts):,} synthetic lines, {nbytes / 1e9:.2f} GB, line counts "
                    "log-uniform 1k-5M, per-shard mean length 25-70",
        "compress": {"batched_ms": ms_b, "batched_kernel_ms": kern_b, "per_shard_ms": ms_p,
                     "speedup": ms_p / ms_b, "batched_gbps_in": nbytes / ms_b / 1e6,
                     "per_shard_gbps_in": nbytes / ms_p / 1e6, "variant": zs.zs_kernel_variant_name(0, plan.variant),
                     "tuned_ms": {zs.zs_kernel_variant_name(0, v): plan.tuned_ms(v)
                                  for v in range(zs.zs_kernel_variants(0))},
                     "autotune_s": tune_s, "identical_output": bool(same_c),
                     "hbm_gbps": c_alg / kern_b / 1e6, "hbm_frac": c_alg / kern_b / 1e6 / peak,
                     "hbm_frac_nominal": c_alg / kern_b / 1e6 / HBM_NOMINAL_GBS},
        "decompress": {"batched_ms": ms_db, "per_shard_ms": ms_dp, "speedup": ms_dp / ms_db,
                       "batched_gbps_in": cbytes / ms_db / 1e6, "per_shard_gbps_in": cbytes / ms_dp / 1e6,
                       "variant": zs.zs_kernel_variant_name(1, dplan.variant),
                       "tuned_ms": {zs.zs_kernel_variant_name(1, v): dplan.tuned_ms(v)
                                    for v in range(zs.zs_kernel_variants(1))},
                       "identical_output": bool(same_d), "batched_kernel_ms": kern_db,
                       "hbm_gbps": d_alg / kern_db / 1e6, "hbm_frac": d_alg / kern_db / 1e6 / peak,
                       "hbm_frac_nominal": d_alg / kern_db / 1e6 / HBM_NOMINAL_GBS},
        "how": "batched = zs_plan_run of an autotuned plan replaying one CUDA graph (clear, one persistent "
               "launch over all shards, result copy); per-shard = one zs_compress / zs_decompress call per shard; "
               f"wall time per pass with CUDA events, mean of {reps} passes",
    }
    plan.close()
    dplan.close()
    return out


def bench_serving(zs, d, dev, lines: int, n_req: int, rates):
    """Open-loop Poisson request streams (1-100,000 random ids per request, log-uniform) against a
    resident store of `lines` lines: the continuous-batching server vs one launch per request."""
    import torch
    nbytes = synth.lines_size(synth.CFG4, 0, lines)
    host = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    synth.generate_into(synth.CFG4, 0, lines, host.data_ptr(), nbytes)
    x = host.to(dev)
    comp, idx, _ = zs.compress(d, x)
    comp, idx = comp.clone(), idx.clone()
    del x
    srv = zs.Server(d, comp, idx, arena_bytes=2 << 30, max_inflight=4)
    rows = []
    for rate in rates:
        reqs = synth.requests(n_req, 7, lines, rate=float(rate))
        nid = sum(len(i) for _, i in reqs)
        lat, mk = srv.replay(reqs)
        lat2, mk2 = zs.zs_serial_replay(d, comp, idx, reqs)
        rows.append({"rate_req_s": rate, "requests": n_req, "ids": nid,
                     "server": {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                                "lines_per_s": nid / mk},
                     "per_request": {"p50_ms": float(np.percentile(lat2, 50)),
                                     "p99_ms": float(np.percentile(lat2, 99)), "lines_per_s": nid / mk2}})
    st = srv.stats()
    srv.close()
    return {"workload": f"resident store of {lines:,} synthetic lines ({nbytes / 1e9:.2f} GB raw, "
                        f"{comp.numel() / 1e9:.2f} GB compressed + {idx.numel() * 8 / 1e9:.2f} GB index)",
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

    shape = synth.CFG1
    lines = args.lines
    first = rank_first_line(rank, lines)
    nbytes = synth.lines_size(shape, first, lines)
    host_in = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    synth.generate_into(shape, first, lines, host_in.data_ptr(), nbytes)
    x = host_in.to(dev)

    comp = torch.empty(zs.zs_compress_bound(nbytes), dtype=torch.uint8, device=dev)
    idx = torch.empty(lines + 2, dtype=torch.int64, device=dev)
    dec = torch.empty(d.decompress_bound(nbytes) // 2 + nbytes, dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(1000 + rank)
    ids_host = torch.from_numpy(rng.integers(0, lines, size=RA_IDS).astype(np.int64)).pin_memory()
    ids = ids_host.to(dev)
    ra_out = torch.empty(RA_IDS * 256, dtype=torch.uint8, device=dev)
    ra_off = torch.empty(RA_IDS + 1, dtype=torch.int64, device=dev)
    stream = torch.cuda.current_stream(dev)

    kms = {"compress": [], "decompress": [], "lines": []}
    sizes = {}

    def step(record=True):
        r = zs.zs_compress(d, x, zs.PREPROCESS, comp, idx)
        kc = zs.zs_last_kernel_ms()
        c = comp[: r.out_len]
        rd = zs.zs_decompress(d, c, dec)
        kd = zs.zs_last_kernel_ms()
        rl = zs.zs_decompress_lines(d, c, idx[: r.n_lines + 1], ids, ra_out, ra_off)
        kl = zs.zs_last_kernel_ms()
        if record:
            kms["compress"].append(kc)
            kms["decompress"].append(kd)
            kms["lines"].append(kl)
        sizes.update(comp=r.out_len, n_lines=r.n_lines, dec=rd.out_len, ra=rl.out_len)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(max(3, args.warmup)):
        step(record=False)
    assert sizes["n_lines"] == lines and sizes["dec"] >= nbytes * 0.9

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

    # ---- end to end through the host-buffer API: every step compresses the pinned host input into pinned host
    # buffers (zs_compress_host: copies in, kernels and copies out overlapped chunk by chunk), decompresses that
    # host result (zs_decompress_host), and answers the 100,000-id request from host ids into host memory
    # against the device-resident store (ids H2D, zs_decompress_lines, lines and offsets D2H) ----
    host_comp = torch.empty(comp.numel(), dtype=torch.uint8, pin_memory=True)
    host_idx = torch.empty(idx.numel(), dtype=torch.int64, pin_memory=True)
    host_dec = torch.empty(dec.numel(), dtype=torch.uint8, pin_memory=True)
    host_ra = torch.empty(ra_out.numel(), dtype=torch.uint8, pin_memory=True)
    host_off = torch.empty(ra_off.numel(), dtype=torch.int64, pin_memory=True)
    e2e_steps = max(1, min(args.steps, args.e2e_steps))
    r0 = zs.zs_compress(d, x, zs.PREPROCESS, comp, idx)  # the resident store random access reads
    store, store_idx = comp[: r0.out_len], idx[: r0.n_lines + 1]
    # ---- the line index rebuilt from the compressed stream alone (zs_build_line_index), checked against the
    # index the compressor wrote; outside the timed step ----
    idx2 = torch.empty(idx.numel(), dtype=torch.int64, device=dev)
    li_ms = []
    for k in range(6):
        n_li = zs.zs_build_line_index(store, idx2)
        if k:
            li_ms.append(zs.zs_last_kernel_ms())
    li_same = n_li == r0.n_lines and torch.equal(idx2[: n_li + 1], store_idx)
    del idx2
    io = {}

    def e2e_step():
        r = zs.zs_compress_host(d, host_in, zs.PREPROCESS, host_comp, host_idx)
        rd = zs.zs_decompress_host(d, host_comp[: r.out_len], host_dec)
        ids.copy_(ids_host, non_blocking=True)
        rl = zs.zs_decompress_lines(d, store, store_idx, ids, ra_out, ra_off)
        host_ra[: rl.out_len].copy_(ra_out[: rl.out_len], non_blocking=True)
        host_off.copy_(ra_off, non_blocking=True)
        torch.cuda.synchronize(dev)
        io.update(h2d=nbytes + r.out_len + ids_host.numel() * 8,
                  d2h=r.out_len + (r.n_lines + 1) * 8 + rd.out_len + rl.out_len + ra_off.numel() * 8)

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
    h2d, d2h = io["h2d"], io["d2h"]

    (ms_step, e2e_ms), (total_bytes,) = reduce_over_ranks([ms_total / args.steps, e2e_ms], [nbytes], dev)

    value = total_bytes / (ms_step * 1e-3) / 1e9
    peak, peak_kind = hbm_peak()
    kc = float(np.mean(kms["compress"]))
    kd = float(np.mean(kms["decompress"]))
    kl = float(np.mean(kms["lines"]))
    li_k = float(np.median(li_ms))
    li_alg = sizes["comp"] + 8 * (sizes["n_lines"] + 1)  # read the stream, write n_lines + 1 offsets
    comp_bytes = nbytes + sizes["comp"] + 8 * (sizes["n_lines"] + 1)   # read input, write output + index
    dec_bytes = sizes["comp"] + sizes["dec"]                            # read compressed, write decoded
    achieved_c = comp_bytes / (kc * 1e-3) / 1e9
    achieved_d = dec_bytes / (kd * 1e-3) / 1e9
    traffic = kernel_traffic("compress_warp_kernel")

    if rank == 0:
        line = {
            "metric": metric_name(), "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
            "data": "synthetic",
            "config": {"workload": workload_desc(lines, nbytes), "lines_per_rank": lines,
                       "bytes_per_rank": nbytes, "dictionary": "frozen default (Algorithm 1, seed-1 100k-line "
                                                               "training set, L_max 8, T 146)",
                       "dictionary_sha256": hashlib.sha256(open(zs.DEFAULT_DICTIONARY, "rb").read()).hexdigest(),
                       "step": f"zs_compress + zs_decompress + zs_decompress_lines({RA_IDS:,} random ids)",
                       "l2": "inputs (and outputs) larger than the 129 MB L2; no flush",
                       "parallelism": f"{world} independent replica(s)"},
            "clocks": clocks.summary(),
            "e2e": {"value": total_bytes / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms,
                    "how": "wall clock per step of zs_compress_host (pinned host input to pinned host stream and "
                           "index) + zs_decompress_host (that host stream to pinned host text) + 100,000 random "
                           "ids H2D, zs_decompress_lines on the device-resident store, lines and offsets D2H"},
            "gpu_launches": 3 * args.steps,
            "roofline": {"bound": "hbm", "achieved": achieved_c, "peak": peak, "unit": "GB/s",
                         "frac": achieved_c / peak, "traffic": traffic, "kernel": "compress_warp_kernel",
                         "peak_kind": f"{peak_kind} (copy, MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                         else "fallback 6.8 TB/s",
                         "algorithmic_bytes_per_launch": comp_bytes, "kernel_ms": kc},
            "compress": {"kernel_ms": kc, "gbps_in": nbytes / (kc * 1e-3) / 1e9,
                         "lines_per_s": lines / (kc * 1e-3), "hbm_gbps": achieved_c, "hbm_frac": achieved_c / peak,
                         "hbm_frac_nominal": achieved_c / HBM_NOMINAL_GBS, "ratio": sizes["comp"] / nbytes},
            "decompress": {"kernel_ms": kd, "gbps_in": sizes["comp"] / (kd * 1e-3) / 1e9,
                           "gbps_out": sizes["dec"] / (kd * 1e-3) / 1e9, "hbm_gbps": achieved_d,
                           "hbm_frac": achieved_d / peak, "hbm_frac_nominal": achieved_d / HBM_NOMINAL_GBS},
            "line_index": {"kernel_ms": li_k, "gbps_in": sizes["comp"] / (li_k * 1e-3) / 1e9,
                           "hbm_gbps": li_alg / (li_k * 1e-3) / 1e9, "hbm_frac": li_alg / (li_k * 1e-3) / 1e9 / peak,
                           "identical_to_compress_index": bool(li_same)},
            "random_access": {"ids": RA_IDS, "kernel_ms": kl, "lines_per_s": RA_IDS / (kl * 1e-3),
                              "p50_ms": float(np.percentile(kms["lines"], 50)),
                              "p99_ms": float(np.percentile(kms["lines"], 99))},
        }
        if world == 1 and not args.no_batched:
            line["batched"] = bench_batched(zs, d, dev, reps=5, peak=peak)
        if world == 1 and not args.no_serving:
            line["serving"] = bench_serving(zs, d, dev, args.serve_lines, args.serve_requests,
                                            [int(r) for r in args.serve_rates.split(",")])
        if not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args.cpu_sample_lines, shape)
            line["cpu_oracle_cfg0"] = {t: cpu_baseline(synth.CFG0_LINES, synth.CFG0, threads=n,
                                                       stream="the 10,000-line config-0 stream")
                                       for t, n in (("single_thread", 1), ("all_threads", None))}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lines", type=int, default=synth.CFG1_LINES)
    ap.add_argument("--e2e-steps", type=int, default=40)
    ap.add_argument("--cpu-sample-lines", type=int, default=synth.CFG1_LINES)
    ap.add_argument("--ref-sample-lines", type=int, default=400_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-shard batched-form comparison")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving-form request replay")
    ap.add_argument("--serve-lines", type=int, default=synth.CFG4_LINES)
    ap.add_argument("--serve-requests", type=int, default=300)
    ap.add_argument("--serve-rates", default="1000,10000,100000")
    ap.add_argument("--ablation", action="store_true",
                    help="instead of the benchmark line: ratio and kernel times of the ablation dictionaries")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.ablation:
        run_ablation(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
