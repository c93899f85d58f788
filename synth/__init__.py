"""Seeded synthetic SMILES-like inputs shared by the CPU oracle and the CUDA path.

The generator itself is C (``gen.c``), built on first use with the host compiler. It holds none of the
codec's arithmetic. Workload presets follow the library shapes the paper evaluates on (Section V-A:
drug-like lines; macrocycle/peptide-like long lines), sized as the benchmark workloads.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libsynth.so")
_lock = threading.Lock()
_lib = None


class _Params(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("len_mean_milli", ctypes.c_int32),
        ("len_sd_milli", ctypes.c_int32),
        ("len_lo", ctypes.c_int32),
        ("len_hi", ctypes.c_int32),
        ("p_long16", ctypes.c_uint32),
        ("long_lo", ctypes.c_int32),
        ("long_hi", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile gen.c into _build/libsynth.so (integer-only C, portable across x86_64 and aarch64)."""
    src = os.path.join(_HERE, "gen.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
                               "-ffp-contract=off", src, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.synth_lines_mt.restype = ctypes.c_size_t
            lib.synth_lines_mt.argtypes = [ctypes.POINTER(_Params), ctypes.c_uint64, ctypes.c_uint64,
                                           ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t]
            lib.synth_u32.restype = None
            lib.synth_u32.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_void_p]
            _lib = lib
    return _lib


@dataclass(frozen=True)
class LineShape:
    """Distribution of one stream's lines."""
    seed: int
    len_mean: float = 45.0
    len_sd: float = 12.0
    len_lo: int = 15
    len_hi: int = 120
    p_long: float = 0.0
    long_lo: int = 150
    long_hi: int = 400

    def _c(self) -> _Params:
        return _Params(self.seed, int(round(self.len_mean * 1000)), int(round(self.len_sd * 1000)),
                       self.len_lo, self.len_hi, int(round(self.p_long * 65536)), self.long_lo, self.long_hi)


def _threads(n: int | None) -> int:
    return n if n else max(1, min(64, os.cpu_count() or 1))


def lines_size(shape: LineShape, first: int, count: int, nthreads: int | None = None) -> int:
    p = shape._c()
    return int(_load().synth_lines_mt(ctypes.byref(p), first, count, _threads(nthreads), None, 0))


def generate_into(shape: LineShape, first: int, count: int, out_ptr: int, cap: int,
                  nthreads: int | None = None) -> int:
    """Write lines [first, first+count) ('\\n'-terminated) at address out_ptr; returns the byte count."""
    p = shape._c()
    n = _load().synth_lines_mt(ctypes.byref(p), first, count, _threads(nthreads), ctypes.c_void_p(out_ptr), cap)
    if n == ctypes.c_size_t(-1).value:
        raise ValueError("synth: output capacity too small")
    return int(n)


def generate(shape: LineShape, first: int = 0, count: int = 1, nthreads: int | None = None) -> np.ndarray:
    """Lines [first, first+count) of the seeded stream as a uint8 array, each line '\\n'-terminated."""
    size = lines_size(shape, first, count, nthreads)
    buf = np.empty(size, dtype=np.uint8)
    if size:
        generate_into(shape, first, count, buf.ctypes.data, size, nthreads)
    return buf


def uniform_u32(seed: int, index0: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.uint32)
    if n:
        _load().synth_u32(seed, index0, n, out.ctypes.data)
    return out


# ---- workload presets -------------------------------------------------------------------------------

#: small plain stream: 10,000 drug-like lines, mean 45 chars (sd 12, clipped to 15-120)
CFG0 = LineShape(seed=0)
#: dictionary training set: 100,000 lines of the same distribution, separate seed
TRAIN = LineShape(seed=1)
CFG0_LINES = 10_000
TRAIN_LINES = 100_000
#: large single stream: 10M lines of the same distribution
CFG1 = LineShape(seed=2)
CFG1_LINES = 10_000_000
#: long-tail stream: 100M lines, 10% long (150-400 chars, wide bracket set, stereo bonds, %nn rings)
CFG3 = LineShape(seed=4, p_long=0.10)
CFG3_LINES = 100_000_000
#: serving store: 50M lines of the small-stream distribution
CFG4 = LineShape(seed=5)
CFG4_LINES = 50_000_000
CFG2_SEED = 3
CFG2_SHARDS = 64


def batched_shards(n_shards: int = CFG2_SHARDS, seed: int = CFG2_SEED,
                   count_lo: int = 1_000, count_hi: int = 5_000_000) -> list[tuple[LineShape, int]]:
    """Shard table of the batched workload: line counts log-uniform in [count_lo, count_hi]; per-shard
    mean length mu ~ U[25, 70], length ~ N(mu, 0.267 mu) clipped to [mu/3, 8 mu/3]."""
    u = uniform_u32(seed, 0, 2 * n_shards).astype(np.float64) / 2.0 ** 32
    shards = []
    for s in range(n_shards):
        count = int(math.floor(count_lo * (count_hi / count_lo) ** u[2 * s]))
        mu = 25.0 + 45.0 * u[2 * s + 1]
        shape = LineShape(seed=seed * 1000 + s + 1, len_mean=round(mu, 3), len_sd=round(0.267 * mu, 3),
                          len_lo=max(1, int(mu / 3)), len_hi=int(8 * mu / 3))
        shards.append((shape, count))
    return shards


def requests(n: int, seed: int, n_lines: int, max_ids: int = 100_000, rate: float = 1000.0):
    """Serving request stream: Poisson arrivals at `rate` req/s; each request asks for a log-uniform
    number of ids in [1, max_ids], drawn uniformly without replacement from [0, n_lines)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    arrivals = np.cumsum(gaps) - gaps[0]
    sizes = np.floor(np.exp(rng.uniform(0.0, math.log(max_ids + 1), size=n))).astype(np.int64)
    sizes = np.clip(sizes, 1, min(max_ids, n_lines))
    reqs = []
    for k in range(n):
        ids = rng.choice(n_lines, size=int(sizes[k]), replace=False) if sizes[k] < n_lines // 4 \
            else rng.permutation(n_lines)[: int(sizes[k])]
        reqs.append((float(arrivals[k]), ids.astype(np.uint64)))
    return reqs
