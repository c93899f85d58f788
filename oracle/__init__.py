"""ZSMILES CPU oracle (TEST INFRASTRUCTURE ONLY).

A plain, single-threaded restatement of the ZSMILES codec of arXiv 2404.19391 (pre-processing,
Sec. IV-A; shortest-output compression, Sec. IV-D1; table-lookup decompression, Sec. IV-D2; line
separability, Sec. I) in C (``zs_oracle.c``), plus the dictionary-generation procedure (Algorithm 1,
Eq. 1) in Python (``dictgen.py``). Only the tests, the smoke check and the benchmark's CPU-baseline leg
may import it. It shares no code with the CUDA library, and the CUDA library never calls it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID_ARG, ERR_BAD_DICT, ERR_CAPACITY, ERR_MALFORMED = 0, 1, 2, 3, 4
PREPROCESS = 1
PREPROCESS_OUTER = 2  # with PREPROCESS: label rings in opening order (the other reading of Sec. IV-A)


class OracleError(RuntimeError):
    def __init__(self, status: int, where: int | None = None):
        super().__init__(f"oracle status {status} at {where}")
        self.status = status
        self.where = where


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "zs_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", src, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            vp, sz, u = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint
            psz = ctypes.POINTER(ctypes.c_size_t)
            sig = {
                "oz_dict_size": (sz, []),
                "oz_dict_parse": (ctypes.c_int, [vp, sz, vp]),
                "oz_dict_lmax": (ctypes.c_int, [vp]),
                "oz_dict_entries": (ctypes.c_int, [vp]),
                "oz_preprocess_line": (sz, [vp, sz, vp]),
                "oz_preprocess_line_ex": (sz, [vp, sz, vp, ctypes.c_int]),
                "oz_compress_line": (sz, [vp, vp, sz, vp]),
                "oz_parse_cost": (sz, [vp, vp, sz]),
                "oz_decompress_line": (ctypes.c_int, [vp, vp, sz, vp, psz, psz]),
                "oz_count_lines": (sz, [vp, sz]),
                "oz_line_index": (sz, [vp, sz, vp]),
                "oz_preprocess_stream": (ctypes.c_int, [vp, sz, vp, sz, psz]),
                "oz_preprocess_stream_ex": (ctypes.c_int, [vp, sz, ctypes.c_int, vp, sz, psz]),
                "oz_compress_stream": (ctypes.c_int, [vp, vp, sz, u, vp, sz, vp, psz, psz]),
                "oz_decompress_stream": (ctypes.c_int, [vp, vp, sz, vp, sz, psz, psz]),
                "oz_decompress_lines": (ctypes.c_int, [vp, vp, sz, vp, sz, vp, sz, vp, sz, vp, psz, psz]),
            }
            for name, (res, args) in sig.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _buf(data) -> tuple[np.ndarray, int]:
    a = np.frombuffer(data, dtype=np.uint8) if isinstance(data, (bytes, bytearray, memoryview)) \
        else np.ascontiguousarray(data, dtype=np.uint8)
    return a, (a.ctypes.data if a.size else 0)


class Dict:
    """A parsed dictionary file (the .zsd text format)."""

    def __init__(self, file_bytes: bytes):
        L = _L()
        self._mem = ctypes.create_string_buffer(L.oz_dict_size())
        src = np.frombuffer(bytes(file_bytes), dtype=np.uint8)
        st = L.oz_dict_parse(src.ctypes.data if src.size else None, src.size, self._mem)
        if st != OK:
            raise OracleError(st)
        self.lmax = L.oz_dict_lmax(self._mem)
        self.entries = L.oz_dict_entries(self._mem)

    @property
    def ptr(self):
        return ctypes.cast(self._mem, ctypes.c_void_p)


def preprocess_line(line: bytes, outer: bool = False) -> bytes:
    """Ring-ID pre-processing of one line (Sec. IV-A); outer=True takes the opening-order reading."""
    out = ctypes.create_string_buffer(3 * len(line) + 1)
    n = _L().oz_preprocess_line_ex(line, len(line), out, int(bool(outer)))
    return out.raw[:n]


def compress_line(d: Dict, line: bytes) -> bytes:
    out = ctypes.create_string_buffer(2 * len(line) + 1)
    n = _L().oz_compress_line(d.ptr, line, len(line), out)
    return out.raw[:n]


def parse_cost(d: Dict, line: bytes) -> int:
    return int(_L().oz_parse_cost(d.ptr, line, len(line)))


def decompress_line(d: Dict, comp: bytes) -> bytes:
    out = ctypes.create_string_buffer(d.lmax * len(comp) + 1)
    n, e = ctypes.c_size_t(0), ctypes.c_size_t(0)
    st = _L().oz_decompress_line(d.ptr, comp, len(comp), out, ctypes.byref(n), ctypes.byref(e))
    if st != OK:
        raise OracleError(st, e.value)
    return out.raw[: n.value]


def count_lines(data) -> int:
    a, p = _buf(data)
    return int(_L().oz_count_lines(p, a.size))


def line_index(data) -> np.ndarray:
    a, p = _buf(data)
    n = int(_L().oz_line_index(p, a.size, None))
    idx = np.empty(n + 1, dtype=np.uint64)
    _L().oz_line_index(p, a.size, idx.ctypes.data)
    return idx


def preprocess_stream(data, outer: bool = False) -> np.ndarray:
    a, p = _buf(data)
    out = np.empty(3 * a.size + 16, dtype=np.uint8)
    n = ctypes.c_size_t(0)
    st = _L().oz_preprocess_stream_ex(p, a.size, int(bool(outer)), out.ctypes.data, out.size, ctypes.byref(n))
    if st != OK:
        raise OracleError(st)
    return out[: n.value].copy()


def compress_stream(d: Dict, data, flags: int = PREPROCESS):
    """Returns (compressed bytes, uint64 line index [n_lines+1])."""
    a, p = _buf(data)
    out = np.empty(2 * 3 * a.size + 16, dtype=np.uint8)
    nl = count_lines(a)
    idx = np.empty(nl + 1, dtype=np.uint64)
    n, k = ctypes.c_size_t(0), ctypes.c_size_t(0)
    st = _L().oz_compress_stream(d.ptr, p, a.size, flags, out.ctypes.data, out.size, idx.ctypes.data,
                                 ctypes.byref(n), ctypes.byref(k))
    if st != OK:
        raise OracleError(st)
    assert k.value == nl
    return out[: n.value].copy(), idx


def decompress_stream(d: Dict, data) -> np.ndarray:
    a, p = _buf(data)
    out = np.empty(d.lmax * a.size + 16, dtype=np.uint8)
    n, e = ctypes.c_size_t(0), ctypes.c_size_t(0)
    st = _L().oz_decompress_stream(d.ptr, p, a.size, out.ctypes.data, out.size, ctypes.byref(n), ctypes.byref(e))
    if st != OK:
        raise OracleError(st, e.value)
    return out[: n.value].copy()


def decompress_lines(d: Dict, comp, index: np.ndarray, ids: np.ndarray):
    """Returns (decoded lines, each '\\n'-terminated, uint64 out_off [k+1])."""
    a, p = _buf(comp)
    index = np.ascontiguousarray(index, dtype=np.uint64)
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    n_lines = index.size - 1
    spans = [int(index[i + 1] - index[i]) for i in ids if i < n_lines]
    cap = d.lmax * sum(spans) + ids.size + 16
    out = np.empty(cap, dtype=np.uint8)
    off = np.empty(ids.size + 1, dtype=np.uint64)
    n, e = ctypes.c_size_t(0), ctypes.c_size_t(0)
    st = _L().oz_decompress_lines(d.ptr, p, a.size, index.ctypes.data, n_lines,
                                  ids.ctypes.data if ids.size else None, ids.size,
                                  out.ctypes.data, out.size, off.ctypes.data, ctypes.byref(n), ctypes.byref(e))
    if st != OK:
        raise OracleError(st, e.value)
    return out[: n.value].copy(), off


def split_at_lines(a: np.ndarray, parts: int) -> list[tuple[int, int]]:
    """Cut [0, len) into <= parts ranges that end just after a '\\n' (or at the end)."""
    n = a.size
    cuts = [0]
    for k in range(1, parts):
        c = max(cuts[-1], (n * k) // parts)
        nl = np.flatnonzero(a[c:] == 10)
        c = n if nl.size == 0 else c + int(nl[0]) + 1
        if c > cuts[-1]:
            cuts.append(c)
    if cuts[-1] != n:
        cuts.append(n)
    return [(cuts[i], cuts[i + 1]) for i in range(len(cuts) - 1)]


def compress_stream_parallel(d: Dict, data, flags: int = PREPROCESS, threads: int | None = None):
    """The same single-threaded oracle run line-partitioned over host threads (the C calls release
    the GIL); results are concatenated exactly as one call over the whole stream would produce."""
    a, _ = _buf(data)
    threads = threads or (os.cpu_count() or 1)
    ranges = split_at_lines(a, threads)
    if len(ranges) <= 1:
        return compress_stream(d, a, flags)
    with ThreadPoolExecutor(len(ranges)) as ex:
        parts = list(ex.map(lambda r: compress_stream(d, a[r[0]:r[1]], flags), ranges))
    outs, idxs, base = [], [], 0
    for out, idx in parts:
        outs.append(out)
        idxs.append(idx[:-1] + np.uint64(base))
        base += out.size
    return np.concatenate(outs), np.concatenate(idxs + [np.array([base], dtype=np.uint64)])


def decompress_stream_parallel(d: Dict, data, threads: int | None = None) -> np.ndarray:
    a, _ = _buf(data)
    threads = threads or (os.cpu_count() or 1)
    ranges = split_at_lines(a, threads)
    if len(ranges) <= 1:
        return decompress_stream(d, a)
    with ThreadPoolExecutor(len(ranges)) as ex:
        parts = list(ex.map(lambda r: decompress_stream(d, a[r[0]:r[1]]), ranges))
    return np.concatenate(parts)


def preprocess_stream_parallel(data, threads: int | None = None, outer: bool = False) -> np.ndarray:
    a, _ = _buf(data)
    threads = threads or (os.cpu_count() or 1)
    ranges = split_at_lines(a, threads)
    if len(ranges) <= 1:
        return preprocess_stream(a, outer)
    with ThreadPoolExecutor(len(ranges)) as ex:
        parts = list(ex.map(lambda r: preprocess_stream(a[r[0]:r[1]], outer), ranges))
    return np.concatenate(parts)
