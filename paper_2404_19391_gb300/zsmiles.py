"""Python binding of libzsmiles.so (the ZSMILES C ABI, include/zsmiles.h).

Argument marshalling only: every step of compression, decompression, indexing and random access runs in
the library's CUDA kernels. Device buffers are torch CUDA tensors (uint8 / int64 views of uint64 data);
streams are torch.cuda streams (default: the current stream). There is no CPU fallback: importing this
module on a machine where the library cannot be loaded raises.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

from . import build as _build

OK, ERR_INVALID_ARG, ERR_BAD_DICT, ERR_CAPACITY, ERR_MALFORMED, ERR_CUDA, ERR_TIMEOUT, ERR_OOM = range(8)
STATUS_NAMES = ["ZS_OK", "ZS_ERR_INVALID_ARG", "ZS_ERR_BAD_DICT", "ZS_ERR_CAPACITY", "ZS_ERR_MALFORMED",
                "ZS_ERR_CUDA", "ZS_ERR_TIMEOUT", "ZS_ERR_OOM"]
PREPROCESS = 1
PREPROCESS_OUTER = 2  # with PREPROCESS: rings labelled in opening order (the other reading of Sec. IV-A)

DEFAULT_DICTIONARY = os.path.join(os.path.dirname(os.path.abspath(__file__)), "data", "zs_default.zsd")


class ZsError(RuntimeError):
    def __init__(self, status: int, message: str, result: "Result | None" = None):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {message}")
        self.status = status
        self.result = result


class _Result(ctypes.Structure):
    _fields_ = [("out_len", ctypes.c_uint64), ("n_lines", ctypes.c_uint64), ("err_offset", ctypes.c_uint64)]


class _Shard(ctypes.Structure):
    _fields_ = [("in_", ctypes.c_void_p), ("in_len", ctypes.c_size_t), ("out", ctypes.c_void_p),
                ("out_cap", ctypes.c_size_t), ("line_index", ctypes.c_void_p), ("index_cap", ctypes.c_size_t)]


class _PlanOptions(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int), ("use_graph", ctypes.c_int), ("tune_reps", ctypes.c_int),
                ("cut_min", ctypes.c_int), ("tune_cache", ctypes.c_int)]


class _ServerOptions(ctypes.Structure):
    _fields_ = [("arena_bytes", ctypes.c_size_t), ("max_batch_ids", ctypes.c_size_t), ("max_inflight", ctypes.c_int)]


class _ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("ids", ctypes.c_uint64), ("mean_batch_requests", ctypes.c_double), ("max_inflight", ctypes.c_int),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double)]


class _PipelineOptions(ctypes.Structure):
    _fields_ = [("chunk_bytes", ctypes.c_size_t), ("n_streams", ctypes.c_int)]


class _TrainOptions(ctypes.Structure):
    _fields_ = [("lmin", ctypes.c_int), ("lmax", ctypes.c_int), ("T", ctypes.c_int), ("no_alphabet", ctypes.c_int)]


OP_COMPRESS, OP_DECOMPRESS = 0, 1


@dataclass
class Result:
    out_len: int
    n_lines: int
    err_offset: int


_lib = None


def library_path() -> str:
    return _build.LIB


def load_library(rebuild: bool = False) -> ctypes.CDLL:
    """Load (building first if needed) the in-tree libzsmiles.so."""
    global _lib
    if _lib is not None and not rebuild:
        return _lib
    path = os.environ.get("ZS_LIBRARY") or (_build.build() if (rebuild or not os.path.exists(_build.LIB))
                                             else _build.LIB)
    lib = ctypes.CDLL(path)
    vp, sz, u64 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_uint64
    pres = ctypes.POINTER(_Result)
    sig = {
        "zs_load_dictionary": (ctypes.c_int, [vp, sz, ctypes.POINTER(vp)]),
        "zs_free_dictionary": (None, [vp]),
        "zs_dictionary_lmax": (ctypes.c_int, [vp]),
        "zs_compress_bound": (sz, [sz]),
        "zs_decompress_bound": (sz, [vp, sz]),
        "zs_compress": (ctypes.c_int, [vp, vp, sz, ctypes.c_uint, vp, sz, vp, sz, pres, vp]),
        "zs_decompress": (ctypes.c_int, [vp, vp, sz, vp, sz, pres, vp]),
        "zs_build_line_index": (ctypes.c_int, [vp, sz, vp, sz, ctypes.POINTER(sz), vp]),
        "zs_decompress_lines": (ctypes.c_int, [vp, vp, sz, vp, sz, vp, sz, vp, sz, vp, pres, vp]),
        "zs_last_error": (ctypes.c_char_p, []),
        "zs_version": (ctypes.c_char_p, []),
        "zs_last_kernel_ms": (ctypes.c_double, []),
        "zs_dictionary_uses_transducer": (ctypes.c_int, [vp]),
        "zs_kernel_variants": (ctypes.c_int, [ctypes.c_int]),
        "zs_kernel_variant_name": (ctypes.c_char_p, [ctypes.c_int, ctypes.c_int]),
        "zs_compress_batch": (ctypes.c_int, [vp, ctypes.POINTER(_Shard), sz, ctypes.c_uint, pres, vp]),
        "zs_decompress_batch": (ctypes.c_int, [vp, ctypes.POINTER(_Shard), sz, pres, vp]),
        "zs_plan_create": (ctypes.c_int, [vp, ctypes.c_int, ctypes.c_uint, ctypes.POINTER(_Shard), sz,
                                          ctypes.POINTER(_PlanOptions), ctypes.POINTER(vp)]),
        "zs_plan_run": (ctypes.c_int, [vp, pres, vp]),
        "zs_plan_variant": (ctypes.c_int, [vp]),
        "zs_plan_cut_min": (ctypes.c_int, [vp]),
        "zs_plan_tuned_ms": (ctypes.c_double, [vp, ctypes.c_int]),
        "zs_plan_last_ms": (ctypes.c_double, [vp]),
        "zs_plan_destroy": (None, [vp]),
        "zs_server_create": (ctypes.c_int, [vp, vp, sz, vp, sz, ctypes.POINTER(_ServerOptions), ctypes.POINTER(vp)]),
        "zs_server_submit": (ctypes.c_int, [vp, vp, sz, ctypes.POINTER(u64)]),
        "zs_server_wait": (ctypes.c_int, [vp, u64, ctypes.c_double, pres]),
        "zs_server_fetch": (ctypes.c_int, [vp, u64, vp, sz, vp]),
        "zs_server_release": (ctypes.c_int, [vp, u64]),
        "zs_server_get_stats": (ctypes.c_int, [vp, ctypes.POINTER(_ServerStats)]),
        "zs_server_destroy": (None, [vp]),
        "zs_server_replay": (ctypes.c_int, [vp, vp, vp, vp, sz, vp, ctypes.POINTER(ctypes.c_double)]),
        "zs_serial_replay": (ctypes.c_int, [vp, vp, sz, vp, sz, vp, vp, vp, sz, vp, ctypes.POINTER(ctypes.c_double),
                                            vp]),
        "zs_compress_host": (ctypes.c_int, [vp, vp, sz, ctypes.c_uint, vp, sz, vp, sz, pres,
                                            ctypes.POINTER(_PipelineOptions)]),
        "zs_decompress_host": (ctypes.c_int, [vp, vp, sz, vp, sz, pres, ctypes.POINTER(_PipelineOptions)]),
        "zs_train_dictionary": (ctypes.c_int, [vp, sz, ctypes.c_uint, ctypes.POINTER(_TrainOptions), vp, sz,
                                               ctypes.POINTER(sz), vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _L():
    return _lib if _lib is not None else load_library()


def _ptr(t: torch.Tensor | None) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr() if t.numel() else None


def _stream(stream) -> int | None:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream or None


def _check(st: int, res: _Result | None = None):
    if st != OK:
        r = Result(res.out_len, res.n_lines, res.err_offset) if res is not None else None
        raise ZsError(st, _L().zs_last_error().decode(), r)


def zs_version() -> str:
    return _L().zs_version().decode()


def zs_last_kernel_ms() -> float:
    return float(_L().zs_last_kernel_ms())


def zs_compress_bound(in_len: int) -> int:
    return int(_L().zs_compress_bound(in_len))


class Dictionary:
    """A loaded dictionary (zs_load_dictionary / zs_free_dictionary)."""

    def __init__(self, file_bytes: bytes | None = None, path: str | None = None):
        if file_bytes is None:
            with open(path or DEFAULT_DICTIONARY, "rb") as f:
                file_bytes = f.read()
        self._bytes = bytes(file_bytes)
        torch.cuda.init()
        h = ctypes.c_void_p()
        buf = ctypes.create_string_buffer(self._bytes, len(self._bytes))
        _check(_L().zs_load_dictionary(buf, len(self._bytes), ctypes.byref(h)))
        self.handle = h
        self.lmax = int(_L().zs_dictionary_lmax(h))

    def close(self):
        if getattr(self, "handle", None):
            _L().zs_free_dictionary(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def uses_transducer(self) -> bool:
        return bool(_L().zs_dictionary_uses_transducer(self.handle))

    def decompress_bound(self, in_len: int) -> int:
        return int(_L().zs_decompress_bound(self.handle, in_len))


def zs_load_dictionary(file_bytes: bytes) -> Dictionary:
    return Dictionary(file_bytes)


def zs_compress(d: Dictionary, d_in: torch.Tensor, flags: int, d_out: torch.Tensor,
                d_line_index: torch.Tensor | None = None, stream=None) -> Result:
    res = _Result()
    st = _L().zs_compress(d.handle, _ptr(d_in), d_in.numel(), flags, _ptr(d_out), d_out.numel(),
                          _ptr(d_line_index), 0 if d_line_index is None else d_line_index.numel(),
                          ctypes.byref(res), _stream(stream))
    _check(st, res)
    return Result(res.out_len, res.n_lines, res.err_offset)


def zs_decompress(d: Dictionary, d_in: torch.Tensor, d_out: torch.Tensor, stream=None) -> Result:
    res = _Result()
    st = _L().zs_decompress(d.handle, _ptr(d_in), d_in.numel(), _ptr(d_out), d_out.numel(), ctypes.byref(res),
                            _stream(stream))
    _check(st, res)
    return Result(res.out_len, res.n_lines, res.err_offset)


def zs_build_line_index(d_in: torch.Tensor, d_index: torch.Tensor, stream=None) -> int:
    n = ctypes.c_size_t(0)
    st = _L().zs_build_line_index(_ptr(d_in), d_in.numel(), _ptr(d_index), d_index.numel(), ctypes.byref(n),
                                  _stream(stream))
    if st != OK:
        raise ZsError(st, _L().zs_last_error().decode(), Result(0, n.value, 0))
    return int(n.value)


def zs_decompress_lines(d: Dictionary, d_comp: torch.Tensor, d_index: torch.Tensor, d_ids: torch.Tensor,
                        d_out: torch.Tensor, d_out_off: torch.Tensor, stream=None) -> Result:
    res = _Result()
    st = _L().zs_decompress_lines(d.handle, _ptr(d_comp), d_comp.numel(), _ptr(d_index), d_index.numel() - 1,
                                  _ptr(d_ids), d_ids.numel(), _ptr(d_out), d_out.numel(), _ptr(d_out_off),
                                  ctypes.byref(res), _stream(stream))
    _check(st, res)
    return Result(res.out_len, res.n_lines, res.err_offset)


def _shards(shards) -> "ctypes.Array":
    """shards: sequence of (in, out, line_index or None) CUDA tensors."""
    arr = (_Shard * max(1, len(shards)))()
    for i, (src, dst, idx) in enumerate(shards):
        arr[i] = _Shard(_ptr(src), src.numel(), _ptr(dst), dst.numel(), _ptr(idx),
                        0 if idx is None else idx.numel())
    return arr


def _results(res_arr, n) -> list[Result]:
    return [Result(res_arr[i].out_len, res_arr[i].n_lines, res_arr[i].err_offset) for i in range(n)]


def zs_kernel_variants(op: int) -> int:
    return int(_L().zs_kernel_variants(op))


def zs_kernel_variant_name(op: int, v: int) -> str | None:
    r = _L().zs_kernel_variant_name(op, v)
    return r.decode() if r is not None else None


def zs_compress_batch(d: Dictionary, shards, flags: int = PREPROCESS, stream=None) -> list[Result]:
    arr = _shards(shards)
    res = (_Result * max(1, len(shards)))()
    st = _L().zs_compress_batch(d.handle, arr, len(shards), flags, res, _stream(stream))
    if st != OK:
        raise ZsError(st, _L().zs_last_error().decode())
    return _results(res, len(shards))


def zs_decompress_batch(d: Dictionary, shards, stream=None) -> list[Result]:
    arr = _shards(shards)
    res = (_Result * max(1, len(shards)))()
    st = _L().zs_decompress_batch(d.handle, arr, len(shards), res, _stream(stream))
    if st != OK:
        raise ZsError(st, _L().zs_last_error().decode())
    return _results(res, len(shards))


class Plan:
    """zs_plan_create / zs_plan_run / zs_plan_destroy over a fixed list of (in, out, index) tensors."""

    def __init__(self, d: Dictionary, op: int, shards, flags: int = PREPROCESS, variant: int = -1,
                 use_graph: bool = True, tune_reps: int = 3, cut_min: int = 0, tune_cache: bool = False):
        self._keep = list(shards)  # the tensors must outlive the plan
        self.n = len(shards)
        arr = _shards(shards)
        opt = _PlanOptions(variant, 1 if use_graph else 0, tune_reps, cut_min, 1 if tune_cache else 0)
        h = ctypes.c_void_p()
        _check(_L().zs_plan_create(d.handle, op, flags, arr, self.n, ctypes.byref(opt), ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None) -> list[Result]:
        res = (_Result * max(1, self.n))()
        st = _L().zs_plan_run(self.handle, res, _stream(stream))
        if st != OK:
            raise ZsError(st, _L().zs_last_error().decode())
        return _results(res, self.n)

    @property
    def variant(self) -> int:
        return int(_L().zs_plan_variant(self.handle))

    @property
    def cut_min(self) -> int:
        """The span cut threshold the plan runs with, in bytes (0: no cuts)."""
        return int(_L().zs_plan_cut_min(self.handle))

    def tuned_ms(self, v: int) -> float:
        return float(_L().zs_plan_tuned_ms(self.handle, v))

    @property
    def last_ms(self) -> float:
        return float(_L().zs_plan_last_ms(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            _L().zs_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _replay_arrays(requests):
    """requests: list of (arrival seconds, uint64 ids array). Returns the C arrays and the keep-alive list."""
    import numpy as np
    arr = np.ascontiguousarray([a for a, _ in requests], dtype=np.float64)
    ks = np.ascontiguousarray([len(ids) for _, ids in requests], dtype=np.uint64)
    ids = np.ascontiguousarray(np.concatenate([np.asarray(i, dtype=np.uint64) for _, i in requests])
                               if requests else np.zeros(1, np.uint64))
    lat = np.zeros(max(1, len(requests)), dtype=np.float64)
    return arr, ids, ks, lat


class Server:
    """zs_server_*: continuous-batching random access over a resident store (d_comp + d_index tensors)."""

    def __init__(self, d: Dictionary, d_comp: torch.Tensor, d_index: torch.Tensor, arena_bytes: int = 0,
                 max_batch_ids: int = 0, max_inflight: int = 0):
        self._keep = (d, d_comp, d_index)
        self.n_lines = d_index.numel() - 1
        opt = _ServerOptions(arena_bytes, max_batch_ids, max_inflight)
        h = ctypes.c_void_p()
        _check(_L().zs_server_create(d.handle, _ptr(d_comp), d_comp.numel(), _ptr(d_index), self.n_lines,
                                     ctypes.byref(opt), ctypes.byref(h)))
        self.handle = h

    def submit(self, ids) -> int:
        import numpy as np
        a = np.ascontiguousarray(ids, dtype=np.uint64)
        t = ctypes.c_uint64(0)
        _check(_L().zs_server_submit(self.handle, a.ctypes.data if a.size else None, a.size, ctypes.byref(t)))
        return int(t.value)

    def wait(self, ticket: int, timeout_s: float = -1.0) -> Result:
        res = _Result()
        st = _L().zs_server_wait(self.handle, ticket, timeout_s, ctypes.byref(res))
        if st != OK:
            raise ZsError(st, _L().zs_last_error().decode())
        return Result(res.out_len, res.n_lines, res.err_offset)

    def fetch(self, ticket: int):
        """Waits for the request and returns (bytes, uint64 offsets[k + 1])."""
        import numpy as np
        r = self.wait(ticket)
        out = np.empty(max(1, r.out_len), dtype=np.uint8)
        off = np.empty(r.n_lines + 1, dtype=np.uint64)
        _check(_L().zs_server_fetch(self.handle, ticket, out.ctypes.data, out.size, off.ctypes.data))
        return out[: r.out_len].tobytes(), off

    def release(self, ticket: int):
        _check(_L().zs_server_release(self.handle, ticket))

    def stats(self) -> dict:
        st = _ServerStats()
        _check(_L().zs_server_get_stats(self.handle, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in _ServerStats._fields_}

    def replay(self, requests):
        """Open-loop replay of [(arrival_s, ids)]; returns (latency_ms array, makespan_s)."""
        arr, ids, ks, lat = _replay_arrays(requests)
        mk = ctypes.c_double(0.0)
        st = _L().zs_server_replay(self.handle, arr.ctypes.data, ids.ctypes.data, ks.ctypes.data, len(requests),
                                   lat.ctypes.data, ctypes.byref(mk))
        if st != OK:
            raise ZsError(st, _L().zs_last_error().decode())
        return lat[: len(requests)], mk.value

    def close(self):
        if getattr(self, "handle", None):
            _L().zs_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def zs_serial_replay(d: Dictionary, d_comp: torch.Tensor, d_index: torch.Tensor, requests, stream=None):
    """Decompress-per-request baseline over the same open-loop arrivals; returns (latency_ms, makespan_s)."""
    arr, ids, ks, lat = _replay_arrays(requests)
    mk = ctypes.c_double(0.0)
    st = _L().zs_serial_replay(d.handle, _ptr(d_comp), d_comp.numel(), _ptr(d_index), d_index.numel() - 1,
                               arr.ctypes.data, ids.ctypes.data, ks.ctypes.data, len(requests), lat.ctypes.data,
                               ctypes.byref(mk), _stream(stream))
    if st != OK:
        raise ZsError(st, _L().zs_last_error().decode())
    return lat[: len(requests)], mk.value


def _host_ptr(t) -> tuple[int | None, int]:
    """(address, length) of a host buffer: a CPU torch tensor or a contiguous numpy array."""
    if isinstance(t, torch.Tensor):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError("expected a contiguous CPU tensor")
        return (t.data_ptr() if t.numel() else None), t.numel()
    if not t.flags["C_CONTIGUOUS"]:
        raise ValueError("expected a contiguous array")
    return (t.ctypes.data if t.size else None), t.size


def zs_compress_host(d: Dictionary, h_in, flags: int, h_out, h_line_index=None, chunk_bytes: int = 0,
                     n_streams: int = 0) -> Result:
    """Host buffers in and out (uint8 input/output, uint64/int64 index); pinned memory lets copies overlap."""
    pi, ni = _host_ptr(h_in)
    po, no = _host_ptr(h_out)
    px, nx = _host_ptr(h_line_index) if h_line_index is not None else (None, 0)
    opt = _PipelineOptions(chunk_bytes, n_streams)
    res = _Result()
    st = _L().zs_compress_host(d.handle, pi, ni, flags, po, no, px, nx, ctypes.byref(res), ctypes.byref(opt))
    _check(st, res)
    return Result(res.out_len, res.n_lines, res.err_offset)


def zs_decompress_host(d: Dictionary, h_in, h_out, chunk_bytes: int = 0, n_streams: int = 0) -> Result:
    pi, ni = _host_ptr(h_in)
    po, no = _host_ptr(h_out)
    opt = _PipelineOptions(chunk_bytes, n_streams)
    res = _Result()
    st = _L().zs_decompress_host(d.handle, pi, ni, po, no, ctypes.byref(res), ctypes.byref(opt))
    _check(st, res)
    return Result(res.out_len, res.n_lines, res.err_offset)


def zs_train_dictionary(d_train: torch.Tensor, flags: int = PREPROCESS, lmin: int = 2, lmax: int = 8, T: int = 0,
                        no_alphabet: bool = False, stream=None) -> bytes:
    """Algorithm 1 on a device training stream; returns the .zsd file bytes."""
    opt = _TrainOptions(lmin, lmax, T, 1 if no_alphabet else 0)
    cap = 1 << 16
    for _ in range(2):
        buf = ctypes.create_string_buffer(cap)
        n = ctypes.c_size_t(0)
        st = _L().zs_train_dictionary(_ptr(d_train), d_train.numel(), flags, ctypes.byref(opt), buf, cap,
                                      ctypes.byref(n), _stream(stream))
        if st == ERR_CAPACITY:
            cap = n.value
            continue
        _check(st)
        return buf.raw[: n.value]
    raise ZsError(ERR_CAPACITY, "dictionary text did not fit")


# ---- conveniences built only from the calls above ----------------------------------------------------

def compress(d: Dictionary, d_in: torch.Tensor, flags: int = PREPROCESS, with_index: bool = True, stream=None):
    """Compress a device byte tensor; returns (compressed bytes, line index or None, Result).

    The index buffer starts from a guess (one line per 24 input bytes) and is resized from the call's own
    ZS_ERR_CAPACITY answer (res.n_lines) when the guess is short, so no extra device pass sizes it."""
    out = torch.empty(zs_compress_bound(d_in.numel()), dtype=torch.uint8, device=d_in.device)
    idx = None
    if with_index:
        idx = torch.empty(d_in.numel() // 24 + 2, dtype=torch.int64, device=d_in.device)
    try:
        r = zs_compress(d, d_in, flags, out, idx, stream)
    except ZsError as e:
        if e.status != ERR_CAPACITY or idx is None or e.result is None or e.result.n_lines + 1 <= idx.numel():
            raise
        idx = torch.empty(e.result.n_lines + 1, dtype=torch.int64, device=d_in.device)
        r = zs_compress(d, d_in, flags, out, idx, stream)
    return out[: r.out_len], (idx[: r.n_lines + 1] if idx is not None else None), r


def decompress(d: Dictionary, d_in: torch.Tensor, stream=None):
    out = torch.empty(max(1, d.decompress_bound(d_in.numel())), dtype=torch.uint8, device=d_in.device)
    r = zs_decompress(d, d_in, out, stream)
    return out[: r.out_len], r


def line_index(d_in: torch.Tensor, stream=None) -> torch.Tensor:
    """Line index of a device stream, sized from zs_build_line_index's own answer on ZS_ERR_CAPACITY."""
    idx = torch.empty(d_in.numel() // 16 + 2, dtype=torch.int64, device=d_in.device)
    try:
        n = zs_build_line_index(d_in, idx, stream)
    except ZsError as e:
        if e.status != ERR_CAPACITY or e.result is None:
            raise
        idx = torch.empty(e.result.n_lines + 1, dtype=torch.int64, device=d_in.device)
        n = zs_build_line_index(d_in, idx, stream)
    return idx[: n + 1]


def decompress_lines(d: Dictionary, d_comp: torch.Tensor, d_index: torch.Tensor, d_ids: torch.Tensor,
                     out_cap: int | None = None, stream=None):
    """Random access with the output sized by the call itself: a first guess, then the exact size that
    zs_decompress_lines reports (res.out_len) on ZS_ERR_CAPACITY."""
    guess = out_cap if out_cap is not None else 64 * d_ids.numel() + 64
    out = torch.empty(max(1, guess), dtype=torch.uint8, device=d_comp.device)
    off = torch.empty(d_ids.numel() + 1, dtype=torch.int64, device=d_comp.device)
    try:
        r = zs_decompress_lines(d, d_comp, d_index, d_ids, out, off, stream)
    except ZsError as e:
        if out_cap is not None or e.status != ERR_CAPACITY or e.result is None:
            raise
        out = torch.empty(max(1, e.result.out_len), dtype=torch.uint8, device=d_comp.device)
        r = zs_decompress_lines(d, d_comp, d_index, d_ids, out, off, stream)
    return out[: r.out_len], off, r
