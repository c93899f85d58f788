"""zs_decompress_noalloc: the allocation-free decode entry point, checked against zs_decompress.

It serves callers that cannot let the library allocate (device memory held by another allocator, or
loops where cudaMalloc/cudaFree would synchronise the device). It must give exactly the bytes
zs_decompress gives (byte codec: exact equality), on two calls in a row (its fixed scratch keeps the
previous call's contents), and refuse inputs larger than its fixed scratch allows. This file runs last.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_INPUT = 262142 * 2048  # tile records in the 8 MiB scratch x compressed bytes per tile


class _Result(ctypes.Structure):
    _fields_ = [("out_len", ctypes.c_uint64), ("n_lines", ctypes.c_uint64), ("err_offset", ctypes.c_uint64)]


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19391_gb300 import zsmiles as zs
    lib = zs.load_library()
    f = lib.zs_decompress_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_size_t,
                  ctypes.POINTER(_Result), ctypes.c_void_p]
    lib.zs_decompress_noalloc_limit.restype = ctypes.c_size_t
    assert lib.zs_decompress_noalloc_limit() == MAX_INPUT
    return zs, lib, zs.Dictionary()


def _noalloc(env, comp, out):
    zs, lib, d = env
    r = _Result()
    st = lib.zs_decompress_noalloc(d.handle, comp.data_ptr(), comp.numel(), out.data_ptr(), out.numel(),
                                   ctypes.byref(r), torch.cuda.current_stream().cuda_stream or None)
    return st, r


def test_matches_zs_decompress_two_calls_in_a_row(env):
    zs, lib, d = env
    streams = [synth.generate(synth.CFG0, 0, 20000), synth.generate(synth.CFG3, 0, 8000)]
    for raw in streams:
        comp, _, _ = zs.compress(d, torch.from_numpy(raw).cuda(), with_index=False)
        comp = comp.clone()
        ref = torch.empty(d.decompress_bound(comp.numel()), dtype=torch.uint8, device="cuda")
        rr = zs.zs_decompress(d, comp, ref)
        for _ in range(2):
            out = torch.full((d.decompress_bound(comp.numel()),), 0xAB, dtype=torch.uint8, device="cuda")
            st, r = _noalloc(env, comp, out)
            assert st == zs.OK, lib.zs_last_error()
            assert r.out_len == rr.out_len and r.n_lines == rr.n_lines
            assert torch.equal(out[: r.out_len], ref[: rr.out_len])
            assert torch.all(out[r.out_len:] == 0xAB)


def _decompress_status(env, comp, out):
    zs, lib, d = env
    r = zs._Result()  # the binding declares zs_decompress with its own result type
    st = lib.zs_decompress(d.handle, comp.data_ptr(), comp.numel(), out.data_ptr(), out.numel(), ctypes.byref(r),
                           torch.cuda.current_stream().cuda_stream or None)
    return st, r


def test_same_errors_as_zs_decompress(env):
    """Malformed input (status and first bad offset) and a short output buffer (ZS_ERR_CAPACITY with the
    size needed) come back exactly as zs_decompress reports them."""
    zs, lib, d = env
    raw = synth.generate(synth.CFG0, 0, 4000)
    comp, _, _ = zs.compress(d, torch.from_numpy(raw).cuda(), with_index=False)
    good = comp.clone()
    cases = []
    bad = good.clone()
    bad[1234] = 0x01  # a byte that is no symbol of the default dictionary
    cases.append(bad)
    bad2 = good.clone()
    nl = torch.nonzero(bad2 == 10).flatten()
    bad2[int(nl[7]) - 1] = 32  # an escape with nothing after it in its line
    cases.append(bad2)
    cases.append(torch.cat([good, torch.tensor([32], dtype=torch.uint8, device="cuda")]))  # dangling at the end
    for c in cases:
        out_a = torch.empty(d.decompress_bound(c.numel()), dtype=torch.uint8, device="cuda")
        out_b = torch.empty_like(out_a)
        st_a, ra = _decompress_status(env, c, out_a)
        st_b, rb = _noalloc(env, c, out_b)
        assert st_a == zs.ERR_MALFORMED
        assert (st_b, rb.err_offset) == (st_a, ra.err_offset)
    small_a = torch.empty(1000, dtype=torch.uint8, device="cuda")
    small_b = torch.empty(1000, dtype=torch.uint8, device="cuda")
    st_a, ra = _decompress_status(env, good, small_a)
    st_b, rb = _noalloc(env, good, small_b)
    assert st_a == zs.ERR_CAPACITY
    assert (st_b, rb.out_len, rb.n_lines) == (st_a, ra.out_len, ra.n_lines)


def test_allocates_nothing_across_calls(env):
    """After a first call (which may load the library's device module), further calls leave the device's
    free memory and torch's allocator untouched."""
    zs, lib, d = env
    raw = synth.generate(synth.CFG0, 0, 20000)
    comp, _, _ = zs.compress(d, torch.from_numpy(raw).cuda(), with_index=False)
    comp = comp.clone()
    out = torch.empty(d.decompress_bound(comp.numel()), dtype=torch.uint8, device="cuda")
    st, _ = _noalloc(env, comp, out)
    assert st == zs.OK
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        st, _ = _noalloc(env, comp, out)
        assert st == zs.OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.memory_reserved() == reserved0


def test_rejects_inputs_beyond_its_scratch(env):
    zs, lib, d = env
    comp = torch.zeros(16, dtype=torch.uint8, device="cuda")
    out = torch.zeros(16, dtype=torch.uint8, device="cuda")
    r = _Result()
    # only the size is inspected: nothing is launched for a rejected input
    st = lib.zs_decompress_noalloc(d.handle, comp.data_ptr(), MAX_INPUT + 1, out.data_ptr(), out.numel(),
                                   ctypes.byref(r), None)
    assert st == zs.ERR_INVALID_ARG
    assert b"scratch" in lib.zs_last_error()
