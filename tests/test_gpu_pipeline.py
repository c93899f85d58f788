"""GPU tests of the host-to-host pipelines (zs_compress_host / zs_decompress_host): chunked at line ends,
several chunks in flight; the output, line index and errors must be exactly those of the device calls and
of the CPU oracle."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19391_gb300 import zsmiles
    zsmiles.load_library()
    data = open(zsmiles.DEFAULT_DICTIONARY, "rb").read()
    return zsmiles, zsmiles.Dictionary(data), oracle.Dict(data)


def _pinned(a: np.ndarray) -> torch.Tensor:
    t = torch.empty(a.size, dtype=torch.uint8, pin_memory=True)
    t.copy_(torch.from_numpy(np.array(a, dtype=np.uint8, copy=True)))
    return t


def _round_trip(env, raw: np.ndarray, chunk: int, streams: int, pinned: bool = True, flags: int = 1):
    zs, d, od = env
    h_in = _pinned(raw) if pinned else torch.from_numpy(raw.copy())
    exp_c, exp_i = oracle.compress_stream(od, raw, flags)
    out = torch.full((zs.zs_compress_bound(raw.size),), 0xEE, dtype=torch.uint8, pin_memory=pinned)
    idx = torch.full((exp_i.size + 3,), -7, dtype=torch.int64, pin_memory=pinned)
    r = zs.zs_compress_host(d, h_in, flags, out, idx, chunk_bytes=chunk, n_streams=streams)
    assert r.out_len == exp_c.size and r.n_lines == exp_i.size - 1
    assert np.array_equal(out[: r.out_len].numpy(), exp_c)
    assert np.array_equal(idx[: exp_i.size].numpy().astype(np.uint64), exp_i)
    assert torch.all(out[r.out_len:] == 0xEE) and torch.all(idx[exp_i.size:] == -7)
    dec = torch.full((max(1, d.decompress_bound(exp_c.size)),), 0xEE, dtype=torch.uint8, pin_memory=pinned)
    h_c = _pinned(exp_c) if pinned else torch.from_numpy(exp_c.copy())
    r2 = zs.zs_decompress_host(d, h_c, dec, chunk_bytes=chunk, n_streams=streams)
    want = oracle.decompress_stream(od, exp_c)
    assert r2.out_len == want.size and np.array_equal(dec[: r2.out_len].numpy(), want)
    return r, r2


@pytest.mark.parametrize("chunk,streams", [(4096, 1), (4096, 3), (65536, 4), (1 << 20, 2), (0, 0)])
def test_pipeline_parity(env, chunk, streams):
    raw = synth.generate(synth.CFG0, 0, 20000)
    _round_trip(env, raw, chunk, streams)


def test_pipeline_long_tail_and_no_final_newline(env):
    raw = synth.generate(synth.CFG3, 0, 6000)
    _round_trip(env, raw, 8192, 3)
    _round_trip(env, raw[:-1], 8192, 3)  # no final newline
    _round_trip(env, raw, 8192, 3, flags=0)


def test_pipeline_pageable_buffers(env):
    raw = synth.generate(synth.CFG0, 3, 5000)
    _round_trip(env, raw, 16384, 2, pinned=False)


def test_pipeline_edges(env):
    zs, d, od = env
    for data in [b"\n", b"C", b"C1CC1\n" * 3000, b"\n" * 10000 + b"CCO"]:
        _round_trip(env, np.frombuffer(data, dtype=np.uint8), 4096, 3)
    out = torch.empty(16, dtype=torch.uint8)
    idx = torch.full((2,), -1, dtype=torch.int64)
    r = zs.zs_compress_host(d, torch.empty(0, dtype=torch.uint8), 1, out, idx)
    assert r.out_len == 0 and r.n_lines == 0 and idx[0].item() == 0


def test_pipeline_errors(env):
    zs, d, od = env
    raw = np.frombuffer(b"CCO\n" + b"C" * 10000 + b"\nCC\n", dtype=np.uint8)
    out = torch.empty(zs.zs_compress_bound(raw.size), dtype=torch.uint8)
    with pytest.raises(zs.ZsError) as e:  # a line longer than the chunk
        zs.zs_compress_host(d, torch.from_numpy(raw.copy()), 1, out, None, chunk_bytes=4096)
    assert e.value.status == zs.ERR_CAPACITY
    good = synth.generate(synth.CFG0, 0, 3000)
    exp_c, _ = oracle.compress_stream(od, good, 1)
    small = torch.empty(exp_c.size - 1, dtype=torch.uint8)
    with pytest.raises(zs.ZsError) as e:
        zs.zs_compress_host(d, torch.from_numpy(good.copy()), 1, small, None, chunk_bytes=8192, n_streams=2)
    assert e.value.status == zs.ERR_CAPACITY and e.value.result.out_len == exp_c.size
    bad = exp_c.copy()
    pos = next(j for j in range(bad.size // 2, bad.size) if bad[j - 1] != 0x20 and bad[j] not in (0x20, 0x0A))
    bad[pos] = 0x01
    dec = torch.empty(d.decompress_bound(bad.size), dtype=torch.uint8)
    with pytest.raises(zs.ZsError) as e:
        zs.zs_decompress_host(d, torch.from_numpy(bad), dec, chunk_bytes=4096, n_streams=3)
    assert e.value.status == zs.ERR_MALFORMED and e.value.result.err_offset == pos
