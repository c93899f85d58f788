"""GPU parity of the batched form (many shards, one persistent launch, CUDA graph replay, autotuned
kernel geometry) against the CPU oracle, byte for byte, shard by shard, for every compiled variant."""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def zs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19391_gb300 import zsmiles
    zsmiles.load_library()
    return zsmiles


@pytest.fixture(scope="module")
def dicts(zs):
    data = open(zs.DEFAULT_DICTIONARY, "rb").read()
    d = zs.Dictionary(data)
    assert d.uses_transducer
    return d, oracle.Dict(data)


def _raw_shards():
    """Uneven shards: generator shards of 1 to 20k lines with different length mixes, plus edge shards
    (empty, a lone newline, no trailing newline, a line longer than any tile, the long-tail mix)."""
    out = [bytes(synth.generate(shape, 0, count)) for shape, count in
           synth.batched_shards(n_shards=10, seed=11, count_lo=1, count_hi=20000)]
    out.insert(2, b"")
    out.insert(5, b"\n")
    out.append(b"C1CC1O\nc1ccccc1")
    out.append(b"CCO\n" + (b"c1ccccc1C(=O)N" * 700) + b"\nC\n")
    out.insert(0, b"")
    out.append(bytes(synth.generate(synth.CFG3, 0, 3000)))
    return out


RAW = _raw_shards()


def _dev(b: bytes):
    t = torch.empty(max(1, len(b)), dtype=torch.uint8, device="cuda")
    if b:
        t[: len(b)].copy_(torch.frombuffer(bytearray(b), dtype=torch.uint8))
    return t[: len(b)]


@pytest.fixture(scope="module")
def expected(dicts):
    _, od = dicts
    return [oracle.compress_stream(od, np.frombuffer(b, dtype=np.uint8), 1) for b in RAW]


def _compress_shards(zs, raws, exp=None, fill=0xEE):
    ins = [_dev(b) for b in raws]
    outs = [torch.full((zs.zs_compress_bound(len(b)) + 16,), fill, dtype=torch.uint8, device="cuda") for b in raws]
    idxs = [torch.full((b.count(b"\n") + 4,), -7, dtype=torch.int64, device="cuda") for b in raws]
    return [(i, o[:-16], x) for i, o, x in zip(ins, outs, idxs)], outs, idxs


def _check_compressed(res, shards, outs, idxs, exp):
    for k, (r, (_, out, idx), (ec, ei)) in enumerate(zip(res, shards, exp)):
        assert r.out_len == ec.size, f"shard {k}"
        assert r.n_lines == ei.size - 1, f"shard {k}"
        assert np.array_equal(out[: r.out_len].cpu().numpy(), ec), f"shard {k}"
        assert np.array_equal(idx[: ei.size].cpu().numpy().astype(np.uint64), ei), f"shard {k}"
        assert torch.all(outs[k][r.out_len:] == 0xEE), f"shard {k} wrote past its output"
        assert torch.all(idx[ei.size:] == -7), f"shard {k} wrote past its index"


def _decompress_shards(zs, d, comps):
    ins = [_dev(c.tobytes()) for c in comps]
    outs = [torch.full((max(1, d.decompress_bound(c.size)) + 16,), 0xEE, dtype=torch.uint8, device="cuda")
            for c in comps]
    return [(i, o[:-16], None) for i, o in zip(ins, outs)], outs


def test_plan_every_variant(zs, dicts, expected):
    for variant in range(zs.zs_kernel_variants(zs.OP_COMPRESS)):
        d, od = dicts
        shards, outs, idxs = _compress_shards(zs, RAW)
        p = zs.Plan(d, zs.OP_COMPRESS, shards, flags=1, variant=variant, use_graph=True)
        assert p.variant == variant
        for _ in range(2):  # graph replay: the scratch is cleared by the graph itself
            res = p.run()
            _check_compressed(res, shards, outs, idxs, expected)
        p.close()
        comps = [ec for ec, _ in expected]
        dv = variant % zs.zs_kernel_variants(zs.OP_DECOMPRESS)
        dsh, douts = _decompress_shards(zs, d, comps)
        q = zs.Plan(d, zs.OP_DECOMPRESS, dsh, variant=dv, use_graph=True)
        for _ in range(2):
            res = q.run()
            for k, (r, raw) in enumerate(zip(res, RAW)):
                want = oracle.preprocess_stream(np.frombuffer(raw, dtype=np.uint8))
                assert r.out_len == want.size, f"shard {k}"
                assert np.array_equal(douts[k][: r.out_len].cpu().numpy(), want), f"shard {k}"
                assert torch.all(douts[k][r.out_len:] == 0xEE)
        q.close()


def test_autotuned_plan(zs, dicts, expected):
    """The autotuner times every geometry that can run the batch and keeps the fastest. RAW holds a line
    longer than a span tile plus its halo: the span kernel codes it in place (one lane, from memory), so its
    geometries are timed too, with and without that line."""
    d, _ = dicts
    nv = zs.zs_kernel_variants(zs.OP_COMPRESS)
    span = {v for v in range(nv) if "span" in zs.zs_kernel_variant_name(zs.OP_COMPRESS, v)}
    assert span
    for raws, exp in ((RAW, expected), (RAW[:-2], expected[:-2])):
        shards, outs, idxs = _compress_shards(zs, raws)
        p = zs.Plan(d, zs.OP_COMPRESS, shards, flags=1, variant=-1, tune_reps=2)
        times = [p.tuned_ms(v) for v in range(nv)]
        assert all(t > 0 for t in times), times
        assert p.variant == min(range(nv), key=lambda v: times[v])
        _check_compressed(p.run(), shards, outs, idxs, exp)
        assert p.last_ms > 0
        p.close()


def test_one_shot_batch_calls(zs, dicts, expected):
    d, _ = dicts
    shards, outs, idxs = _compress_shards(zs, RAW)
    _check_compressed(zs.zs_compress_batch(d, shards, 1), shards, outs, idxs, expected)
    dsh, douts = _decompress_shards(zs, d, [ec for ec, _ in expected])
    res = zs.zs_decompress_batch(d, dsh)
    for k, (r, raw) in enumerate(zip(res, RAW)):
        want = oracle.preprocess_stream(np.frombuffer(raw, dtype=np.uint8))
        assert np.array_equal(douts[k][: r.out_len].cpu().numpy(), want), f"shard {k}"


def test_batch_equals_single_calls(zs, dicts):
    """Each shard gets exactly the bytes the single-stream call gives it alone (no preprocessing too)."""
    d, _ = dicts
    raws = [bytes(synth.generate(shape, 0, count)) for shape, count in
            synth.batched_shards(n_shards=6, seed=5, count_lo=100, count_hi=30000)]
    shards, _, _ = _compress_shards(zs, raws)
    res = zs.zs_compress_batch(d, shards, 0)
    for (x, out, idx), r in zip(shards, res):
        c, i, r1 = zs.compress(d, x, flags=0)
        assert r.out_len == r1.out_len and r.n_lines == r1.n_lines
        assert torch.equal(out[: r.out_len], c) and torch.equal(idx[: r.n_lines + 1], i)


def test_many_small_shards(zs, dicts):
    """More shards than one 32-way search round covers, many of them empty."""
    d, od = dicts
    rng = np.random.default_rng(2)
    raws = []
    for k in range(1500):
        n = int(rng.integers(0, 4))
        raws.append(b"" if n == 0 else bytes(synth.generate(synth.CFG0, k * 10, n)))
    exp = [oracle.compress_stream(od, np.frombuffer(b, dtype=np.uint8), 1) for b in raws]
    shards, outs, idxs = _compress_shards(zs, raws)
    p = zs.Plan(d, zs.OP_COMPRESS, shards, flags=1, variant=0)
    _check_compressed(p.run(), shards, outs, idxs, exp)


def test_tile_boundaries_every_variant(zs, dicts):
    """Lines ending just before, at and after each variant's tile and halo boundaries."""
    for variant in range(zs.zs_kernel_variants(zs.OP_COMPRESS)):
        d, od = dicts
        name = zs.zs_kernel_variant_name(zs.OP_COMPRESS, variant)
        tile = int(name.split("t")[-1])
        raws = []
        for edge in (tile, 2 * tile, 3 * tile + 512, 2 * tile + 1024):
            for delta in (-2, -1, 0, 1, 2):
                line = (b"c1ccccc1C(=O)N" * 800)[: edge + delta - 3]
                raws.append(b"CC\n" + line + b"\nCCO\n" + b"C1CC1\n" * 50)
        exp = [oracle.compress_stream(od, np.frombuffer(b, dtype=np.uint8), 1) for b in raws]
        shards, outs, idxs = _compress_shards(zs, raws)
        p = zs.Plan(d, zs.OP_COMPRESS, shards, flags=1, variant=variant, use_graph=False)
        _check_compressed(p.run(), shards, outs, idxs, exp)
        comps = [ec for ec, _ in exp]
        for dv in range(zs.zs_kernel_variants(zs.OP_DECOMPRESS)):
            dsh, douts = _decompress_shards(zs, d, comps)
            res = zs.Plan(d, zs.OP_DECOMPRESS, dsh, variant=dv).run()
            for k, r in enumerate(res):
                want = oracle.decompress_stream(od, comps[k])
                assert np.array_equal(douts[k][: r.out_len].cpu().numpy(), want), f"variant {dv} shard {k}"


def test_graph_replay_sees_new_data(zs, dicts):
    """A plan fixes buffers, not contents: new input in the same buffers gives the new output."""
    d, od = dicts
    a = bytes(synth.generate(synth.CFG0, 0, 3000))
    b = bytes(synth.generate(synth.CFG0, 50_000, 3000))
    n = min(len(a), len(b))
    a, b = a[:n], b[:n]
    shards, outs, idxs = _compress_shards(zs, [a])
    p = zs.Plan(d, zs.OP_COMPRESS, shards, flags=1, variant=0, use_graph=True)
    _check_compressed(p.run(), shards, outs, idxs, [oracle.compress_stream(od, np.frombuffer(a, np.uint8), 1)])
    shards[0][0].copy_(_dev(b))
    outs[0].fill_(0xEE)
    idxs[0].fill_(-7)
    _check_compressed(p.run(), shards, outs, idxs, [oracle.compress_stream(od, np.frombuffer(b, np.uint8), 1)])


def test_batch_capacity_error_names_the_shard(zs, dicts, expected):
    d, _ = dicts
    shards, _, _ = _compress_shards(zs, RAW)
    k = next(i for i in range(3, len(RAW)) if expected[i][0].size > 100)
    x, out, idx = shards[k]
    shards[k] = (x, out[: max(0, expected[k][0].size - 1)], idx)
    with pytest.raises(zs.ZsError) as ei:
        zs.zs_compress_batch(d, shards, 1)
    assert ei.value.status == zs.ERR_CAPACITY and f"shard {k}" in str(ei.value)


def test_batch_malformed_shard(zs, dicts, expected):
    d, _ = dicts
    comps = [ec.copy() for ec, _ in expected]
    k = next(i for i in range(3, len(RAW)) if expected[i][0].size > 100)
    bad = comps[k]
    i = next(j for j in range(bad.size // 2, bad.size) if bad[j - 1] not in (0x20,) and bad[j] not in (0x20, 0x0A))
    bad[i] = 0x01  # not a symbol, and not escaped
    dsh, _ = _decompress_shards(zs, d, comps)
    with pytest.raises(zs.ZsError) as ei:
        zs.zs_decompress_batch(d, dsh)
    assert ei.value.status == zs.ERR_MALFORMED and f"shard {k}" in str(ei.value)


def test_plan_argument_errors(zs, dicts):
    d, _ = dicts
    x = _dev(b"CCO\n")
    out = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(zs.ZsError) as ei:
        zs.Plan(d, zs.OP_COMPRESS, [(x, out, None)], variant=99)
    assert ei.value.status == zs.ERR_INVALID_ARG
    with pytest.raises(zs.ZsError) as ei:
        zs.Plan(d, 7, [(x, out, None)])
    assert ei.value.status == zs.ERR_INVALID_ARG
    p = zs.Plan(d, zs.OP_COMPRESS, [], variant=0)
    assert p.run() == []


def test_tuned_cut_setting_and_tuning_cache(zs, dicts, tmp_path):
    """Autotuning also times the span geometries' long-line cut setting both ways; with tune_cache, a second
    plan of the same shape takes the choice from the cache (untimed) and the cache file records it; a fixed
    span variant runs with cuts forced off or at a given threshold, all with oracle parity."""
    import os
    d, od = dicts
    raws = [bytes(synth.generate(synth.CFG3, 0, 4000)), bytes(synth.generate(synth.CFG3, 4000, 2500))]
    exp = [oracle.compress_stream(od, np.frombuffer(b, dtype=np.uint8), 1) for b in raws]
    path = tmp_path / "tune.txt"
    old = os.environ.get("ZS_TUNE_CACHE")
    os.environ["ZS_TUNE_CACHE"] = str(path)
    try:
        nv = zs.zs_kernel_variants(zs.OP_COMPRESS)
        shards, outs, idxs = _compress_shards(zs, raws)
        p = zs.Plan(d, zs.OP_COMPRESS, shards, flags=1, variant=-1, tune_reps=1, tune_cache=True)
        v, c = p.variant, p.cut_min
        assert all(p.tuned_ms(k) > 0 for k in range(nv))
        _check_compressed(p.run(), shards, outs, idxs, exp)
        p.close()
        shards, outs, idxs = _compress_shards(zs, raws)
        q = zs.Plan(d, zs.OP_COMPRESS, shards, flags=1, variant=-1, tune_cache=True)
        assert (q.variant, q.cut_min) == (v, c)
        assert all(q.tuned_ms(k) < 0 for k in range(nv))
        _check_compressed(q.run(), shards, outs, idxs, exp)
        q.close()
        lines = path.read_text().split("\n")
        assert len([l for l in lines if l.strip()]) == 1 and lines[0].split()[1:] == [str(v), str(c)]
    finally:
        if old is None:
            os.environ.pop("ZS_TUNE_CACHE", None)
        else:
            os.environ["ZS_TUNE_CACHE"] = old
    for sv in range(nv):
        if "span" not in zs.zs_kernel_variant_name(zs.OP_COMPRESS, sv):
            continue
        for cm in (-1, 64):
            shards, outs, idxs = _compress_shards(zs, raws)
            r = zs.Plan(d, zs.OP_COMPRESS, shards, flags=1, variant=sv, use_graph=False, cut_min=cm)
            assert r.cut_min == (0 if cm < 0 else cm)
            _check_compressed(r.run(), shards, outs, idxs, exp)
            r.close()
