"""GPU parity: every call of the C ABI against the CPU oracle, byte for byte (integer/byte work: exact)."""
import os

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DICT_PATH = os.path.join(ROOT, "paper_2404_19391_gb300", "data", "zs_default.zsd")


@pytest.fixture(scope="module")
def zs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19391_gb300 import zsmiles
    zsmiles.load_library()
    return zsmiles


@pytest.fixture(scope="module", params=["transducer", "generic"])
def dicts(zs, request):
    """The default dictionary loaded twice: with its parse transducer (the normal path) and with the
    transducer disabled, which runs the generic per-byte automaton kernel."""
    data = open(DICT_PATH, "rb").read()
    if request.param == "generic":
        os.environ["ZS_FORCE_GENERIC"] = "1"
    try:
        d = zs.Dictionary(data)
    finally:
        os.environ.pop("ZS_FORCE_GENERIC", None)
    assert d.uses_transducer == (request.param == "transducer")
    return d, oracle.Dict(data)


def dev(a):
    return torch.from_numpy(np.array(a, dtype=np.uint8, copy=True)).cuda()


def check_compress(zs, dicts, raw, flags=1, offset_in=0, offset_out=0):
    d, od = dicts
    raw = np.frombuffer(bytes(raw), dtype=np.uint8) if isinstance(raw, (bytes, bytearray)) else raw
    buf = torch.zeros(raw.size + offset_in + 16, dtype=torch.uint8, device="cuda")
    x = buf[offset_in:offset_in + raw.size]
    if raw.size:
        x.copy_(torch.from_numpy(raw.copy()))
    exp_comp, exp_idx = oracle.compress_stream(od, raw, flags)
    cap = zs.zs_compress_bound(raw.size)
    obuf = torch.full((cap + offset_out,), 0xEE, dtype=torch.uint8, device="cuda")
    out = obuf[offset_out:]
    idx = torch.full((exp_idx.size + 3,), -7, dtype=torch.int64, device="cuda")
    r = zs.zs_compress(d, x, flags, out, idx)
    got = out[: r.out_len].cpu().numpy()
    assert r.out_len == exp_comp.size
    assert r.n_lines == exp_idx.size - 1
    if not np.array_equal(got, exp_comp):
        bad = int(np.flatnonzero(got != exp_comp)[0])
        pytest.fail(f"compress differs at byte {bad}: got {bytes(got[max(0, bad - 20):bad + 20])!r} "
                    f"want {bytes(exp_comp[max(0, bad - 20):bad + 20])!r}")
    assert np.array_equal(idx[: exp_idx.size].cpu().numpy().astype(np.uint64), exp_idx)
    assert torch.all(idx[exp_idx.size:] == -7)  # nothing written past the index
    assert torch.all(obuf[:offset_out] == 0xEE) and torch.all(out[r.out_len:] == 0xEE)  # nor past the output
    return out[: r.out_len], idx[: exp_idx.size], exp_comp, exp_idx


def check_decompress(zs, dicts, comp_np, expect=None):
    d, od = dicts
    x = dev(comp_np)
    exp = oracle.decompress_stream(od, comp_np) if expect is None else expect
    cap = max(1, d.decompress_bound(comp_np.size))
    out = torch.full((cap + 16,), 0xEE, dtype=torch.uint8, device="cuda")
    r = zs.zs_decompress(d, x, out[:cap])
    got = out[: r.out_len].cpu().numpy()
    assert r.out_len == exp.size
    assert np.array_equal(got, exp)
    assert torch.all(out[r.out_len:] == 0xEE)
    assert r.n_lines == oracle.count_lines(comp_np)
    return got


# ---- full streams -------------------------------------------------------------------------------------

def test_small_stream_parity(zs, dicts):
    raw = synth.generate(synth.CFG0, 0, synth.CFG0_LINES)
    comp, idx, exp_comp, exp_idx = check_compress(zs, dicts, raw)
    check_decompress(zs, dicts, exp_comp, expect=oracle.preprocess_stream(raw))
    # the index over the compressed stream, rebuilt from scratch
    gidx = zs.line_index(comp)
    assert np.array_equal(gidx.cpu().numpy().astype(np.uint64), exp_idx)


def test_without_preprocessing(zs, dicts):
    raw = synth.generate(synth.CFG0, 100, 3000)
    _, _, exp_comp, _ = check_compress(zs, dicts, raw, flags=0)
    check_decompress(zs, dicts, exp_comp, expect=raw)


def test_long_tail_stream_parity(zs, dicts):
    raw = synth.generate(synth.CFG3, 0, 40000)
    _, _, exp_comp, _ = check_compress(zs, dicts, raw)
    check_decompress(zs, dicts, exp_comp)


@pytest.mark.parametrize("seed", [3, 4, 7])
def test_batched_shard_shapes(zs, dicts, seed):
    shards = synth.batched_shards(n_shards=8, seed=seed, count_lo=10, count_hi=20000)
    for shape, count in shards[:4]:
        raw = synth.generate(shape, 0, count)
        check_compress(zs, dicts, raw)


@pytest.mark.parametrize("off_in,off_out", [(1, 0), (3, 7), (15, 1), (0, 9)])
def test_unaligned_buffers(zs, dicts, off_in, off_out):
    raw = synth.generate(synth.CFG0, 7, 2500)
    check_compress(zs, dicts, raw, offset_in=off_in, offset_out=off_out)


# ---- edge cases -------------------------------------------------------------------------------------

EDGE = {
    "empty": b"",
    "one_newline": b"\n",
    "newlines_only": b"\n" * 40000,
    "no_trailing_newline": b"C1CC1O\nc1ccccc1",
    "empty_lines": b"CCO\n\n\nC1CC1\n\n",
    "single_char": b"C",
    "escapes_only": bytes([0x41, 0x47, 0x51, 0x5a, 0x7c]) * 5,
    "cr_tab": b"C1CC1\r\nCCO\tname 1\nC C\n",
    "invalid_rings": b"C1CC\nC[NH3+C1CC1\nC%1CC\nC%(12)CC%(12)\n",
    "percent_labels": b"C%12CC%12\nC%45C%67CC%67C%45\n",
    "percent_low_labels": b"C%05CC5\nC5CC%05\nC%01CC%01\nC%00C%09CC%09C%00\nC%07C%12CC7C%12\n",
    "bracket_digits": b"[13CH3]C1CC1\n[NH3+]C5CC5\n",
    "space_field": b"C1CC1 id12 C2\n",
}


@pytest.mark.parametrize("name", sorted(EDGE))
def test_edge_cases(zs, dicts, name):
    raw = EDGE[name]
    if raw == b"":
        d, _ = dicts
        idx = torch.full((2,), -1, dtype=torch.int64, device="cuda")
        out = torch.empty(16, dtype=torch.uint8, device="cuda")
        r = zs.zs_compress(d, torch.empty(0, dtype=torch.uint8, device="cuda"), 1, out, idx)
        assert r.out_len == 0 and r.n_lines == 0 and idx[0].item() == 0
        return
    for flags in (0, 1):
        _, _, exp_comp, _ = check_compress(zs, dicts, raw, flags=flags)
        check_decompress(zs, dicts, exp_comp)


def _nested(k):
    opens = "".join(f"C%{10 + i}" for i in range(k))
    closes = "".join(f"C%{10 + i}" for i in reversed(range(k)))
    return opens + closes


def test_irregular_lines_take_the_exact_slow_path(zs, dicts):
    lines = [
        _nested(11),                      # needs label 10 -> '%10' (grows)
        _nested(20),                      # more than 16 rings open at once
        "".join(f"C{k}" for k in range(1, 10)) + "C%11C%12C%12C%11" + "".join(f"C{k}" for k in reversed(range(1, 10))),
        "C1CCX1",                         # escape in a relabelled line
        "C%12CCQ%12",                     # escape after a shrunk label
    ]
    raw = ("\n".join(lines) + "\n").encode()
    for flags in (0, 1):
        _, _, exp_comp, _ = check_compress(zs, dicts, raw, flags=flags)
        check_decompress(zs, dicts, exp_comp)


@pytest.mark.parametrize("length", [4000, 4097, 20000, 100_000, 1_000_000])
def test_long_lines(zs, dicts, length):
    rng = np.random.default_rng(length)
    base = bytes(synth.generate(synth.CFG3, 0, 20000)).replace(b"\n", b"")
    start = int(rng.integers(0, len(base) - length - 1)) if len(base) > length + 1 else 0
    line = (base * (1 + length // max(1, len(base))))[start:start + length]
    raw = b"CCO\n" + line + b"\nC1CC1\n" + line[: length // 3] + b"\n"
    _, _, exp_comp, _ = check_compress(zs, dicts, raw)
    check_decompress(zs, dicts, exp_comp)


@pytest.mark.parametrize("pad", [16382, 16383, 16384, 16385, 20479, 20480, 20481])
def test_lines_on_tile_boundaries(zs, dicts, pad):
    """A line that ends exactly at, just before and just after a tile / halo boundary."""
    line = (b"c1ccccc1C(=O)N" * 2000)[: pad - 4]
    raw = b"CC\n" + line + b"\nCCO\n" + b"C1CC1\n" * 3000
    check_compress(zs, dicts, raw)
    raw2 = line + b"\n" + line[:100] + b"\n" + line
    check_compress(zs, dicts, raw2)


def test_many_tiny_lines_in_one_tile(zs, dicts):
    """More lines in a tile than one batch holds (multi-batch, chained tile)."""
    raw = b"C\n" * 50000 + b"\n" * 20000 + b"CO\n" * 10000
    _, _, exp_comp, _ = check_compress(zs, dicts, raw)
    check_decompress(zs, dicts, exp_comp)


def test_random_bytes(zs, dicts):
    rng = np.random.default_rng(5)
    raw = rng.integers(0, 256, size=300_000, dtype=np.uint8)
    raw[rng.integers(0, raw.size, 3000)] = 10
    _, _, exp_comp, _ = check_compress(zs, dicts, raw)
    check_decompress(zs, dicts, exp_comp)
    _, _, exp_comp0, _ = check_compress(zs, dicts, raw, flags=0)
    check_decompress(zs, dicts, exp_comp0, expect=raw)


def test_deterministic(zs, dicts):
    d, _ = dicts
    raw = dev(synth.generate(synth.CFG3, 5, 20000))
    a, ia, _ = zs.compress(d, raw)
    for _ in range(3):
        b, ib, _ = zs.compress(d, raw)
        assert torch.equal(a, b) and torch.equal(ia, ib)


# ---- errors -----------------------------------------------------------------------------------------

def test_capacity_errors(zs, dicts):
    d, od = dicts
    raw = synth.generate(synth.CFG0, 0, 2000)
    exp_comp, exp_idx = oracle.compress_stream(od, raw)
    x = dev(raw)
    out = torch.empty(exp_comp.size - 1, dtype=torch.uint8, device="cuda")
    with pytest.raises(zs.ZsError) as e:
        zs.zs_compress(d, x, 1, out, None)
    assert e.value.status == zs.ERR_CAPACITY and e.value.result.out_len == exp_comp.size
    out = torch.empty(exp_comp.size, dtype=torch.uint8, device="cuda")
    idx = torch.empty(exp_idx.size - 1, dtype=torch.int64, device="cuda")
    with pytest.raises(zs.ZsError) as e:
        zs.zs_compress(d, x, 1, out, idx)
    assert e.value.status == zs.ERR_CAPACITY
    r = zs.zs_compress(d, x, 1, out, None)  # exact capacity suffices
    assert np.array_equal(out.cpu().numpy(), exp_comp)
    c = dev(exp_comp)
    dout = torch.empty(raw.size - 5, dtype=torch.uint8, device="cuda")
    with pytest.raises(zs.ZsError) as e:
        zs.zs_decompress(d, c, dout)
    assert e.value.status == zs.ERR_CAPACITY


def test_malformed_inputs(zs, dicts):
    d, od = dicts
    good, _ = oracle.compress_stream(od, synth.generate(synth.CFG0, 0, 3000))
    undefined = next(b for b in range(0x80, 0xA1))
    cases = []
    a = good.copy()
    a[20000] = undefined
    cases.append(a)
    b = bytearray(good.tobytes())
    nl = b.index(b"\n", 30000)
    b[nl - 1] = 32  # line ends in an unpaired escape
    cases.append(np.frombuffer(bytes(b), dtype=np.uint8))
    cases.append(np.frombuffer(bytes(good.tobytes()[:-1] + b" "), dtype=np.uint8))  # stream ends in one
    for case in cases:
        with pytest.raises(oracle.OracleError) as oe:
            oracle.decompress_stream(od, case)
        out = torch.empty(d.decompress_bound(case.size), dtype=torch.uint8, device="cuda")
        with pytest.raises(zs.ZsError) as ge:
            zs.zs_decompress(d, dev(case), out)
        assert ge.value.status == zs.ERR_MALFORMED
        assert ge.value.result.err_offset == oe.value.where


def test_escape_runs(zs, dicts):
    """Runs of spaces (escaped spaces) straddling thread slices and tiles."""
    d, od = dicts
    lines = [b" " * k + b"C" for k in range(1, 40)] + [b"C" + b" " * 9000 + b"O"]
    raw = b"\n".join(lines) + b"\n"
    _, _, exp_comp, _ = check_compress(zs, dicts, raw, flags=0)
    check_decompress(zs, dicts, exp_comp, expect=np.frombuffer(raw, dtype=np.uint8))


def test_tiles_that_outgrow_the_decoder_stage(zs, dicts):
    """Compressed stretches made of the dictionary's longer patterns (3 bytes and more) expand more than the
    decoder stages per tile (2.25x): those tiles write straight to memory after their look-back, between ordinary
    tiles whose output is staged, and the whole output must still equal the oracle's."""
    d, od = dicts
    longer = []
    for s in range(33, 256):  # one-symbol lines through the oracle decoder give each symbol's pattern length
        try:
            n = oracle.decompress_stream(od, np.array([s, 10], dtype=np.uint8)).size - 1
        except oracle.OracleError:
            continue
        if n >= 3:
            longer.append(s)
    assert len(longer) >= 8
    rng = np.random.default_rng(11)
    ordinary = oracle.compress_stream(od, synth.generate(synth.CFG0, 0, 2000), 1)[0]
    parts = []
    for k in range(5):
        lines = rng.choice(longer, size=(int(rng.integers(60, 160)), 40)).astype(np.uint8)
        stretch = np.concatenate([lines, np.full((lines.shape[0], 1), 10, dtype=np.uint8)], axis=1).ravel()
        cut = int(rng.integers(1, ordinary.size))
        cut = int(np.flatnonzero(ordinary[cut:] == 10)[0]) + cut + 1 if (ordinary[cut:] == 10).any() else ordinary.size
        parts += [ordinary[:cut], stretch]
    comp = np.concatenate(parts)
    check_decompress(zs, dicts, comp)


# ---- line index and random access ---------------------------------------------------------------------

@pytest.mark.parametrize("data", [b"\n", b"a", b"a\n", b"a\nb", b"a\nb\n", b"\n\n\nx", b"xy\n\nz\n"])
def test_line_index_small(zs, data):
    idx = zs.line_index(dev(np.frombuffer(data, dtype=np.uint8)))
    assert np.array_equal(idx.cpu().numpy().astype(np.uint64), oracle.line_index(data))


def test_line_index_large(zs):
    rng = np.random.default_rng(2)
    raw = rng.integers(0, 256, size=5_000_001, dtype=np.uint8)
    for off in (0, 5):
        x = dev(raw)[off:]
        idx = zs.line_index(x)
        assert np.array_equal(idx.cpu().numpy().astype(np.uint64), oracle.line_index(raw[off:]))


@pytest.mark.parametrize("off", [0, 3])
def test_line_index_dense_and_sparse_tiles(zs, off):
    """Runs of newlines put more entries in a tile than the index kernel stages in shared memory (those tiles
    write directly), between tiles with no newline and ordinary lines; the index must still equal a plain
    newline scan, aligned or not, with no final newline."""
    rng = np.random.default_rng(11)
    parts = []
    for k in range(12):
        if k % 3 == 0:
            parts.append(np.full(40000 + k, 10, dtype=np.uint8))
        elif k % 3 == 1:
            parts.append(rng.integers(11, 256, size=70000 + 17 * k).astype(np.uint8))
        else:
            parts.append(np.frombuffer(bytes(synth.generate(synth.CFG0, k, 3000)), dtype=np.uint8))
    raw = np.concatenate(parts + [np.array([65, 66], dtype=np.uint8)])
    x = dev(np.concatenate([np.zeros(off, dtype=np.uint8), raw]))[off:]
    idx = zs.line_index(x)
    assert np.array_equal(idx.cpu().numpy().astype(np.uint64), oracle.line_index(raw))


def test_random_access_parity(zs, dicts):
    d, od = dicts
    raw = synth.generate(synth.CFG3, 0, 30000)
    comp, idx, exp_comp, exp_idx = check_compress(zs, dicts, raw)
    rng = np.random.default_rng(9)
    for k in [1, 7, 256, 257, 5000]:
        ids = rng.integers(0, exp_idx.size - 1, size=k).astype(np.int64)
        out, off, r = zs.decompress_lines(d, comp, idx, torch.from_numpy(ids).cuda())
        exp_out, exp_off = oracle.decompress_lines(od, exp_comp, exp_idx, ids.astype(np.uint64))
        assert np.array_equal(out.cpu().numpy(), exp_out)
        assert np.array_equal(off.cpu().numpy().astype(np.uint64), exp_off)


def test_random_access_bad_id(zs, dicts):
    d, od = dicts
    raw = synth.generate(synth.CFG0, 0, 1000)
    comp, idx, _, _ = check_compress(zs, dicts, raw)
    ids = torch.tensor([3, 999, 1000, 5, 1001], dtype=torch.int64, device="cuda")
    out = torch.empty(100000, dtype=torch.uint8, device="cuda")
    off = torch.empty(6, dtype=torch.int64, device="cuda")
    with pytest.raises(zs.ZsError) as e:
        zs.zs_decompress_lines(d, comp, idx, ids, out, off)
    assert e.value.status == zs.ERR_MALFORMED and e.value.result.err_offset == 2


# ---- failure detection: a look-back record that is never published ------------------------------------

def test_stalled_tile_times_out(zs, dicts, monkeypatch):
    d, _ = dicts
    raw = dev(synth.generate(synth.CFG0, 0, 5000))
    out = torch.empty(zs.zs_compress_bound(raw.numel()), dtype=torch.uint8, device="cuda")
    monkeypatch.setenv("ZS_WAIT_LIMIT_MS", "300")
    monkeypatch.setenv("ZS_INJECT_STALL", "2")
    with pytest.raises(zs.ZsError) as e:
        zs.zs_compress(d, raw, 1, out, None)
    assert e.value.status == zs.ERR_TIMEOUT
    comp = dev(oracle.compress_stream(dicts[1], synth.generate(synth.CFG0, 0, 5000))[0])
    dout = torch.empty(d.decompress_bound(comp.numel()), dtype=torch.uint8, device="cuda")
    with pytest.raises(zs.ZsError) as e:
        zs.zs_decompress(d, comp, dout)
    assert e.value.status == zs.ERR_TIMEOUT
    monkeypatch.delenv("ZS_INJECT_STALL")
    monkeypatch.delenv("ZS_WAIT_LIMIT_MS")
    r = zs.zs_compress(d, raw, 1, out, None)  # the context is still usable
    assert r.n_lines == 5000


# ---- a dictionary with patterns longer than 7 bytes (the byte-wise decoder and, if its transducer is too
# large, the generic compression kernel) ---------------------------------------------------------------------

@pytest.fixture(scope="module")
def long_dicts(zs):
    from oracle import dictgen
    train = oracle.preprocess_stream(synth.generate(synth.TRAIN, 0, 3000))
    learned = [bytes.fromhex(ln.split()[1]) for ln in
               dictgen.generate(train, T=130, lmin=2, lmax=12).decode().splitlines()[3:]]
    extra = [b"c0ccccc0C(=O)N", b"C(=O)NCC", b"CCCCCCCCCCCC", b"c0ccc(cc0)", b"C(=O)O)cc0"]
    data = dictgen.dictionary_text(learned + [e for e in extra if e not in learned], dictgen.SMILES_ALPHABET, 2, 16)
    od = oracle.Dict(data)
    longest = max(len(bytes.fromhex(ln.split()[1])) for ln in data.decode().splitlines()[3:])
    assert longest > 7
    return zs.Dictionary(data), od


def test_long_pattern_dictionary(zs, long_dicts):
    raw = synth.generate(synth.CFG0, 500, 4000)
    for flags in (0, 1):
        _, _, exp_comp, _ = check_compress(zs, long_dicts, raw, flags=flags)
        check_decompress(zs, long_dicts, exp_comp)
    for name in ("escapes_only", "cr_tab", "no_trailing_newline", "empty_lines"):
        _, _, exp_comp, _ = check_compress(zs, long_dicts, EDGE[name])
        check_decompress(zs, long_dicts, exp_comp)
    d, od = long_dicts
    _, _, exp_comp, _ = check_compress(zs, long_dicts, raw)
    for v in range(zs.zs_kernel_variants(zs.OP_DECOMPRESS)):
        x = dev(exp_comp)
        out = torch.full((d.decompress_bound(exp_comp.size) + 16,), 0xEE, dtype=torch.uint8, device="cuda")
        if "expand" in zs.zs_kernel_variant_name(zs.OP_DECOMPRESS, v):
            # the expansion kernel keeps a pattern and its length in one 64-bit entry: up to 7 bytes
            with pytest.raises(zs.ZsError) as e:
                zs.Plan(d, zs.OP_DECOMPRESS, [(x, out[:-16], None)], variant=v)
            assert e.value.status == zs.ERR_BAD_DICT
            continue
        r = zs.Plan(d, zs.OP_DECOMPRESS, [(x, out[:-16], None)], variant=v).run()[0]
        assert np.array_equal(out[: r.out_len].cpu().numpy(), oracle.decompress_stream(od, exp_comp))
        assert torch.all(out[r.out_len:] == 0xEE)


@pytest.mark.parametrize("name", ["zs_lmax5.zsd", "zs_lmax15.zsd", "zs_no_alphabet.zsd", "zs_raw_train.zsd",
                                  "zs_outer_train.zsd", "zs_printable.zsd", "zs_printable_raw.zsd",
                                  "zs_no_alphabet_raw.zsd"])
def test_ablation_dictionaries(zs, name):
    """Every ablation dictionary (L_max 5 / 15; pre-population printable, SMILES alphabet or none, trained with
    and without ring renumbering; opening-order training) codes exactly like the oracle, with pre-processing
    off and in either reading."""
    data = open(os.path.join(ROOT, "paper_2404_19391_gb300", "data", name), "rb").read()
    pair = (zs.Dictionary(data), oracle.Dict(data))
    raw = synth.generate(synth.CFG0, 900, 3000)
    for flags in (0, 1, 3):
        _, _, exp_comp, _ = check_compress(zs, pair, raw, flags=flags)
        check_decompress(zs, pair, exp_comp)
