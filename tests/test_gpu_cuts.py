"""GPU parity of the span kernel on long lines, which it cuts between lanes at reset points (positions after a
ring-bond token that leaves no ring open, where the relabelling of Sec. IV-A restarts exactly) and mends at
each cut (the parse state and the piece chain of Sec. IV-D1 carry across). Every case is compared byte for
byte with the CPU oracle, for both relabelling orders and without pre-processing, at the default cut
threshold and at thresholds small enough to cut almost every line several times."""
import os

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
    return zs.Dictionary(data), oracle.Dict(data)


def _ring_chain(n: int) -> bytes:
    """n rings in a row, each closed before the next opens: a reset point after every closure."""
    return b"".join(b"C%dCC%d" % (k % 10, k % 10) for k in range(n))


def _nested(depth: int) -> bytes:
    """depth rings opened before any closes: no reset point inside; depth > 10 needs two-digit labels."""
    labels = [b"%d" % k if k < 10 else b"%%%02d" % k for k in range(depth)]
    return b"C" + b"C".join(labels) + b"CC" + b"C".join(reversed(labels)) + b"O"


def _pct_nested(n: int) -> bytes:
    """n %nn rings (labels 10 and up) opened before any closes: a lane follows six at once, more take the
    one-line path."""
    labels = [b"%%%02d" % (10 + k) for k in range(n)]
    return b"C" + b"C".join(labels) + b"CC" + b"C".join(reversed(labels)) + b"O"


def _long_lines() -> list[bytes]:
    rng = np.random.default_rng(7)
    cfg3 = [l for l in bytes(synth.generate(synth.CFG3, 0, 4000)).split(b"\n")[:-1] if len(l) >= 96]
    lines = list(cfg3[:300])
    lines += [_ring_chain(k) for k in (8, 20, 40, 90, 200)]
    lines += [b"N[NH3+]" + _ring_chain(30) + b"[13CH3]c1ccc%12cc1%12[O-]" * 4]
    lines.append(_ring_chain(25) + b"C1CCC")                # unclosed ring at the end: left as it is
    lines.append(_ring_chain(25) + b"C%1xC" + _ring_chain(10))  # a bad %: left as it is
    lines.append(_ring_chain(12) + _nested(12) + _ring_chain(12))  # labels above 9 in the middle
    lines += [_ring_chain(10) + _pct_nested(k) + _ring_chain(10) for k in (4, 5, 6, 7, 9)]
    lines.append(_ring_chain(15) + b" " + _ring_chain(15))  # a second field
    lines.append(_ring_chain(15) + b"\t" + _ring_chain(15))
    lines.append(_ring_chain(10) + b"[C[N]]" + _ring_chain(10))  # nested bracket
    lines.append(_ring_chain(10) + b"]" + _ring_chain(10))  # unmatched bracket
    lines.append(_ring_chain(10) + b"C%05CC%05" + _ring_chain(10))  # %0n is label n
    lines.append(_ring_chain(20) + bytes([0xC3, 0xA9]) + _ring_chain(20))  # bytes >= 0x80
    lines.append(b"C" * 300)
    lines.append(b"c1ccccc1" * 40)
    out = []
    for k, l in enumerate(lines):  # interleave short lines, in runs of random length
        out.append(l)
        for _ in range(int(rng.integers(0, 6))):
            out.append(b"CC(=O)N%dCC%d" % (k % 10, k % 10))
    return out


def _streams() -> list[bytes]:
    lines = _long_lines()
    whole = b"\n".join(lines) + b"\n"
    return [whole, whole[:-1], b"\n".join(lines[::-1]) + b"\n", b"\n".join(l for l in lines if len(l) >= 96) + b"\n"]


def _span_variants(zs):
    return [v for v in range(zs.zs_kernel_variants(zs.OP_COMPRESS))
            if "span" in zs.zs_kernel_variant_name(zs.OP_COMPRESS, v)]


def _run(zs, d, raw: bytes, flags: int, variant: int):
    x = torch.empty(max(1, len(raw)), dtype=torch.uint8, device="cuda")
    x[: len(raw)].copy_(torch.frombuffer(bytearray(raw), dtype=torch.uint8))
    x = x[: len(raw)]
    out = torch.full((zs.zs_compress_bound(len(raw)) + 16,), 0xEE, dtype=torch.uint8, device="cuda")
    idx = torch.full((raw.count(b"\n") + 4,), -7, dtype=torch.int64, device="cuda")
    p = zs.Plan(d, zs.OP_COMPRESS, [(x, out[:-16], idx)], flags=flags, variant=variant, use_graph=False)
    r = p.run()[0]
    p.close()
    return r, out, idx


@pytest.mark.parametrize("cut_min", [None, 8, 40])
@pytest.mark.parametrize("flags", [1, 3, 0])
def test_cut_lines_match_oracle(zs, dicts, cut_min, flags):
    d, od = dicts
    old = os.environ.get("ZS_SPAN_CUT_MIN")
    if cut_min is not None:
        os.environ["ZS_SPAN_CUT_MIN"] = str(cut_min)
    try:
        for raw in _streams():
            ec, ei = oracle.compress_stream(od, np.frombuffer(raw, dtype=np.uint8), flags)
            for v in _span_variants(zs):
                r, out, idx = _run(zs, d, raw, flags, v)
                tag = f"variant {v} flags {flags} cut_min {cut_min}"
                assert r.out_len == ec.size and r.n_lines == ei.size - 1, tag
                assert np.array_equal(out[: r.out_len].cpu().numpy(), ec), tag
                assert np.array_equal(idx[: ei.size].cpu().numpy().astype(np.uint64), ei), tag
                assert torch.all(out[r.out_len:] == 0xEE), tag
                assert torch.all(idx[ei.size:] == -7), tag
    finally:
        if old is None:
            os.environ.pop("ZS_SPAN_CUT_MIN", None)
        else:
            os.environ["ZS_SPAN_CUT_MIN"] = old


def test_long_tail_stream_every_cut_threshold(zs, dicts):
    """The long-tail mix (10% of 150-400 byte lines) at several thresholds, including none (0)."""
    d, od = dicts
    raw = bytes(synth.generate(synth.CFG3, 1000, 20000))
    ec, ei = oracle.compress_stream(od, np.frombuffer(raw, dtype=np.uint8), 1)
    old = os.environ.get("ZS_SPAN_CUT_MIN")
    try:
        for cm in ("0", "16", "64", "96", "200"):
            os.environ["ZS_SPAN_CUT_MIN"] = cm
            for v in _span_variants(zs):
                r, out, idx = _run(zs, d, raw, 1, v)
                assert r.out_len == ec.size and np.array_equal(out[: r.out_len].cpu().numpy(), ec), (cm, v)
                assert np.array_equal(idx[: ei.size].cpu().numpy().astype(np.uint64), ei), (cm, v)
    finally:
        if old is None:
            os.environ.pop("ZS_SPAN_CUT_MIN", None)
        else:
            os.environ["ZS_SPAN_CUT_MIN"] = old


def _stage_long_lines() -> list[bytes]:
    """Lines longer than any tile and its halo (4-12 KB), built from long-tail fragments, with the cases the
    warp-wide line coder must keep exact."""
    rng = np.random.default_rng(11)
    frag = [l for l in bytes(synth.generate(synth.CFG3, 0, 6000)).split(b"\n")[:-1] if len(l) >= 150]
    out = []
    for k in range(12):
        target, cur = int(rng.integers(4000, 12001)), b""
        while len(cur) < target:
            cur += frag[int(rng.integers(0, len(frag)))]
        out.append(cur)
    big = out[0]
    out.append(big + b"C1CC")                               # unclosed ring: left as it is
    out.append(big[:3000] + b"C%1xC" + big[3000:])          # a bad %
    out.append(big[:2000] + _nested(14) + big[2000:])       # labels above 9
    out.append(big[:2500] + _pct_nested(9) + big[2500:])    # many open %nn
    out.append(big[:4000] + b" second field 12 %34" + big[4000:6000])
    out.append(big[:1000] + bytes([0xC3, 0xA9]) + big[1000:])
    out.append(b"c1ccccc1" * 900)
    return out


@pytest.mark.parametrize("flags", [1, 3, 0])
def test_lines_longer_than_the_stage(zs, dicts, flags):
    d, od = dicts
    longs = _stage_long_lines()
    rng = np.random.default_rng(5)
    short = bytes(synth.generate(synth.CFG1, 0, 3000)).split(b"\n")[:-1]
    lines = []
    for k, l in enumerate(longs):
        lines += short[k * 100:(k * 100) + int(rng.integers(0, 60))]
        lines.append(l)
    raws = [b"\n".join(lines) + b"\n", b"\n".join(lines), longs[-1], longs[0] + b"\n" + longs[1]]
    for raw in raws:
        ec, ei = oracle.compress_stream(od, np.frombuffer(raw, dtype=np.uint8), flags)
        for v in _span_variants(zs):
            r, out, idx = _run(zs, d, raw, flags, v)
            tag = f"variant {v} flags {flags} bytes {len(raw)}"
            assert r.out_len == ec.size and r.n_lines == ei.size - 1, tag
            assert np.array_equal(out[: r.out_len].cpu().numpy(), ec), tag
            assert np.array_equal(idx[: ei.size].cpu().numpy().astype(np.uint64), ei), tag
            assert torch.all(out[r.out_len:] == 0xEE), tag
