"""GPU parity of the opening-order reading of ring-ID pre-processing (ZS_PREPROCESS | ZS_PREPROCESS_OUTER,
the other reading of Sec. IV-A): every compress path (the transducer kernel in each geometry, the generic
kernel, the batched plan, the host pipeline, dictionary training) must give the oracle's bytes exactly."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests import test_gpu_codec as codec

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

OUTER = 3  # ZS_PREPROCESS | ZS_PREPROCESS_OUTER
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def zs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19391_gb300 import zsmiles
    zsmiles.load_library()
    return zsmiles


@pytest.fixture(scope="module", params=["transducer", "generic"])
def dicts(zs, request):
    data = open(codec.DICT_PATH, "rb").read()
    if request.param == "generic":
        os.environ["ZS_FORCE_GENERIC"] = "1"
    try:
        d = zs.Dictionary(data)
    finally:
        os.environ.pop("ZS_FORCE_GENERIC", None)
    assert d.uses_transducer == (request.param == "transducer")
    return d, oracle.Dict(data)


def ring_soup(seed: int, n_lines: int, digits_only: bool = False, max_steps: int = 160) -> bytes:
    """Lines dense in ring labels: up to 14 rings open at once, labels 0-99 written as digits or %nn (a few
    below 10 as %0d), bracket atoms with digits inside, some lines with a second field, some left with an
    unclosed ring. digits_only: labels 0-9 written as digits (short lines then stay on the bit-mask path)."""
    rng = np.random.default_rng(seed)

    def tok(lab):
        return (f"%0{lab}" if not digits_only and rng.random() < 0.1 else str(lab)) if lab < 10 else f"%{lab}"

    atoms = ["C", "c", "N", "O", "[13CH3]", "[NH3+]", "Cl", "n"]
    out = []
    for _ in range(n_lines):
        max_open = int(rng.integers(1, 11 if digits_only else 15))
        steps = int(rng.integers(2, max_steps))
        open_labels, parts = [], ["C"]
        for _ in range(steps):
            u = rng.random()
            if u < 0.45:
                parts.append(atoms[int(rng.integers(len(atoms)))])
            elif u < 0.55:
                parts.append("=")
            elif u < 0.8 and len(open_labels) < max_open:
                free = [l for l in range(10 if digits_only else 100) if l not in open_labels]
                lab = int(rng.choice(free[:12] if rng.random() < 0.8 else free))
                open_labels.append(lab)
                parts.append(tok(lab))
            elif open_labels:
                lab = open_labels.pop(int(rng.integers(len(open_labels))))
                parts.append(tok(lab))
        leave = rng.random() < 0.05
        while open_labels and not (leave and len(open_labels) == 1):
            lab = open_labels.pop(int(rng.integers(len(open_labels))))
            parts.append("C" + tok(lab))
        line = "".join(parts)
        if rng.random() < 0.05:
            line += " id 12 C1"
        out.append(line)
    return ("\n".join(out) + "\n").encode()


def test_synthetic_streams(zs, dicts):
    for cfg, n in ((synth.CFG0, synth.CFG0_LINES), (synth.CFG3, 20000)):
        raw = synth.generate(cfg, 11, n)
        _, _, exp_comp, _ = codec.check_compress(zs, dicts, raw, flags=OUTER)
        codec.check_decompress(zs, dicts, exp_comp, expect=oracle.preprocess_stream(raw, outer=True))


@pytest.mark.parametrize("seed,digits_only,max_steps", [(1, False, 160), (2, False, 60), (3, True, 60),
                                                        (4, True, 160)])
def test_ring_soup(zs, dicts, seed, digits_only, max_steps):
    raw = ring_soup(seed, 3000, digits_only, max_steps)
    for flags in (1, OUTER):  # the dense-ring lines check the default reading too
        _, _, exp_comp, _ = codec.check_compress(zs, dicts, raw, flags=flags)
        codec.check_decompress(zs, dicts, exp_comp)


@pytest.mark.parametrize("name", sorted(codec.EDGE))
def test_edge_cases(zs, dicts, name):
    raw = codec.EDGE[name]
    if not raw:
        return
    _, _, exp_comp, _ = codec.check_compress(zs, dicts, raw, flags=OUTER)
    codec.check_decompress(zs, dicts, exp_comp)


def test_irregular_lines(zs, dicts):
    lines = [
        codec._nested(10),                # labels 0..9 from the outside in: the fast path
        codec._nested(11),                # the innermost needs %10: the slow path
        codec._nested(20),
        "c1ccc2ccccc2c1",
        "C1CCX1", "C%12CCQ%12",           # escapes in relabelled lines
        "C1C2C3C4C5C6C7C8C9C%10C%11CC%11C%10C9C8C7C6C5C4C3C2C1",
        "c1ccccc1" * 20,                  # longer than the bit-mask path's limit
        "C%12C%13C%14C%15C%16C%17C%18C%19C%20CC%20C%19C%18C%17C%16C%15C%14C%13C%12",  # > 8 open %nn
    ]
    raw = ("\n".join(lines) + "\n").encode()
    _, _, exp_comp, _ = codec.check_compress(zs, dicts, raw, flags=OUTER)
    codec.check_decompress(zs, dicts, exp_comp)
    # the flag changes nested lines only
    out = codec.check_decompress(zs, dicts, exp_comp).tobytes().split(b"\n")
    assert out[3] == b"c0ccc1ccccc1c0"


@pytest.mark.parametrize("length", [4000, 100_000])
def test_long_lines(zs, dicts, length):
    line = (ring_soup(length, 200).replace(b"\n", b"") * 50)[:length]
    raw = b"C1CC1\n" + line + b"\nc1ccc2ccccc2c1\n"
    codec.check_compress(zs, dicts, raw, flags=OUTER)


def test_modifier_alone_is_refused(zs, dicts):
    d, _ = dicts
    x = codec.dev(np.frombuffer(b"C1CC1\n", dtype=np.uint8))
    out = torch.empty(64, dtype=torch.uint8, device="cuda")
    for flags in (2, 4, 7):
        with pytest.raises(zs.ZsError) as e:
            zs.zs_compress(d, x, flags, out, None)
        assert e.value.status == zs.ERR_INVALID_ARG


def test_every_geometry_through_a_plan(zs):
    for variant in range(zs.zs_kernel_variants(zs.OP_COMPRESS)):
        data = open(codec.DICT_PATH, "rb").read()
        d, od = zs.Dictionary(data), oracle.Dict(data)
        raws = [ring_soup(40 + k, 500 * (k + 1)) for k in range(3)] + [bytes(synth.generate(synth.CFG3, 5, 4000))]
        ins = [codec.dev(np.frombuffer(b, dtype=np.uint8)) for b in raws]
        outs = [torch.full((zs.zs_compress_bound(len(b)),), 0xEE, dtype=torch.uint8, device="cuda") for b in raws]
        idxs = [torch.full((b.count(b"\n") + 1,), -7, dtype=torch.int64, device="cuda") for b in raws]
        p = zs.Plan(d, zs.OP_COMPRESS, list(zip(ins, outs, idxs)), flags=OUTER, variant=variant)
        res = p.run()
        for r, b, o, x in zip(res, raws, outs, idxs):
            ec, ei = oracle.compress_stream(od, np.frombuffer(b, dtype=np.uint8), OUTER)
            assert r.out_len == ec.size and np.array_equal(o[: r.out_len].cpu().numpy(), ec)
            assert np.array_equal(x[: ei.size].cpu().numpy().astype(np.uint64), ei)
        p.close()


def test_host_pipeline(zs):
    data = open(codec.DICT_PATH, "rb").read()
    d, od = zs.Dictionary(data), oracle.Dict(data)
    raw = np.frombuffer(ring_soup(9, 20000), dtype=np.uint8)
    ec, ei = oracle.compress_stream(od, raw, OUTER)
    h_in = torch.from_numpy(raw.copy()).pin_memory()
    out = torch.empty(zs.zs_compress_bound(raw.size), dtype=torch.uint8).pin_memory()
    idx = torch.empty(ei.size, dtype=torch.int64).pin_memory()
    r = zs.zs_compress_host(d, h_in, OUTER, out, idx, chunk_bytes=1 << 16, n_streams=3)
    assert r.out_len == ec.size and np.array_equal(out[: r.out_len].numpy(), ec)
    assert np.array_equal(idx.numpy().astype(np.uint64), ei)


def test_training_on_open_order_lines(zs):
    """Algorithm 1 over lines pre-processed in opening order, against the oracle's; the committed
    open-order ablation dictionary is what the full training set gives."""
    from oracle import dictgen
    raw = synth.generate(synth.TRAIN, 0, 6000)
    want = dictgen.generate(oracle.preprocess_stream(raw, outer=True), T=146, lmin=2, lmax=8)
    got = zs.zs_train_dictionary(torch.from_numpy(np.array(raw, copy=True)).cuda(), OUTER, lmin=2, lmax=8, T=146)
    assert got == want
    full = synth.generate(synth.TRAIN, 0, synth.TRAIN_LINES)
    got = zs.zs_train_dictionary(torch.from_numpy(np.array(full, copy=True)).cuda(), OUTER, lmin=2, lmax=8, T=146)
    path = os.path.join(ROOT, "paper_2404_19391_gb300", "data", "zs_outer_train.zsd")
    assert got == open(path, "rb").read()
