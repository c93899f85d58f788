"""The seeded input generator: reproducible, range-independent, shaped as stated."""
import hashlib

import numpy as np

import synth
from oracle import dictgen
from tests.smiles_graph import ring_bonds


def test_ranges_are_independent():
    whole = synth.generate(synth.CFG0, 0, 500)
    parts = np.concatenate([synth.generate(synth.CFG0, 0, 123), synth.generate(synth.CFG0, 123, 377)])
    assert np.array_equal(whole, parts)
    assert np.array_equal(whole, synth.generate(synth.CFG0, 0, 500, nthreads=1))


def test_small_stream_shape():
    raw = synth.generate(synth.CFG0, 0, synth.CFG0_LINES)
    lines = bytes(raw).split(b"\n")[:-1]
    assert len(lines) == synth.CFG0_LINES
    lens = np.array([len(l) for l in lines])
    assert 44 < lens.mean() < 54 and lens.min() >= 15
    assert set(bytes(raw)) - {10} <= set(dictgen.SMILES_ALPHABET)
    assert all(ring_bonds(l.decode()) is not None for l in lines[:2000])
    digest = hashlib.sha256(raw.tobytes()).hexdigest()
    with open(__file__.replace("test_synth.py", "golden/synth_cfg0.sha256")) as f:
        assert digest == f.read().split()[0]


def test_long_tail_stream_shape():
    raw = synth.generate(synth.CFG3, 0, 20000)
    lines = bytes(raw).split(b"\n")[:-1]
    long = [l for l in lines if len(l) >= 150]
    assert 0.07 < len(long) / len(lines) < 0.13
    assert any(b"%" in l for l in long) and any(b"/" in l for l in long)
    assert set(bytes(raw)) - {10} <= set(dictgen.SMILES_ALPHABET)


def test_batched_shards_shape():
    shards = synth.batched_shards()
    counts = [c for _, c in shards]
    assert len(shards) == 64 and min(counts) >= 1000 and max(counts) <= 5_000_000
    mus = [s.len_mean for s, _ in shards]
    assert 25 <= min(mus) and max(mus) <= 70
