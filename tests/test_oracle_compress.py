"""Pins for the oracle's compression (Sec. IV-D1), decompression (Sec. IV-D2), streams and line index."""
import itertools
import random

import numpy as np
import pytest

import oracle
import synth
from oracle import dictgen

ALPHA = dictgen.SMILES_ALPHABET


def make_dict(patterns, alphabet=ALPHA, lmax=None):
    lmax = lmax or max([len(p) for p in patterns] + [2])
    return oracle.Dict(dictgen.dictionary_text(list(patterns), alphabet, 1, lmax))


def brute_force(d_entries: dict, line: bytes) -> bytes:
    """Enumerate every segmentation of `line` into dictionary pieces (cost 1) and escapes (cost 2),
    keep the minimum-cost ones, and among them the lexicographically greatest sequence of piece
    lengths (longest piece first at every step), an escape counting as a piece of length 1 that
    loses to a dictionary piece of length 1."""
    n = len(line)
    best = None

    def rec(i, pieces, cost):
        nonlocal best
        if i == n:
            key = (cost, [(-l, esc) for l, esc, _ in pieces])
            if best is None or key < best[0]:
                best = (key, list(pieces))
            return
        if best is not None and cost > best[0][0]:
            return
        for l in range(1, n - i + 1):
            sym = d_entries.get(line[i:i + l])
            if sym is not None:
                pieces.append((l, 0, bytes([sym])))
                rec(i + l, pieces, cost + 1)
                pieces.pop()
        pieces.append((1, 1, b" " + line[i:i + 1]))
        rec(i + 1, pieces, cost + 2)
        pieces.pop()

    rec(0, [], 0)
    return b"".join(p for _, _, p in best[1])


def entries_of(patterns, alphabet=ALPHA):
    ent = {bytes([c]): c for c in alphabet}
    for sym, p in zip(dictgen.code_space(alphabet), patterns):
        ent[p] = sym
    return ent


def test_brute_force_small_alphabet():
    """Random tiny dictionaries over a 3-letter alphabet (so patterns overlap heavily and ties abound)."""
    rng = random.Random(7)
    letters = b"abc"
    for trial in range(300):
        pool = sorted({bytes(rng.choice(letters) for _ in range(rng.randint(2, 4))) for _ in range(12)})
        pats = rng.sample(pool, min(len(pool), rng.randint(1, 8)))
        alphabet = bytes(rng.sample(list(letters), rng.randint(0, 3)))
        d = make_dict(pats, alphabet=alphabet, lmax=4)
        ent = entries_of(pats, alphabet)
        for _ in range(6):
            line = bytes(rng.choice(letters + b"x") for _ in range(rng.randint(0, 11)))
            assert oracle.compress_line(d, line) == brute_force(ent, line), (pats, alphabet, line)


def test_brute_force_smiles_like():
    rng = random.Random(11)
    lines = [l for l in bytes(synth.generate(synth.CFG0, 0, 400)).split(b"\n") if l]
    for trial in range(120):
        src = oracle.preprocess_line(rng.choice(lines))
        a = rng.randrange(0, max(1, len(src) - 12))
        line = src[a:a + rng.randint(1, 12)]
        subs = sorted({src[i:i + l] for i in range(len(src)) for l in range(2, 6) if i + l <= len(src)})
        pats = rng.sample(subs, min(len(subs), 20))
        d = make_dict(pats, lmax=5)
        assert oracle.compress_line(d, line) == brute_force(entries_of(pats), line)


def test_identity_only_dictionary_is_identity():
    d = make_dict([], lmax=2)
    for line in bytes(synth.generate(synth.CFG0, 0, 200)).split(b"\n"):
        assert oracle.compress_line(d, line) == line


def test_empty_dictionary_escapes_everything():
    d = make_dict([], alphabet=b"", lmax=2)
    for line in [b"", b"C", b"CCO", b"c1ccccc1"]:
        out = oracle.compress_line(d, line)
        assert len(out) == 2 * len(line)
        assert out == b"".join(b" " + bytes([c]) for c in line)


def test_known_parse():
    """'CCCC' with D = alphabet + {CC, CCC}: minimum cost 2 (CC+CC or CCC+C); the longest-first rule
    picks CCC then C."""
    d = make_dict([b"CC", b"CCC"])
    sym = dict(zip([b"CC", b"CCC"], dictgen.code_space(ALPHA)))
    assert oracle.compress_line(d, b"CCCC") == bytes([sym[b"CCC"], ord("C")])
    # greedy-longest is not the rule: 'abcd' with {abc, ab, cd} -> ab+cd (2), not abc+d... d is not in
    # the alphabet, so abc + escape(d) costs 3
    d2 = make_dict([b"abc", b"ab", b"cd"], alphabet=b"abc")
    s2 = dict(zip([b"abc", b"ab", b"cd"], dictgen.code_space(b"abc")))
    assert oracle.compress_line(d2, b"abcd") == bytes([s2[b"ab"], s2[b"cd"]])


@pytest.fixture(scope="module")
def default_dict():
    import os
    p = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2404_19391_gb300", "data", "zs_default.zsd")
    return oracle.Dict(open(p, "rb").read())


def test_roundtrip_and_invariants(default_dict):
    raw = np.concatenate([synth.generate(synth.CFG0, 0, 3000), synth.generate(synth.CFG3, 0, 1000)])
    comp, idx = oracle.compress_stream(default_dict, raw)
    pre = oracle.preprocess_stream(raw)
    assert np.array_equal(oracle.decompress_stream(default_dict, comp), pre)
    # one output line per input line
    assert oracle.count_lines(comp) == oracle.count_lines(raw) == idx.size - 1
    # readable output (Sec. I): alphabet-only input gives printable bytes only
    b = comp[comp != 10]
    assert np.all(((b >= 0x21) & (b <= 0x7E)) | (b >= 0xA1))
    # pre-population guarantee (Sec. IV-B): no line grows
    plines = bytes(pre).split(b"\n")
    clines = bytes(comp).split(b"\n")
    assert all(len(c) <= len(p) for c, p in zip(clines, plines))
    # without pre-processing the round trip returns the input itself
    comp2, _ = oracle.compress_stream(default_dict, raw, flags=0)
    assert np.array_equal(oracle.decompress_stream(default_dict, comp2), raw)


def test_line_index_matches_newline_scan(default_dict):
    for data in [b"", b"\n", b"a", b"a\n", b"a\nb", b"a\nb\n", b"\n\n\nx", b"xy\n\nz\n"]:
        idx = oracle.line_index(data)
        starts = [0] + [i + 1 for i, c in enumerate(data) if c == 10 and i + 1 < len(data)] if data else []
        assert list(idx[:-1]) == starts
        assert idx[-1] == len(data)
        assert len(data.split(b"\n")) - (1 if data.endswith(b"\n") or not data else 0) == idx.size - 1


def test_escape_and_final_newline(default_dict):
    raw = b"CCX\n\nC C\r\nZ"
    comp, idx = oracle.compress_stream(default_dict, raw, flags=0)
    assert bytes(oracle.decompress_stream(default_dict, comp)) == raw
    assert not bytes(comp).endswith(b"\n")
    assert b" X" in bytes(comp) and b" \r" in bytes(comp) and b"  " in bytes(comp)


def test_malformed(default_dict):
    with pytest.raises(oracle.OracleError) as e:
        oracle.decompress_stream(default_dict, b"CC\nC \n")
    assert e.value.status == oracle.ERR_MALFORMED and e.value.where == 4
    undefined = next(b for b in range(256) if b not in (10, 32) and
                     b not in set(ALPHA) and b not in dictgen.code_space(ALPHA)[:146])
    with pytest.raises(oracle.OracleError) as e:
        oracle.decompress_stream(default_dict, bytes([ord("C"), undefined]))
    assert e.value.where == 1


def test_random_access_equals_cut_from_full(default_dict):
    raw = synth.generate(synth.CFG0, 0, 2000)
    comp, idx = oracle.compress_stream(default_dict, raw)
    full = bytes(oracle.decompress_stream(default_dict, comp)).split(b"\n")
    rng = np.random.default_rng(3)
    ids = rng.integers(0, idx.size - 1, size=300).astype(np.uint64)
    out, off = oracle.decompress_lines(default_dict, comp, idx, ids)
    for r, i in enumerate(ids):
        assert bytes(out[off[r]:off[r + 1]]) == full[int(i)] + b"\n"
    with pytest.raises(oracle.OracleError):
        oracle.decompress_lines(default_dict, comp, idx, np.array([idx.size - 1], dtype=np.uint64))


def test_parallel_partition_equals_single(default_dict):
    raw = synth.generate(synth.CFG0, 0, 3000)
    a = oracle.compress_stream(default_dict, raw)
    b = oracle.compress_stream_parallel(default_dict, raw, threads=5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
