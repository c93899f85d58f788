"""Pins for dictionary generation (Algorithm 1, Eq. 1, Sec. IV-C) and pre-population (Sec. IV-B)."""
import hashlib
import os
import random

import numpy as np
import pytest

import oracle
import synth
from oracle import dictgen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_alphabet_and_code_space():
    a = dictgen.SMILES_ALPHABET
    assert len(a) == len(set(a)) == 43
    cs = dictgen.code_space(a)
    assert len(cs) == 146
    assert not (set(cs) & set(a)) and 10 not in cs and 32 not in cs
    assert all(0x21 <= b <= 0x7E or 0xA1 <= b <= 0xFF for b in cs)


def test_hand_computed_ranks():
    """Training set {'CCCC'}, L in [2,4]: occ CC=3, CCC=2, CCCC=1; Eq. 1 at t=0 gives 6, 6, 4, the tie
    goes to the higher occ (CC). At t=1 CC lies inside both others (overlap 2): CCC -> 2*1 = 2,
    CCCC -> 1*2 = 2; tie -> higher occ (CCC). At t=2 CCCC contains CCC (overlap 3): 1*1 = 1."""
    occ = dictgen.count_substrings([b"CCCC"], 2, 4)
    assert occ == {b"CC": 3, b"CCC": 2, b"CCCC": 1}
    assert dictgen.select_naive(occ, 5) == [b"CC", b"CCC", b"CCCC"]
    assert dictgen.select_lazy(occ, 5) == [b"CC", b"CCC", b"CCCC"]
    assert dictgen.rank(b"CCCC", 1, [b"CC", b"CCC"]) == 1


def test_overlap_cases():
    assert dictgen.overlap(b"ab", b"xaby") == 2      # p inside w
    assert dictgen.overlap(b"xaby", b"ab") == 2      # w inside p
    assert dictgen.overlap(b"abc", b"cde") == 1      # suffix of p = prefix of w
    assert dictgen.overlap(b"cde", b"abc") == 1      # the other order
    assert dictgen.overlap(b"abcd", b"cdab") == 2
    assert dictgen.overlap(b"ab", b"cd") == 0


def test_stops_when_rank_not_positive():
    occ = dictgen.count_substrings([b"abab"], 2, 2)   # ab x2, ba x1
    # after 'ab', 'ba' overlaps it by 1 -> rank 1*(2-1) = 1 > 0, still chosen; nothing else remains
    assert dictgen.select_lazy(occ, 10) == [b"ab", b"ba"]
    occ = dictgen.count_substrings([b"aaa"], 2, 3)    # aa x2, aaa x1; aa inside aaa
    sel = dictgen.select_naive(occ, 10)
    assert sel == dictgen.select_lazy(occ, 10)


@pytest.mark.parametrize("seed", range(12))
def test_lazy_equals_naive(seed):
    rng = random.Random(seed)
    letters = b"CcN()=1"
    lines = [bytes(rng.choice(letters) for _ in range(rng.randint(3, 16))) for _ in range(rng.randint(3, 20))]
    occ = dictgen.count_substrings(lines, 2, rng.randint(2, 5))
    T = rng.randint(1, 25)
    assert dictgen.select_lazy(occ, T) == dictgen.select_naive(occ, T)


def test_fast_count_equals_plain_count():
    raw = synth.generate(synth.TRAIN, 0, 800)
    pre = oracle.preprocess_stream(raw)
    lines = bytes(pre).split(b"\n")[:-1]
    assert dictgen.count_substrings(lines, 2, 8) == dictgen.count_substrings_fast(pre, 2, 8)
    # spaces and newlines never enter a pattern
    assert dictgen.count_substrings([b"ab cd"], 2, 3) == {b"ab": 1, b"cd": 1}


def test_patterns_are_training_substrings_and_deterministic():
    raw = synth.generate(synth.TRAIN, 0, 1500)
    pre = oracle.preprocess_stream(raw)
    t1 = dictgen.generate(pre, T=60)
    t2 = dictgen.generate(pre, T=60)
    assert t1 == t2
    d = oracle.Dict(t1)
    assert d.entries == 43 + 60
    body = bytes(pre)
    for line in t1.split(b"\n")[3:]:
        if line:
            pat = bytes.fromhex(line.split(b" ")[1].decode())
            assert 2 <= len(pat) <= 8 and pat in body


def test_frozen_default_dictionary_regenerates():
    """The committed dictionary file is exactly what Algorithm 1 writes for the seed-1 training set."""
    from oracle.make_dictionary import build_default
    path = os.path.join(ROOT, "paper_2404_19391_gb300", "data", "zs_default.zsd")
    with open(path, "rb") as f:
        committed = f.read()
    assert hashlib.sha256(build_default()).digest() == hashlib.sha256(committed).digest()


def test_dictionary_file_validation():
    good = dictgen.dictionary_text([b"CC"], dictgen.SMILES_ALPHABET, 2, 8)
    oracle.Dict(good)
    bad = [
        good.replace(b"ZSDICT 1", b"ZSDICT 2"),
        good.replace(b"2 8 1", b"2 8 2"),                 # missing entry
        good + b"22 6363\n",                              # extra line
        good.replace(b"21 4343", b"43 4343"),             # symbol 'C' already an alphabet entry
        good.replace(b"21 4343", b"21 43"),               # pattern 'C' duplicates an alphabet entry
        good.replace(b"21 4343", b"20 4343"),             # space as a symbol
        good.replace(b"21 4343", b"21 4320"),             # space inside a pattern
        good.replace(b"2 8 1", b"2 17 1"),                # lmax above 16
    ]
    for b in bad:
        with pytest.raises(oracle.OracleError):
            oracle.Dict(b)


def test_ablation_dictionaries_load():
    """The committed ablation dictionaries (one varied choice each) are valid files with the stated settings."""
    import os
    data_dir = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2404_19391_gb300",
                            "data")
    want = {"zs_lmax5.zsd": (5, True), "zs_lmax15.zsd": (15, True), "zs_no_alphabet.zsd": (8, False),
            "zs_raw_train.zsd": (8, True), "zs_outer_train.zsd": (8, True), "zs_printable.zsd": (8, True),
            "zs_printable_raw.zsd": (8, True), "zs_no_alphabet_raw.zsd": (8, False)}
    for name, (lmax, alpha) in want.items():
        text = open(os.path.join(data_dir, name), "rb").read()
        lines = text.decode().splitlines()
        assert lines[0] == "ZSDICT 1"
        assert int(lines[1].split()[1]) == lmax
        assert (lines[2] != "alphabet -") == alpha
        oracle.Dict(text)  # parses and validates
        if name.startswith("zs_printable"):  # Table I "Printable": every printable byte pre-populated, so the
            # learned patterns take the 95 symbols 0xA1-0xFF
            assert bytes.fromhex(lines[2].split()[1]) == bytes(range(0x21, 0x7F))
            assert int(lines[1].split()[2]) == 95
            assert all(0xA1 <= int(ln.split()[0], 16) <= 0xFF for ln in lines[3:] if ln)


def test_printable_dictionary_regenerates():
    """The committed Table I 'Printable' dictionary is what Algorithm 1 writes for the seed-1 training set with
    the printable pre-population (T cut to the 95 free symbols)."""
    from oracle.make_dictionary import build_default
    path = os.path.join(ROOT, "paper_2404_19391_gb300", "data", "zs_printable.zsd")
    with open(path, "rb") as f:
        committed = f.read()
    assert build_default(T=95, alphabet=dictgen.PRINTABLE_ALPHABET) == committed
