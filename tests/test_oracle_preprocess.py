"""Pins for the oracle's ring-ID pre-processing (Sec. IV-A)."""
import os

import pytest

import oracle
import synth
from tests.smiles_graph import ring_bonds, ring_intervals

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "preprocess_examples.txt")


def _goldens():
    cases = []
    with open(GOLDEN, encoding="ascii") as f:
        for line in f.read().split("\n"):
            if not line or line.startswith("#"):
                if line == "":
                    continue
                continue
            src, exp = line.split("\t", 1)
            cases.append((src, exp))
    return cases


@pytest.mark.parametrize("src,exp", _goldens())
def test_golden(src, exp):
    assert oracle.preprocess_line(src.encode()) == exp.encode()


def test_empty_line_golden_present():
    assert ("", "") in _goldens()


def _sample_lines():
    a = bytes(synth.generate(synth.CFG0, 0, 1500)).split(b"\n")[:-1]
    b = bytes(synth.generate(synth.CFG3, 0, 1500)).split(b"\n")[:-1]
    return a + b


def test_graph_preserved():
    """Same atoms and the same multiset of ring bonds (atom pair + bond symbol) before and after."""
    checked = 0
    for line in _sample_lines():
        before = ring_bonds(line.decode())
        after = ring_bonds(oracle.preprocess_line(line).decode())
        assert before is not None
        assert before == after, line
        checked += before[1].total()
    assert checked > 1000


def test_idempotent():
    for line in _sample_lines():
        p = oracle.preprocess_line(line)
        assert oracle.preprocess_line(p) == p


def test_overlapping_rings_never_share_a_label():
    for line in _sample_lines():
        iv = ring_intervals(oracle.preprocess_line(line).decode())
        for i, (o1, c1, l1) in enumerate(iv):
            for o2, c2, l2 in iv[i + 1:]:
                if o1 < c2 and o2 < c1:
                    assert l1 != l2, line


def test_inner_ring_gets_lower_label():
    """For strictly nested rings the inner one carries the lower ID (the paper's 'innermost')."""
    nested = 0
    for line in _sample_lines():
        iv = ring_intervals(oracle.preprocess_line(line).decode())
        for o1, c1, l1 in iv:
            for o2, c2, l2 in iv:
                if o1 < o2 and c2 < c1:  # ring 2 strictly inside ring 1
                    nested += 1
                    assert l2 < l1, line
    assert nested > 50


def test_labels_restart_and_reuse():
    """Every ring that overlaps no earlier-closing ring gets label 0 (IDs restart and are reused)."""
    for line in _sample_lines():
        iv = ring_intervals(oracle.preprocess_line(line).decode())
        iv.sort(key=lambda t: t[1])
        for k, (o, c, lab) in enumerate(iv):
            if not any(o < c2 and o2 < c for o2, c2, _ in iv[:k]):
                assert lab == 0


def test_two_digit_labels_when_needed():
    """Eleven mutually nested rings need labels 0..10; the outermost is written %10."""
    opens = "".join(f"C%{10 + k}" for k in range(11))
    closes = "".join(f"C%{10 + k}" for k in reversed(range(11)))
    out = oracle.preprocess_line((opens + closes).encode()).decode()
    assert out.startswith("C%10C9C8C7C6C5C4C3C2C1C0")
    assert out.endswith("C0C1C2C3C4C5C6C7C8C9C%10")


def test_length_changes_both_ways():
    assert oracle.preprocess_line(b"C%45CC%45") == b"C0CC0"
    s = "".join(f"C{k}" for k in range(1, 10)) + "C%11C%12" + "C%12C%11" + "".join(f"C{k}" for k in reversed(range(1, 10)))
    out = oracle.preprocess_line(s.encode())
    assert ring_bonds(out.decode()) == ring_bonds(s)
    assert b"%10" in out


def test_stream_preserves_lines_and_final_newline():
    raw = b"C1CC1\n\nC2CC2"
    assert bytes(oracle.preprocess_stream(raw)) == b"C0CC0\n\nC0CC0"
    assert bytes(oracle.preprocess_stream(raw + b"\n")) == b"C0CC0\n\nC0CC0\n"
