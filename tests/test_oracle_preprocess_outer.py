"""Pins for the oracle's other reading of ring-ID pre-processing (Sec. IV-A): rings labelled in the order
they open, so among nested rings the outermost gets the lower ID. The paper's worked example has no nested
rings and holds under both readings; where no ring nests inside another the two readings must agree."""
import os

import numpy as np
import pytest

import oracle
import synth
from tests.smiles_graph import ring_bonds, ring_intervals

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "preprocess_examples.txt")


def _outer(s: bytes) -> bytes:
    return oracle.preprocess_line(s, outer=True)


def _sample_lines():
    a = bytes(synth.generate(synth.CFG0, 1, 1500)).split(b"\n")[:-1]
    b = bytes(synth.generate(synth.CFG3, 1, 1500)).split(b"\n")[:-1]
    return a + b


def _has_nesting(iv):
    return any(o1 < o2 and c2 < c1 for o1, c1, _ in iv for o2, c2, _ in iv)


def _goldens():
    with open(GOLDEN, encoding="ascii") as f:
        rows = [l for l in f.read().split("\n") if l and not l.startswith("#")]
    return [tuple(r.split("\t", 1)) for r in rows]


@pytest.mark.parametrize("src,exp", _goldens())
def test_goldens_without_nesting_agree(src, exp):
    """Without nesting, opening order and closing order visit the rings alike: same output."""
    if ring_bonds(src) is None:
        pytest.skip("not a well-formed ring line: left unchanged by both readings")
    iv = ring_intervals(src)
    if _has_nesting(iv):
        pytest.skip("nested rings (or not a ring line): the readings may differ")
    assert _outer(src.encode()) == exp.encode()


def test_paper_example_under_both_readings():
    src = b"C1=CC=C(C=C1)C(=O)CC(=O)C2=CC=CC=C2"  # Sec. IV-A worked example (dibenzoylmethane)
    want = b"C0=CC=C(C=C0)C(=O)CC(=O)C0=CC=CC=C0"
    assert oracle.preprocess_line(src) == want
    assert _outer(src) == want


def test_nested_closed_form():
    """k rings nested like shells: labels count up from the outside in; the default counts from the inside."""
    for k in range(1, 11):
        src = "".join(f"C{j + 1 if j < 9 else '%' + str(j + 1)}" for j in range(k)) + "C"
        src += "".join(f"C{j + 1 if j < 9 else '%' + str(j + 1)}" for j in reversed(range(k)))
        want = "".join(f"C{j}" for j in range(k)) + "C" + "".join(f"C{j}" for j in reversed(range(k)))
        inner = "".join(f"C{k - 1 - j}" for j in range(k)) + "C" + "".join(f"C{k - 1 - j}" for j in reversed(range(k)))
        assert _outer(src.encode()).decode() == want, k
        assert oracle.preprocess_line(src.encode()).decode() == inner, k
    assert _outer(b"c1ccc2ccccc2c1") == b"c0ccc1ccccc1c0"


def test_two_digit_labels_when_needed():
    """Eleven nested rings under the opening-order reading: the innermost is written %10."""
    opens = "".join(f"C%{20 + k}" for k in range(11))
    closes = "".join(f"C%{20 + k}" for k in reversed(range(11)))
    out = _outer((opens + closes).encode()).decode()
    assert out == "C0C1C2C3C4C5C6C7C8C9C%10" + "C%10C9C8C7C6C5C4C3C2C1C0"


def test_graph_preserved():
    checked = 0
    for line in _sample_lines():
        before = ring_bonds(line.decode())
        after = ring_bonds(_outer(line).decode())
        assert before == after, line
        checked += before[1].total()
    assert checked > 1000


def test_idempotent_and_overlaps_distinct():
    for line in _sample_lines():
        p = _outer(line)
        assert _outer(p) == p
        iv = ring_intervals(p.decode())
        for i, (o1, c1, l1) in enumerate(iv):
            for o2, c2, l2 in iv[i + 1:]:
                if o1 < c2 and o2 < c1:
                    assert l1 != l2, line


def test_outer_ring_gets_lower_label():
    """Ring 2 nested in ring 1 with no ring closing between their openings: every label held when ring 1
    opened is still held when ring 2 opens, and so is ring 1's, so ring 2's label is above ring 1's. (A ring
    that closes in between frees its label, and the inner ring may take it: then the order can flip.)"""
    nested = 0
    for line in _sample_lines():
        iv = ring_intervals(_outer(line).decode())
        closes = sorted(c for _, c, _ in iv)
        for o1, c1, l1 in iv:
            for o2, c2, l2 in iv:
                if o1 < o2 and c2 < c1 and not any(o1 < c < o2 for c in closes):
                    nested += 1
                    assert l1 < l2, line
    assert nested > 50


def test_each_opening_takes_the_smallest_free_label():
    """Read off the output: a ring opening at o carries the smallest label held by no ring open at o."""
    for line in _sample_lines():
        iv = ring_intervals(_outer(line).decode())
        for o, c, lab in iv:
            held = {l2 for o2, c2, l2 in iv if o2 < o < c2}
            assert lab == min(set(range(101)) - held), line


def test_opening_order_uses_the_fewest_labels():
    """Greedy colouring of an interval graph in opening order is optimal (the rings already labelled and
    overlapping a new one all hold its opening point): the labels in use are exactly 0 .. (most rings open
    at once) - 1. Closing order has no such bound: the default reading may need more."""
    more = 0
    for line in _sample_lines():
        src = ring_intervals(line.decode())
        if not src:
            continue
        depth = max(sum(1 for o2, c2, _ in src if o2 <= o < c2) for o, _, _ in src)
        assert {l for _, _, l in ring_intervals(_outer(line).decode())} == set(range(depth)), line
        dflt = {l for _, _, l in ring_intervals(oracle.preprocess_line(line).decode())}
        assert len(dflt) >= depth
        more += len(dflt) > depth
    # e.g. CC6C(Cn6C)(C[nH]4n=nc4C(C)O(Oc9(c7cS2c9c5C76=C2ccn6C3c5c=ncc3CO(c1c1)))): closing order
    # labels it with 0..3, while at most three of its rings are open at once
    assert more > 0


def test_stream_and_compress_flags():
    raw = synth.generate(synth.CFG0, 2, 2000)
    lines = bytes(raw).split(b"\n")
    want = b"\n".join(_outer(l) for l in lines)
    assert bytes(oracle.preprocess_stream(raw, outer=True)) == want
    d = oracle.Dict(open(oracle_default_dict(), "rb").read())
    comp, idx = oracle.compress_stream(d, raw, oracle.PREPROCESS | oracle.PREPROCESS_OUTER)
    comp0, idx0 = oracle.compress_stream(d, np.frombuffer(want, dtype=np.uint8), 0)
    assert np.array_equal(comp, comp0) and np.array_equal(idx, idx0)
    with pytest.raises(oracle.OracleError):
        oracle.compress_stream(d, raw, oracle.PREPROCESS_OUTER)  # the modifier alone is refused


def oracle_default_dict():
    return os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2404_19391_gb300", "data", "zs_default.zsd")
