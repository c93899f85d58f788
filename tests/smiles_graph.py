"""A small SMILES reader for tests: atoms in order, and ring bonds as atom-index pairs.

Independent of the oracle's pre-processing code (it never renumbers anything); it reads ring closures
the way SMILES defines them (Sec. II: a ring is written by cutting one bond and giving both atoms the
same numeric ID), so "pre-processed SMILES remain valid" (Sec. IV-A) can be checked as equality of the
molecular graph before and after.
"""
from __future__ import annotations

from collections import Counter

ORGANIC_TWO = ("Cl", "Br")
ORGANIC_ONE = set("BCNOPSFI" "bcnops" "*")
BONDS = set("-=#$:/\\")


def ring_bonds(smiles: str):
    """Returns (atom_count, Counter of (atom_a, atom_b, bond_char)) or None if the line is not a
    well-formed ring structure (unclosed ring or bracket)."""
    field = smiles.split(" ")[0].split("\t")[0]
    i, n = 0, len(field)
    atom = -1
    pending_bond = ""
    open_rings: dict[int, tuple[int, str]] = {}
    bonds: Counter = Counter()
    while i < n:
        c = field[i]
        if c == "[":
            j = field.find("]", i)
            if j < 0:
                return None
            atom += 1
            pending_bond = ""
            i = j + 1
        elif field.startswith(ORGANIC_TWO, i):
            atom += 1
            pending_bond = ""
            i += 2
        elif c in ORGANIC_ONE:
            atom += 1
            pending_bond = ""
            i += 1
        elif c in BONDS:
            pending_bond = c
            i += 1
        elif c.isdigit() or c == "%":
            if c == "%":
                if i + 2 >= n or not field[i + 1:i + 3].isdigit():
                    return None
                label = int(field[i + 1:i + 3])
                i += 3
            else:
                label = int(c)
                i += 1
            if label in open_rings:
                a, b0 = open_rings.pop(label)
                bond = pending_bond or b0
                bonds[(min(a, atom), max(a, atom), bond)] += 1
            else:
                open_rings[label] = (atom, pending_bond)
            pending_bond = ""
        else:
            i += 1
    if open_rings:
        return None
    return atom + 1, bonds


def ring_intervals(smiles: str):
    """(open_token, close_token, label) for each ring bond, tokens counted over ring labels only."""
    field = smiles.split(" ")[0].split("\t")[0]
    out, open_at, k, i = [], {}, 0, 0
    while i < len(field):
        c = field[i]
        if c == "[":
            i = field.find("]", i) + 1
            continue
        if c == "%":
            label, i = int(field[i + 1:i + 3]), i + 3
        elif c.isdigit():
            label, i = int(c), i + 1
        else:
            i += 1
            continue
        if label in open_at:
            out.append((open_at.pop(label), k, label))
        else:
            open_at[label] = k
        k += 1
    return out
