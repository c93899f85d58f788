"""Dictionary generation, Algorithm 1 with the rank of Eq. 1 (Sec. IV-C), and pre-population (Sec. IV-B).

TEST INFRASTRUCTURE ONLY (part of the CPU oracle): it produces the frozen dictionary file that both the
oracle and the CUDA library load, and it is pinned by tests against a naive recomputation.

Algorithm 1, as read here:
  1. D starts as the pre-populated single characters C (the SMILES alphabet, Sec. IV-B).
  2. Count every occurrence (overlapping occurrences count) of every substring s of every pre-processed
     training line with L_min <= |s| <= L_max (substrings holding the reserved bytes ' ' or '\\n' are
     skipped: they can never be patterns).
  3. T times: take the substring of highest rank_{p,t} = occ_p * (l_p - overlap_{p,t}) (Eq. 1), add it to
     D, remove it from the candidates. The paper's loop over t in {0..T} picks T patterns (the extra
     iteration is read as an off-by-one), and stops early once the best rank is <= 0.
  4. overlap_{p,t} (only described as "the overlap with patterns selected in previous iterations") is
     read as the maximum over the already-selected patterns w (not the pre-populated singles) of:
     |p| if p occurs inside w; else |w| if w occurs inside p; else the longest proper suffix of one
     that is a prefix of the other (either order); else 0.
  5. Ties: higher occ, then longer, then bytewise smaller.
Symbols are assigned in pick order, in ascending byte order, from the code space left after the
alphabet: printable ASCII 0x21-0x7E outside the alphabet, then 0xA1-0xFF (readable output, Sec. I).
"""
from __future__ import annotations

import heapq
from collections import Counter

import numpy as np

#: pre-populated SMILES alphabet (Sec. IV-B): digits, bond/branch/bracket/charge/chirality marks, the
#: organic-subset element letters, the second letters of Cl and Br, and the aromatic atoms.
SMILES_ALPHABET = b"0123456789()[]=#$:/\\.+-@%*BCNOPSFIHlrbcnops"
#: printable ASCII pre-population variant (Table I "Printable")
PRINTABLE_ALPHABET = bytes(range(0x21, 0x7F))
RESERVED = (ord("\n"), ord(" "))


def code_space(alphabet: bytes) -> list[int]:
    """Symbol bytes available to learned patterns, ascending."""
    a = set(alphabet)
    return [b for b in range(0x21, 0x7F) if b not in a] + [b for b in range(0xA1, 0x100) if b not in a]


def count_substrings(lines, lmin: int, lmax: int) -> Counter:
    """Occurrences of every substring with lmin <= len <= lmax (Algorithm 1, counting loop)."""
    occ: Counter = Counter()
    for line in lines:
        n = len(line)
        for i in range(n):
            for l in range(lmin, min(lmax, n - i) + 1):
                s = line[i:i + l]
                if 32 in s or 10 in s:
                    continue
                occ[s] += 1
    return occ


def count_substrings_fast(stream: np.ndarray, lmin: int, lmax: int) -> Counter:
    """Same counts as count_substrings over the lines of a '\\n'-separated stream, using np.unique over
    sliding windows (windows holding '\\n' or ' ' are dropped, so lines never run together)."""
    a = np.ascontiguousarray(stream, dtype=np.uint8)
    n = a.size
    occ: Counter = Counter()
    bad = ((a == 10) | (a == 32)).astype(np.int64)
    bad_prefix = np.concatenate([[0], np.cumsum(bad)])
    for l in range(lmin, lmax + 1):
        if n < l:
            break
        m = n - l + 1
        ok = (bad_prefix[l:l + m] - bad_prefix[:m]) == 0
        starts = np.flatnonzero(ok)
        if starts.size == 0:
            continue
        win = np.lib.stride_tricks.sliding_window_view(a, l)[starts]
        keys = np.ascontiguousarray(win).view(np.dtype((np.void, l))).ravel()
        uniq, counts = np.unique(keys, return_counts=True)
        for k, c in zip(uniq, counts):
            occ[bytes(k)] += int(c)
    return occ


def overlap(p: bytes, w: bytes) -> int:
    if p in w:
        return len(p)
    if w in p:
        return len(w)
    best = 0
    for k in range(1, min(len(p), len(w))):
        if p[-k:] == w[:k] or w[-k:] == p[:k]:
            best = k
    return best


def rank(p: bytes, occ: int, selected: list[bytes]) -> int:
    """Eq. 1: occ_p * (l_p - overlap_{p,t})."""
    ov = max((overlap(p, w) for w in selected), default=0)
    return occ * (len(p) - ov)


def _key(p: bytes, r: int, occ: int):
    # smallest tuple = highest rank, then higher occ, then longer, then bytewise smaller
    return (-r, -occ, -len(p), p)


def select_naive(occ: Counter, T: int) -> list[bytes]:
    """Algorithm 1 selection loop, recomputing every rank at every step."""
    cand = dict(occ)
    selected: list[bytes] = []
    for _ in range(T):
        if not cand:
            break
        best = min(cand, key=lambda p: _key(p, rank(p, cand[p], selected), cand[p]))
        if rank(best, cand[best], selected) <= 0:
            break
        selected.append(best)
        del cand[best]
    return selected


def select_lazy(occ: Counter, T: int) -> list[bytes]:
    """The same selection with a lazily re-evaluated max-heap. Ranks never rise as D grows (overlap is a
    max over a growing set), so a stored key bounds the current one and the first popped entry whose
    re-evaluated key still beats the heap top is the exact argmax."""
    heap = [_key(p, c * len(p), c) for p, c in occ.items()]
    heapq.heapify(heap)
    selected: list[bytes] = []
    while heap and len(selected) < T:
        top = heapq.heappop(heap)
        p = top[3]
        c = -top[1]
        cur = _key(p, rank(p, c, selected), c)
        if heap and cur > heap[0]:
            heapq.heappush(heap, cur)
            continue
        if -cur[0] <= 0:
            break
        selected.append(p)
    return selected


def dictionary_text(patterns: list[bytes], alphabet: bytes, lmin: int, lmax: int) -> bytes:
    """Serialise D as a .zsd file: header, alphabet (identity entries), then symbol/pattern pairs."""
    space = code_space(alphabet)
    if len(patterns) > len(space):
        raise ValueError("more patterns than free symbol bytes")
    out = [b"ZSDICT 1", f"{lmin} {lmax} {len(patterns)}".encode(),
           b"alphabet " + (alphabet.hex().encode() if alphabet else b"-")]
    for sym, p in zip(space, patterns):
        out.append(f"{sym:02x} {p.hex()}".encode())
    return b"\n".join(out) + b"\n"


def generate(lines_or_stream, T: int, lmin: int = 2, lmax: int = 8, alphabet: bytes = SMILES_ALPHABET,
             lazy: bool = True) -> bytes:
    """Train a dictionary on already pre-processed lines (a list of bytes, or a '\\n'-separated stream)."""
    if isinstance(lines_or_stream, np.ndarray):
        occ = count_substrings_fast(lines_or_stream, lmin, lmax)
    else:
        occ = count_substrings(lines_or_stream, lmin, lmax)
    T = min(T, len(code_space(alphabet)))
    pats = (select_lazy if lazy else select_naive)(occ, T)
    return dictionary_text(pats, alphabet, lmin, lmax)
