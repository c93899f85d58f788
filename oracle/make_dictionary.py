"""Writes the frozen default dictionary with the oracle's Algorithm 1 (Sec. IV-C).

Training set: the 100,000-line seed-1 synthetic stream, pre-processed by the oracle (Sec. IV-A), with the
SMILES-alphabet pre-population (Sec. IV-B), L_min = 2 (Sec. IV-C), L_max = 8 (the middle of the paper's
{5, 8, 15} sweep, Sec. V-C) and T = 146 (every free symbol byte). Only ``oracle`` and the seeded input
generator are used.

    python -m oracle.make_dictionary [--lmax 8] [--out paper_2404_19391_gb300/data/zs_default.zsd]

The ablation dictionaries next to it vary one choice each (the paper's sweeps, Sec. V-C):

    python -m oracle.make_dictionary --lmax 5  --out paper_2404_19391_gb300/data/zs_lmax5.zsd
    python -m oracle.make_dictionary --lmax 15 --out paper_2404_19391_gb300/data/zs_lmax15.zsd
    python -m oracle.make_dictionary --no-alphabet --out paper_2404_19391_gb300/data/zs_no_alphabet.zsd
    python -m oracle.make_dictionary --no-preprocess --out paper_2404_19391_gb300/data/zs_raw_train.zsd

and one varies the reading of Sec. IV-A: the training lines are pre-processed with rings labelled in
opening order (the outermost of a nest gets the lower ID):

    python -m oracle.make_dictionary --outer --out paper_2404_19391_gb300/data/zs_outer_train.zsd

Table I's pre-population rows are {printable ASCII, SMILES alphabet, none}, each with and without
pre-processing. The printable pre-population takes every printable byte 0x21-0x7E as a single-character entry,
which leaves 0xA1-0xFF (95 symbols) for learned patterns:

    python -m oracle.make_dictionary --printable --out paper_2404_19391_gb300/data/zs_printable.zsd
    python -m oracle.make_dictionary --printable --no-preprocess --out paper_2404_19391_gb300/data/zs_printable_raw.zsd
    python -m oracle.make_dictionary --no-alphabet --no-preprocess \
        --out paper_2404_19391_gb300/data/zs_no_alphabet_raw.zsd
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if _ROOT not in sys.path:
    sys.path.insert(0, _ROOT)

import oracle  # noqa: E402
from oracle import dictgen  # noqa: E402
import synth  # noqa: E402


def build_default(lmax: int = 8, lmin: int = 2, T: int = 146, lines: int = synth.TRAIN_LINES,
                  alphabet: bytes = dictgen.SMILES_ALPHABET, preprocess: bool = True, outer: bool = False) -> bytes:
    raw = synth.generate(synth.TRAIN, 0, lines)
    pre = oracle.preprocess_stream(raw, outer=outer) if preprocess else raw
    return dictgen.generate(pre, T=T, lmin=lmin, lmax=lmax, alphabet=alphabet)


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--lmax", type=int, default=8)
    ap.add_argument("--T", type=int, default=146)
    ap.add_argument("--out", default=os.path.join(_ROOT, "paper_2404_19391_gb300", "data", "zs_default.zsd"))
    ap.add_argument("--no-alphabet", action="store_true", help="no pre-populated SMILES alphabet (Sec. IV-B)")
    ap.add_argument("--no-preprocess", action="store_true", help="train on lines without ring-ID renumbering")
    ap.add_argument("--outer", action="store_true", help="renumber ring IDs in opening order (outermost lower)")
    ap.add_argument("--printable", action="store_true",
                    help="pre-populate every printable byte (Table I 'Printable'); T is cut to the 95 free symbols")
    args = ap.parse_args()
    if args.printable and args.no_alphabet:
        ap.error("--printable and --no-alphabet exclude each other")
    alphabet = b"" if args.no_alphabet else (dictgen.PRINTABLE_ALPHABET if args.printable else dictgen.SMILES_ALPHABET)
    T = min(args.T, len(dictgen.code_space(alphabet)))
    text = build_default(lmax=args.lmax, T=T, alphabet=alphabet, preprocess=not args.no_preprocess,
                         outer=args.outer)
    with open(args.out, "wb") as f:
        f.write(text)
    print(args.out, len(text), hashlib.sha256(text).hexdigest())


if __name__ == "__main__":
    main()
