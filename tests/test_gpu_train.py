"""GPU dictionary generation (Algorithm 1, Eq. 1) against the oracle's: the .zsd text must be identical byte
for byte, and the frozen default dictionary must come out of its own training set."""
import os

import numpy as np
import pytest

import oracle
import synth
from oracle import dictgen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def zs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19391_gb300 import zsmiles
    zsmiles.load_library()
    return zsmiles


def _dev(a: np.ndarray):
    return torch.from_numpy(np.array(a, dtype=np.uint8, copy=True)).cuda()


@pytest.mark.parametrize("lmax,no_alpha,pre", [(8, False, True), (5, False, True), (8, True, True), (8, False, False),
                                               (3, False, True)])
def test_matches_oracle(zs, lmax, no_alpha, pre):
    raw = synth.generate(synth.TRAIN, 0, 6000)
    text = oracle.preprocess_stream(raw) if pre else raw
    alphabet = b"" if no_alpha else dictgen.SMILES_ALPHABET
    want = dictgen.generate(text, T=146, lmin=2, lmax=lmax, alphabet=alphabet)
    got = zs.zs_train_dictionary(_dev(raw), zs.PREPROCESS if pre else 0, lmin=2, lmax=lmax, T=146,
                                 no_alphabet=no_alpha)
    assert got == want


def test_small_T_and_lmin(zs):
    raw = synth.generate(synth.TRAIN, 100, 2000)
    text = oracle.preprocess_stream(raw)
    for T, lmin in [(1, 2), (10, 3), (40, 2)]:
        want = dictgen.generate(text, T=T, lmin=lmin, lmax=6)
        assert zs.zs_train_dictionary(_dev(raw), zs.PREPROCESS, lmin=lmin, lmax=6, T=T) == want


def test_frozen_default_dictionary(zs):
    """The committed default dictionary is exactly what Algorithm 1 gives on its 100,000-line training set."""
    raw = synth.generate(synth.TRAIN, 0, synth.TRAIN_LINES)
    got = zs.zs_train_dictionary(_dev(raw), zs.PREPROCESS, lmin=2, lmax=8, T=146)
    assert got == open(os.path.join(ROOT, "paper_2404_19391_gb300", "data", "zs_default.zsd"), "rb").read()


def test_errors(zs):
    with pytest.raises(zs.ZsError) as e:
        zs.zs_train_dictionary(_dev(np.frombuffer(b"CC\x00C\n", dtype=np.uint8)), 0)
    assert e.value.status == zs.ERR_INVALID_ARG
    with pytest.raises(zs.ZsError) as e:
        zs.zs_train_dictionary(_dev(np.frombuffer(b"CCCC\n", dtype=np.uint8)), 0, lmax=9)
    assert e.value.status == zs.ERR_INVALID_ARG
    assert zs.zs_train_dictionary(torch.empty(0, dtype=torch.uint8, device="cuda"), 0, T=5) == \
        dictgen.dictionary_text([], dictgen.SMILES_ALPHABET, 2, 8)
