"""Parity at the benchmark's full sizes, in the launch configurations bench.py times.

- The 10,000,000-line stream (config 1), one launch: the whole compressed stream, its line index and its
  decompression equal the CPU oracle's, which runs line-partitioned over the host threads.
- The 64-shard batch (config 2) through an autotuned, graph-captured plan, and the long-tail mix (config 3)
  at 20,000,000 lines through one launch: sampled lines. Lines are coded independently (Sec. I), so each
  sampled line's output must equal the oracle's encoding of that line alone, and random access to it must
  return the oracle's pre-processed line.
"""
import hashlib

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19391_gb300 import zsmiles
    zsmiles.load_library()
    data = open(zsmiles.DEFAULT_DICTIONARY, "rb").read()
    return zsmiles, zsmiles.Dictionary(data), oracle.Dict(data)


def _sha(a) -> bytes:
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).digest()


def _check_sampled_lines(zs, d, od, raw: np.ndarray, comp: torch.Tensor, idx: torch.Tensor, ids: np.ndarray):
    """Each sampled line's compressed bytes (from the line index) equal the oracle's encoding of that line
    alone; random access to the sampled lines returns the oracle's pre-processed lines."""
    raw_idx = oracle.line_index(raw)
    comp_np = comp.cpu().numpy()
    idx_np = idx.cpu().numpy().astype(np.uint64)
    want_dec = []
    for i in ids:
        line = bytes(raw[int(raw_idx[i]):int(raw_idx[i + 1])])
        nl = line.endswith(b"\n")
        body = line[:-1] if nl else line
        pre = oracle.preprocess_line(body)
        want = oracle.compress_line(od, pre) + (b"\n" if nl else b"")
        got = bytes(comp_np[int(idx_np[i]):int(idx_np[i + 1])])
        assert got == want, f"line {i}: {body[:60]!r}"
        want_dec.append(pre + b"\n")
    out, off, _ = zs.decompress_lines(d, comp, idx, torch.from_numpy(ids.astype(np.int64)).cuda())
    assert out.cpu().numpy().tobytes() == b"".join(want_dec)


def test_config1_whole_stream(env):
    zs, d, od = env
    raw = synth.generate(synth.CFG1, 0, synth.CFG1_LINES)
    comp, idx, r = zs.compress(d, torch.from_numpy(raw).cuda())
    assert r.n_lines == synth.CFG1_LINES
    exp_c, exp_i = oracle.compress_stream_parallel(od, raw, oracle.PREPROCESS)
    assert comp.numel() == exp_c.size and _sha(comp.cpu().numpy()) == _sha(exp_c)
    assert np.array_equal(idx.cpu().numpy().astype(np.uint64), exp_i)
    dec, rd = zs.decompress(d, comp)
    exp_d = oracle.preprocess_stream_parallel(raw)
    assert rd.out_len == exp_d.size and _sha(dec.cpu().numpy()) == _sha(exp_d)


def test_config2_batched_plan_sampled(env):
    zs, d, od = env
    specs = synth.batched_shards()
    raws = [synth.generate(shape, 0, count) for shape, count in specs]
    ins = [torch.from_numpy(r).cuda() for r in raws]
    outs = [torch.empty(zs.zs_compress_bound(r.size), dtype=torch.uint8, device="cuda") for r in raws]
    idxs = [torch.empty(c + 2, dtype=torch.int64, device="cuda") for _, c in specs]
    plan = zs.Plan(d, zs.OP_COMPRESS, list(zip(ins, outs, idxs)), flags=zs.PREPROCESS, variant=-1, tune_reps=1)
    res = plan.run()
    rng = np.random.default_rng(21)
    for k, ((_, count), r) in enumerate(zip(specs, res)):
        assert r.n_lines == count, f"shard {k}"
        ids = np.unique(np.concatenate([[0, count - 1], rng.integers(0, count, size=30)]))
        _check_sampled_lines(zs, d, od, raws[k], outs[k][: r.out_len], idxs[k][: r.n_lines + 1], ids)
    plan.close()


def test_config3_long_tail_sampled(env):
    zs, d, od = env
    n = 20_000_000
    raw = synth.generate(synth.CFG3, 0, n)
    comp, idx, r = zs.compress(d, torch.from_numpy(raw).cuda())
    assert r.n_lines == n
    lens = np.diff(oracle.line_index(raw).astype(np.int64))
    rng = np.random.default_rng(22)
    longest = np.argsort(lens)[-200:]  # the long tail, where the class-code and slow paths run
    ids = np.unique(np.concatenate([rng.integers(0, n, size=2000), longest, [0, n - 1]]))
    _check_sampled_lines(zs, d, od, raw, comp, idx, ids)
