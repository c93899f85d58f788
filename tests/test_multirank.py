"""The N>1 path of the benchmark on CPU: world size 2 over gloo. Each rank takes its own line range of the
synthetic stream (no data exchange, lines are independent, Sec. I); timings reduce by max and work by sum."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, lines, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist

    import bench
    import oracle
    import synth
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first = bench.rank_first_line(rank, lines)
        raw = synth.generate(synth.CFG1, first, lines)
        d = oracle.Dict(open(os.path.join(bench.ROOT, "paper_2404_19391_gb300", "data", "zs_default.zsd"),
                             "rb").read())
        comp, idx = oracle.compress_stream(d, raw, oracle.PREPROCESS)
        maxes, sums = bench.reduce_over_ranks([float(rank + 1), 10.0 * (world - rank)], [raw.size, comp.size],
                                              "cpu")
        q.put((rank, first, maxes, sums, comp.tobytes()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo():
    import multiprocessing as mp

    import oracle
    import synth
    lines, world = 1500, 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, lines, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    whole = synth.generate(synth.CFG1, 0, world * lines)
    d = oracle.Dict(open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                                      "paper_2404_19391_gb300", "data", "zs_default.zsd"), "rb").read())
    whole_comp, _ = oracle.compress_stream(d, whole, oracle.PREPROCESS)
    assert [g[1] for g in got] == [0, lines]  # disjoint consecutive ranges
    for _, _, maxes, sums, _ in got:  # every rank sees the same reduced values
        assert maxes == [2.0, 20.0]
        assert sums[0] == whole.size
        assert sums[1] == whole_comp.size
    # no exchange is needed: the ranks' outputs, concatenated, are the compression of the whole stream
    assert b"".join(g[4] for g in got) == whole_comp.tobytes()
    assert np.array_equal(np.frombuffer(b"".join(g[4] for g in got), np.uint8), whole_comp)
