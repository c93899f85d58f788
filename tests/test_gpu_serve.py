"""GPU tests of the serving form: continuous batching of random-access requests over a resident store.
Every request's result must be byte-identical to the same request served alone (zs_decompress_lines)
and to the CPU oracle, however it was batched with others."""
import threading

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_LINES = 20000


@pytest.fixture(scope="module")
def zs():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2404_19391_gb300 import zsmiles
    zsmiles.load_library()
    return zsmiles


@pytest.fixture(scope="module")
def store(zs):
    data = open(zs.DEFAULT_DICTIONARY, "rb").read()
    d, od = zs.Dictionary(data), oracle.Dict(data)
    raw = synth.generate(synth.CFG4, 0, N_LINES)
    comp, idx, r = zs.compress(d, torch.from_numpy(raw).cuda())
    assert r.n_lines == N_LINES
    return d, od, comp, idx, comp.cpu().numpy(), idx.cpu().numpy().astype(np.uint64)


def _alone(zs, store, ids):
    d, _, comp, idx, _, _ = store
    out, off, _ = zs.decompress_lines(d, comp, idx, torch.from_numpy(ids.astype(np.int64)).cuda())
    return out.cpu().numpy().tobytes(), off.cpu().numpy().astype(np.uint64)


def _requests(n, seed, max_ids=3000):
    return [ids for _, ids in synth.requests(n, seed, N_LINES, max_ids=max_ids)]


def test_same_alone_and_in_the_mix(zs, store):
    d, od, comp, idx, comp_np, idx_np = store
    # a large first request keeps the single slot busy while the others queue up behind it, so they
    # share the next launches
    big = np.random.default_rng(4).integers(0, N_LINES, size=200_000).astype(np.uint64)
    reqs = [big] + _requests(60, 1)
    srv = zs.Server(d, comp, idx, max_inflight=1)
    tickets = [srv.submit(ids) for ids in reqs]
    for k, (t, ids) in enumerate(zip(tickets, reqs)):
        got, off = srv.fetch(t)
        want, want_off = _alone(zs, store, ids)
        assert got == want, f"request {k}"
        assert np.array_equal(off, want_off), f"request {k}"
        if k % 10 == 0:
            o_out, o_off = oracle.decompress_lines(od, comp_np, idx_np, ids)
            assert got == o_out.tobytes() and np.array_equal(off, o_off)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["submitted"] == len(reqs)
    assert st["mean_batch_requests"] > 1.0, st  # requests really were batched together
    assert st["ids"] == sum(len(i) for i in reqs)
    srv.close()


def test_many_client_threads(zs, store):
    d = store[0]
    srv = zs.Server(d, store[2], store[3], max_inflight=4)
    errors = []

    def client(seed):
        try:
            for ids in _requests(15, 100 + seed, max_ids=2000):
                got, off = srv.fetch(srv.submit(ids))
                want, want_off = _alone(zs, store, ids)
                if got != want or not np.array_equal(off, want_off):
                    errors.append(seed)
        except Exception as e:  # noqa: BLE001
            errors.append(repr(e))

    th = [threading.Thread(target=client, args=(s,)) for s in range(6)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errors
    srv.close()


def test_small_arena_admits_by_memory(zs, store):
    """An arena that holds only a few requests at once: the queue head waits for room, results unchanged."""
    d = store[0]
    reqs = _requests(40, 7, max_ids=400)
    srv = zs.Server(d, store[2], store[3], arena_bytes=256 << 10, max_batch_ids=1024, max_inflight=2)
    tickets = [srv.submit(ids) for ids in reqs]
    for t, ids in zip(tickets, reqs):
        got, off = srv.fetch(t)
        want, want_off = _alone(zs, store, ids)
        assert got == want and np.array_equal(off, want_off)
    assert srv.stats()["batches"] > 1
    srv.close()


def test_requests_are_checked(zs, store):
    d = store[0]
    srv = zs.Server(d, store[2], store[3], arena_bytes=16 << 10, max_batch_ids=500)
    with pytest.raises(zs.ZsError) as e:
        srv.submit(np.array([1, N_LINES], dtype=np.uint64))
    assert e.value.status == zs.ERR_INVALID_ARG
    with pytest.raises(zs.ZsError) as e:
        srv.submit(np.arange(501, dtype=np.uint64))
    assert e.value.status == zs.ERR_INVALID_ARG
    with pytest.raises(zs.ZsError) as e:
        srv.submit(np.zeros(500, dtype=np.uint64) + 3)  # 500 copies of one line: bound above 16 KiB
    assert e.value.status in (zs.ERR_CAPACITY,)
    t = srv.submit(np.zeros(0, dtype=np.uint64))
    got, off = srv.fetch(t)
    assert got == b"" and off.tolist() == [0]
    with pytest.raises(zs.ZsError):
        srv.fetch(t)  # forgotten after the fetch
    srv.close()


def test_repeated_and_duplicate_ids(zs, store):
    d = store[0]
    srv = zs.Server(d, store[2], store[3])
    ids = np.array([5, 5, 0, N_LINES - 1, 5, 17], dtype=np.uint64)
    got, off = srv.fetch(srv.submit(ids))
    want, want_off = _alone(zs, store, ids)
    assert got == want and np.array_equal(off, want_off)
    srv.close()


def test_open_loop_replay_and_serial_baseline(zs, store):
    d, _, comp, idx, _, _ = store
    reqs = synth.requests(200, 3, N_LINES, max_ids=2000, rate=20000.0)
    srv = zs.Server(d, comp, idx)
    lat, mk = srv.replay(reqs)
    assert lat.shape == (200,) and np.all(lat >= 0) and mk > 0
    st = srv.stats()
    assert st["completed"] == 200
    srv.close()
    lat2, mk2 = zs.zs_serial_replay(d, comp, idx, reqs)
    assert lat2.shape == (200,) and np.all(lat2 >= 0) and mk2 > 0


def test_close_with_queued_requests(zs, store):
    d = store[0]
    srv = zs.Server(d, store[2], store[3], max_inflight=1)
    for ids in _requests(20, 9):
        srv.submit(ids)
    srv.close()  # must not hang
