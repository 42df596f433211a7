"""Row-sharded evaluation across two processes (gloo, CPU): each rank
evaluates its row window with the CPU oracle, one all-reduce of 7 doubles
gives the whole, which must equal the unsharded oracle; and a rank that
fails before the collective is detected by the other rank's timeout instead
of a hang."""
import datetime
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _data():
    from paper_2407_11349_gb300 import synth
    return synth.grid_dataset(700, 50.0, 10, 10, seed=3)


def _worker(rank, world, port, out_path):
    import oracle
    from paper_2407_11349_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ds = _data()
    p = ds.params

    def evaluate(a, b):
        o = oracle.loglik_grad(ds.t, ds.x, ds.y, p, s=ds.s, row_begin=a, row_end=b, threads=1)
        return o[0], o[1:]

    ll, g = shard.sharded_loglik_grad(evaluate, ds.n, rank, world)
    if rank == 0:
        np.save(out_path, np.concatenate([[ll], g]))
    dist.destroy_process_group()


def _failing_worker(rank, world, port, out_path):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))
    if rank == 1:
        raise SystemExit(3)  # this rank dies before its collective
    t = torch.ones(7, dtype=torch.float64)
    try:
        dist.all_reduce(t)
        status = "completed"
    except Exception as e:  # the surviving rank learns of the failure
        status = "error: " + type(e).__name__
    with open(out_path, "w") as f:
        f.write(status)
    # Leave without running the broken process group's destructors: gloo's
    # teardown after a lost peer can abort the process, which is not what
    # this test is about (the status above is).
    os._exit(0)


def test_row_bounds_partition():
    from paper_2407_11349_gb300 import shard
    for n, w in ((10, 3), (1, 4), (1_000_000, 8)):
        b = shard.row_bounds(n, w)
        assert b[0][0] == 0 and b[-1][1] == n
        assert all(b[k][1] == b[k + 1][0] for k in range(w - 1))
        sizes = [e - a for a, e in b]
        assert max(sizes) - min(sizes) <= 1


def _symmetric_worker(rank, world, port, out_path):
    """Each rank evaluates the rows of its symmetric shard (bounds from the
    library's host-only partition) with the CPU oracle; one all-reduce of 7
    doubles gives the whole."""
    import oracle
    from paper_2407_11349_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ds = _data()
    b = shard.symmetric_row_bounds(ds.n, 128, world)
    o = oracle.loglik_grad(ds.t, ds.x, ds.y, ds.params, s=ds.s, row_begin=int(b[rank]),
                           row_end=int(b[rank + 1]), threads=1)
    t = torch.tensor(o, dtype=torch.float64)
    dist.all_reduce(t)
    if rank == 0:
        np.save(out_path, t.numpy())
    dist.destroy_process_group()


def test_symmetric_bounds_balance_pairs():
    """Whole row tiles, covering [0, n) in order, each shard's pairs (i, j < i)
    within one tile's worth of an equal share."""
    from paper_2407_11349_gb300 import shard
    for n, tr, w in ((1_000_000, 2048, 2), (1_000_000, 2048, 4), (1_000_000, 1024, 8), (250_000, 2048, 3),
                     (5000, 2048, 4), (1, 2048, 2)):
        b = shard.symmetric_row_bounds(n, tr, w)
        assert b[0] == 0 and b[-1] == n and np.all(np.diff(b) >= 0)
        assert np.all(b[1:-1] % tr == 0)
        pairs = np.array([(e - a) * (a + e - 1) / 2 for a, e in zip(b[:-1], b[1:])])
        total = n * (n - 1) / 2
        last_tile = tr * n  # pairs of the largest row tile
        assert np.all(np.abs(pairs - total / w) <= last_tile), (n, w, pairs)
        if n >= 8 * tr * w:  # boundaries near n sqrt(g / G)
            want = n * np.sqrt(np.arange(w + 1) / w)
            assert np.all(np.abs(b - want) <= tr)


def test_two_rank_symmetric_shard_rows_sum_to_whole(tmp_path):
    import oracle
    out = str(tmp_path / "sym.npy")
    mp.spawn(_symmetric_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    ds = _data()
    ref = oracle.loglik_grad(ds.t, ds.x, ds.y, ds.params, s=ds.s)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)


def test_two_rank_sharded_sum_equals_whole(tmp_path):
    import oracle
    out = str(tmp_path / "sum.npy")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    ds = _data()
    ref = oracle.loglik_grad(ds.t, ds.x, ds.y, ds.params, s=ds.s)
    assert np.allclose(got, ref, rtol=1e-12, atol=0)


def test_dead_rank_is_detected_by_timeout(tmp_path):
    out = str(tmp_path / "status.txt")
    ctx = mp.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=60)
    assert procs[1].exitcode == 3
    assert procs[0].exitcode == 0
    assert open(out).read().startswith("error")
