"""The multi-process side of bench.py on CPU: two gloo ranks rendezvous on 127.0.0.1, take the
maximum of their times and draw different molecules (weak scaling, no shared data)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "PB_BENCH_BACKEND": "gloo"})
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist

    r, w, _ = bench.dist_setup(world)
    bench.barrier(w)
    m = bench.dist_max(1.5 + r, w)
    _, sizes = bench.batch_sizes(r, 4, 8000)
    out.put((r, w, m, [int(v) for v in sizes]))
    bench.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _, _ in res] == [0, 1]
    assert all(w == 2 for _, w, _, _ in res)
    assert all(m == 2.5 for _, _, m, _ in res)  # the slowest rank's time on both
    assert res[0][3] != res[1][3]  # each rank its own molecules
