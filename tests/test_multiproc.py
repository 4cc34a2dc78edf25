"""The multi-rank host logic of bench.py on CPU: world size 2 over gloo.
Each rank works on its own pairs (no data-path collective); the timing takes
a barrier and the max over ranks, and the value counts every rank's work."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import sys
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    import synth
    ws2, r2, _ = bench.dist_env()
    assert (ws2, r2) == (ws, rank)
    bench.init_dist(ws, "gloo")
    bench.barrier(ws)
    # every rank times its own work; the slowest rank sets the job time
    my_ms = 10.0 + 5.0 * rank
    mx = bench.max_over_ranks(my_ms, ws)
    seeds = [bench.rank_seed(rank, i, 16) for i in range(3)]
    pair = synth.config_pair("plain_320x240", seed=bench.rank_seed(rank))
    q.put((rank, mx, seeds, int(pair.left.sum())))
    dist.destroy_process_group()


def test_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = {}
    for _ in range(2):
        r, mx, seeds, s = q.get(timeout=120)
        out[r] = (mx, seeds, s)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 15.0            # max over ranks
    assert set(out[0][1]).isdisjoint(out[1][1])      # independent pairs per rank
    assert out[0][2] != out[1][2]                    # different inputs
    import bench
    assert bench.aggregate_value(2, 640 * 480, 10, 15.0) == pytest.approx(2 * 640 * 480 * 10 / 0.015 / 1e6)
