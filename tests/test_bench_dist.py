"""Multi-GPU host logic of bench.py on CPU: two gloo ranks shard the pairs
(weak scaling, no data-path collective) and reduce the timing (max) and the
work (sum) exactly as the GPU run does."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.dist_env()
    idx = bench.shard_pairs(256, r)
    t = bench.reduce_max(1.5 + r, w)
    n = bench.reduce_sum(float(len(idx)) * (r + 1), w)
    bench.barrier(w)
    q.put((r, idx[0], idx[-1], len(idx), t, n))
    dist.destroy_process_group()


def test_two_rank_sharding_and_reductions():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, a0, b0, n0, t0, s0), (r1, a1, b1, n1, t1, s1) = out
    assert (a0, b0, n0) == (0, 255, 256) and (a1, b1, n1) == (256, 511, 256)   # disjoint, weak scaling
    assert t0 == t1 == 2.5                                                       # max over ranks
    assert s0 == s1 == 256 * 1 + 256 * 2                                         # sum over ranks


def test_reference_arm_other_ranks_exit_quietly(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    assert bench.main(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]) == 0
    assert capsys.readouterr().out == ""
