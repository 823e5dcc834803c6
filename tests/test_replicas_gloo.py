"""The multi-GPU path is replicas only (each rank searches its own beam, no
data-path collective): its host logic -- per-rank seeds, barrier, the slowest
rank's time, the whole-job rate -- checked with world_size 2 over gloo on the
CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["RANK"] = str(rank)
    os.environ["WORLD_SIZE"] = str(world)
    os.environ["LOCAL_RANK"] = str(rank)
    import bench
    r, w, local = bench.dist_setup(world)
    dist.init_process_group("gloo", rank=r, world_size=w)
    dist.barrier()
    ms = 10.0 + 5.0 * r                       # rank 1 is the slower one
    slowest = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.aggregate_rate(w, 1e12, slowest * 1e-3)
    q.put((r, local, bench.beam_seed(r), slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_over_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, l0, s0, t0, v0), (r1, l1, s1, t1, v1) = res
    assert (r0, r1) == (0, 1) and (l0, l1) == (0, 1)
    assert s0 != s1                              # each replica searches its own beam
    assert t0 == t1 == 15.0                      # both report the slowest rank's time
    assert v0 == v1 == pytest.approx(2 * 1e12 / 15e-3)


def test_single_process_defaults():
    import bench
    os.environ.pop("WORLD_SIZE", None)
    assert bench.dist_setup(1) == (0, 1, 0)
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    with pytest.raises(SystemExit):
        bench.dist_setup(2)
