"""The multi-GPU path of the benchmark is independent replicas: every rank
propagates its own problem and only the timing is combined (the slowest
rank's time; value = all ranks' units over it).  That host-side logic runs
here with two gloo ranks on the CPU (no GPU, no collective on any data)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      LOCAL_RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, local, w = bench.dist_env()
    t_local = 1.0 + 0.5 * rank             # rank 1 is the slow one
    slowest = bench.max_over_ranks(t_local, w, dist, "cpu")
    rate = bench.job_rate(100.0, t_local, w, dist, "cpu")
    with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
        f.write("%d %d %d %r %r\n" % (r, local, w, slowest, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_combine_only_the_timing(tmp_path):
    ctx = torch.multiprocessing.get_context("spawn")
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        rr, local, w, slowest, rate = open(tmp_path / ("rank%d.txt" % r)).read().split()
        assert (int(rr), int(local), int(w)) == (r, r, 2)
        assert float(slowest) == 1.5
        assert abs(float(rate) - 2 * 100.0 / 1.5) < 1e-12


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(2.5, 1, None, "cpu") == 2.5
    assert bench.job_rate(10.0, 2.0, 1, None, "cpu") == 5.0
