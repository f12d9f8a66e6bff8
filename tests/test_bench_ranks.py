"""The multi-GPU form of the benchmark is N independent replicas (rays are
independent; no collective on the data path): each rank times its own batch
and the job's numbers are the maximum over ranks of each arm's summed step
time, with aggregate rays/s = world * n * steps / that time.  This runs
that reduction as two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r ran 3 steps of (r + 1) ms on the first arm and 2 (r + 1) ms on the second
    arms = [[1.0 * (rank + 1)] * 3, [2.0 * (rank + 1)] * 3]
    totals, rates = bench.combine_ranks(arms, world, 1000, 3, dist, "cpu")
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(" ".join(repr(v) for v in totals + rates))
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_max_time(tmp_path):
    world = 2
    mp.spawn(rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world, join=True)
    rows = [list(map(float, open(tmp_path / f"r{r}.txt").read().split())) for r in range(world)]
    assert rows[0] == rows[1]                       # every rank agrees
    q, t, vq, vt = rows[0]
    assert q == 6.0 and t == 12.0                   # the slower rank's summed times
    assert vq == pytest.approx(world * 1000 * 3 / 6e-3) and vt == pytest.approx(world * 1000 * 3 / 12e-3)
