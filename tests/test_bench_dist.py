"""bench.py's multi-rank plumbing (replicas only): a world of 2 gloo ranks on
CPU agrees on the max and the sum over ranks and passes barriers."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    d = bench.Dist()
    d.barrier()
    mx = d.max(float(rank + 1) * 1.5)
    sm = d.sum(float(rank + 1))
    d.barrier()
    d.close()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{mx} {sm}")


def test_two_rank_max_and_sum(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        mx, sm = (float(x) for x in open(tmp_path / f"r{r}.txt").read().split())
        assert mx == 3.0 and sm == 3.0
