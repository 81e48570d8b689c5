"""The bench's multi-GPU bookkeeping on two gloo ranks (CPU): replicas, max-over-ranks time, rank-0-only reference."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch
    import bench
    r, w, pg = bench.dist_setup(world)
    assert (r, w) == (rank, world) and pg is not None
    # rank r pretends its timed region took 1 + r seconds for 10 steps of 100 interactions
    value, tmax = bench.aggregate(pg, w, 100.0, 10, 1.0 + r, torch.device("cpu"))
    bench.barrier(pg)

    class A:
        steps, warmup = 1, 0
    ref = bench.run_reference(A, r, w, pg) if r != 0 else None
    with open(os.path.join(out_dir, f"rank{r}.txt"), "w") as f:
        f.write(f"{value} {tmax} {ref is None}\n")
    pg.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, 2, port, str(tmp_path))) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    vals = [open(tmp_path / f"rank{r}.txt").read().split() for r in range(2)]
    for v in vals:
        assert float(v[1]) == 2.0                    # the slowest rank's time
        assert float(v[0]) == 2 * 100.0 * 10 / 2.0  # all ranks' interactions over it
    assert vals[1][2] == "True"                      # the reference arm runs on rank 0 only
