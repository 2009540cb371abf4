"""The multi-GPU path is replicas only (frames are independent): each rank simulates
its own frames and the run's time is the max over ranks.  The host side of that
(frame shares, the one collective) runs here as two gloo ranks on the CPU."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    share = bench.replica_inputs(rank, 8)
    t = bench.max_over_ranks(dist, 10.0 + rank)  # a rank's own elapsed time
    q.put((rank, share["image_seed"], list(map(int, share["philox_seeds"])), list(map(float, share["d_over_r0"])), t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_disjoint_frames_and_max_time():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, img0, seeds0, dr0, t0), (r1, img1, seeds1, dr1, t1) = res
    assert (r0, r1) == (0, 1)
    assert not set(seeds0) & set(seeds1)          # no frame simulated twice
    assert img1 - img0 == 8                       # consecutive image-seed blocks
    assert not np.allclose(dr0, dr1)
    assert t0 == t1 == 11.0                       # both ranks report the slowest rank's time
