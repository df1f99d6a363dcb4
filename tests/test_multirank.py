"""The benchmark's multi-rank plumbing on CPU with gloo (world size 2).

Molecules are independent, so N GPUs run N replicas on their own batches with
no collective on the data path; the only cross-rank operations are the
barrier and the max/sum of the timed region (the timing rule takes the
maximum over ranks).  This runs the host-side logic as two gloo ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b, w, M = bench.rank_batch(6, rank)
    mx = bench.max_over_ranks(10.0 + rank, dist)
    sm = bench.sum_over_ranks(b.n_atoms, dist)
    dist.barrier()
    out[rank] = (b.n_atoms, float(b.pos.sum()), mx, sm, int(w.size), M)
    dist.destroy_process_group()


def test_two_ranks_own_batches_and_reduce_timing():
    world = 2
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    r0, r1 = out[0], out[1]
    # each rank has its own molecules (weak scaling), same networks
    assert r0[1] != r1[1]
    assert r0[4] == r1[4] and r0[5] == r1[5] == 8
    # timing: max over ranks; atoms: summed for the whole-job throughput
    assert r0[2] == r1[2] == 11.0
    assert r0[3] == r1[3] == r0[0] + r1[0]
    # rank 0's batch is exactly workload 3's first molecules
    from paper_2201_08110_gb300 import workloads as W
    b, _, _ = W.config3(6)
    assert r0[0] == b.n_atoms and np.isclose(r0[1], float(b.pos.sum()))
