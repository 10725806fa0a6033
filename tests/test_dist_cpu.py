"""The multi-GPU bench path on CPU: world size 2 over gloo.  Every rank runs its own batch
(weak scaling, no collective on the data path); the only cross-rank step is the max over
ranks of the timed region, from which the job throughput is computed."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist

    import bench
    from paper_1806_07247_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    w, r, _ = bench.dist_env()
    ms = bench.max_over_ranks(100.0 + 50.0 * rank, torch.device("cpu"))
    specs = synth.batched_specs(16, seed=r)
    slices = sum(sp.n3 // 2 + 1 for sp in specs)
    total = bench.sum_over_ranks(slices, torch.device("cpu"))
    value = bench.job_throughput(total, 3, ms)
    out[rank] = (w, r, ms, slices, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_max_time_and_weak_scaling():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    (w0, r0, ms0, s0, v0), (w1, r1, ms1, s1, v1) = out[0], out[1]
    assert (w0, r0, w1, r1) == (2, 0, 2, 1)
    assert ms0 == ms1 == 150.0                     # the slowest rank's time on both
    assert s0 != s1                                # each rank draws its own batch (seed = rank)
    assert v0 == v1 == pytest.approx((s0 + s1) * 3 / 0.150)  # all ranks' units / max time
