"""The multi-GPU path of bench.py is replicas only: every rank runs its own copy of
the workload, no collective touches the data path, the timed region's length is
the maximum over ranks, and the whole-job value counts every rank's cells.  These
world-size-2 gloo runs check that host-side logic on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, local = bench.dist_info()
    local_ms = [120.0, 150.0][rank]  # the slower replica sets the timed region
    ms = bench.max_over_ranks(local_ms, w, "cpu")
    value = bench.replicas_value(2_097_152, 10, w, ms)
    # every rank builds the identical seeded replica of the workload
    from paper_2003_08374_gb300 import workloads as W
    case = W.grf_3d(shape=(16, 12, 10), seed=2, corr_len=3.0, frac_w=2)
    digest = float(case.permeability.sum() + case.porosity.sum())
    d = torch.tensor([digest], dtype=torch.float64)
    dmax, dmin = d.clone(), d.clone()
    dist.all_reduce(dmax, op=dist.ReduceOp.MAX)
    dist.all_reduce(dmin, op=dist.ReduceOp.MIN)
    # the reference arm runs on rank 0 only; the other ranks return at once
    class A:
        n, steps, warmup, gpus = 16, 1, 0, w
    ref_rc = bench.reference_arm(A) if r != 0 else 0
    out[rank] = (r, w, ms, value, float(dmax - dmin), ref_rc)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_all_cells():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    for rank in (0, 1):
        r, w, ms, value, spread, ref_rc = out[rank]
        assert (r, w) == (rank, 2)
        assert ms == 150.0
        assert value == pytest.approx(2_097_152 * 10 * 2 / 0.150)
        assert spread == 0.0
        assert ref_rc == 0
