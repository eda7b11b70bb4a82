"""Multi-GPU placement of independent work (bench.py --workload batched / serving under
torchrun): the domains of a batch are dealt to the ranks by cell count, the requests of a
serving trace round robin; each rank advances only its own share, and only host-side
statistics (timing, latencies, counts) cross ranks.  World-size-2 gloo runs check that
logic on the CPU."""
import os
import socket

import numpy as np
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
    from paper_2003_08374_gb300 import workloads as W
    # every rank builds the same seeded global set and keeps its share
    cases = W.batched_domains(count=10 * world, seed=4, lo3=6, hi3=14, lo2=8, hi2=24)
    cells = [c.cells for c in cases]
    mine = bench.shard_by_cells(cells, world)[rank]
    everyone = bench.gather_lists(mine, world)
    loads = bench.gather_lists([sum(cells[i] for i in mine)], world)
    # serving: requests round robin in arrival order; latencies gathered on the host
    trace = W.poisson_requests(rate=40.0, duration=1.0, seed=5, lo=8, hi=16)
    my_reqs = [i for i in range(len(trace)) if i % world == rank]
    lat = bench.gather_lists([float(i) for i in my_reqs], world)
    ms = bench.max_over_ranks([80.0, 95.0][rank], world, "cpu")
    out[rank] = (sorted(everyone), loads, max(cells), len(cases), sorted(lat), len(trace), ms)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_share_domains_and_requests_without_overlap():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    assert sorted(out.keys()) == [0, 1]
    for rank in (0, 1):
        everyone, loads, biggest, ncases, lat, ntrace, ms = out[rank]
        assert everyone == list(range(ncases))  # every domain on exactly one rank
        assert abs(loads[0] - loads[1]) <= biggest  # balanced by cells to within one domain
        assert lat == [float(i) for i in range(ntrace)]  # every request served once, all latencies gathered
        assert ms == 95.0  # the slower rank sets the timed region


def test_shard_by_cells_is_deterministic_and_balanced():
    import bench
    rng = np.random.default_rng(0)
    cells = [int(x) for x in rng.integers(1, 1000, 37)]
    for world in (1, 2, 3, 8):
        parts = bench.shard_by_cells(cells, world)
        assert parts == bench.shard_by_cells(cells, world)
        assert sorted(i for p in parts for i in p) == list(range(len(cells)))
        loads = [sum(cells[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(cells)


def test_all_cores_oracle_baseline_runs_one_serial_process_per_core():
    """The all-cores CPU baseline: one oracle process per host core, each on its own slab,
    timed together; the aggregate rate counts every process's cells over the slowest one's
    time (so it cannot exceed cores x the fastest single process)."""
    import os
    import bench
    value, cores, secs = bench.time_oracle_all_cores(24, 1)
    assert cores == (os.cpu_count() or 1)
    assert value > 0 and secs > 0
    one, _ = bench.time_oracle(bench.slab_of(bench.workload(24)), 1, 0)
    assert value <= cores * one * 3
