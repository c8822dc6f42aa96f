"""Multi-GPU form of the benchmark: independent replicas (the fit has no
data-path collective), one process per GPU, the step time taken as the
maximum over ranks.  Exercised here on CPU with two gloo ranks."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench._dist()
    assert (ws, r, local) == (world, rank, rank)
    # each replica times its own step; the slowest one is the job's time
    got = bench.max_over_ranks(1.5 + rank, ws, device="cpu")
    # the reference arm runs on rank 0 only; other ranks exit 0 without work
    ref_rc = None
    if rank != 0:
        class A:
            warmup = 1
            steps = 1
            gpus = world
        ref_rc = bench.run_reference(A())
    dist.barrier()
    dist.destroy_process_group()
    out.put((rank, got, ref_rc))


@pytest.mark.parametrize("world", [2])
def test_max_over_ranks_and_rank0_only_reference(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g for _, g, _ in res] == [1.5 + world - 1] * world
    assert [rc for r, _, rc in res if r != 0] == [0] * (world - 1)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.25, 1) == 3.25
