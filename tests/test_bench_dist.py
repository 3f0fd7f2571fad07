"""bench.py's multi-rank logic on CPU: gloo, world size 2 (replicas, max time over ranks)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    bench.barrier(ws)
    t = bench.max_over_ranks(1.5 + rank, ws)  # each rank's step time
    out[rank] = t
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    port = _free_port()
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert out[0] == out[1] == 2.5


def test_single_rank_defaults(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_env() == (1, 0, 0)
    assert bench.max_over_ranks(3.25, 1) == 3.25
    assert bench.spmv_bytes(2, 3, 5) == 8 * 5 + 4 * 3 + 4 * 3 + 4 * 2


def test_bench_reads_traffic_from_the_committed_profile():
    """roofline.traffic comes from the committed ncu summary while it matches the kernel source."""
    import bench
    t = bench.profiled_traffic()
    if t is None:  # the kernels changed since the capture: the summary must say another hash
        assert "kernel_source_sha: " + bench.kernel_source_sha() not in open(bench.PROFILE_SUMMARY).read()
    else:
        assert 150_000_000 < t < 250_000_000
