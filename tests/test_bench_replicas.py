"""The bench's multi-GPU mode runs independent replicas (no data-path
collective); its whole-job timing takes the slowest rank and the units of all
ranks.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, units = bench.job_timing(100.0 + 50.0 * rank, 1000.0 + rank, dist)
    q.put((rank, ms, units))
    dist.destroy_process_group()


def test_job_timing_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    out = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, units in out:
        assert ms == 150.0 and units == 2001.0


def test_job_timing_single_process():
    import bench
    assert bench.job_timing(12.5, 7) == (12.5, 7)


def test_roofline_traffic_comes_from_the_committed_profiles():
    # the bench's roofline.traffic reads dram_bytes_per_unit[<stage>] lines of
    # the ncu summaries under profiles/ (per-unit DRAM bytes of k_tc_pair for
    # S2 and S3, whose traffic is proportional to the units)
    import bench
    for stage in ("S2_G_x_X1", "S3_G_x_X2"):
        t, src = bench.captured_traffic(stage, 2.0)
        assert src is not None and src.startswith("k_tc_pair"), stage
        assert 1e9 < t / 2.0 < 3e9  # ~1.33 GB per unit at N = 96 (X in + out)
    assert bench.captured_traffic("no_such_stage", 1.0) == (None, None)
