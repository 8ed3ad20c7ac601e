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


def test_reference_arm_line_carries_the_contract_keys():
    # the reference arm times the CPU oracle on the host cores and prints one
    # JSON line with the same metric, config and unit as the GPU arm, marked
    # impl=reference, with its cpu_baseline and an e2e block of zero copies
    # (a small basis here so that the check takes seconds)
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                        "--warmup", "0", "--N", "6"], cwd=root, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads([x for x in r.stdout.splitlines() if x.startswith("{")][-1])
    import bench
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "TFLOP/s" and line["higher_is_better"] is True
    assert line["steps"] == 1 and line["warmup"] == 0 and line["n_gpus"] == 1
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert line["config"]["N"] == 6 and line["config"]["workload"].startswith("gkba2b_heun_step")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert cb["sample"]
    e2e = line["e2e"]
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
