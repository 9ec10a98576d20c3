"""The multi-GPU path of bench.py is replicas only: every rank meshes its own
image, the job's time is the slowest rank's, and the job's throughput is all
ranks' units over that time.  The reduction runs here on two gloo ranks on
the CPU; the reference arm prints on rank 0 only."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, world: int, port: int, out_dir: str):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [3.0, 5.0][rank]  # the ranks' own step times
    ms_max = bench.max_over_ranks(ms, dist, "cpu")
    value = bench.job_rate(world, 1000.0, ms_max)
    with open(os.path.join(out_dir, "r%d.json" % rank), "w") as f:
        json.dump({"ms_max": ms_max, "value": value}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp

    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    for r in range(2):
        d = json.load(open(tmp_path / ("r%d.json" % r)))
        assert d["ms_max"] == 5.0  # the slowest rank's time on every rank
        assert d["value"] == pytest.approx(2 * 1000.0 / 5e-3)


def test_single_process_helpers():
    import bench

    assert bench.max_over_ranks(2.5, None, "cpu") == 2.5
    assert bench.job_rate(1, 500.0, 2.0) == pytest.approx(250000.0)


def test_reference_arm_prints_on_rank_zero_only(tmp_path):
    # the oracle arm under a world of two: rank 1 exits without output
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "disk64",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
    env["RANK"] = "0"
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "disk64",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0


def test_roofline_stage_skips_the_latency_bound_tier_g_stage():
    """The Tier-G stage runs beside the emission and is bound by latency:
    the HBM roofline entry describes the busiest byte-bound stage even when
    the Tier-G stage's event time is the longest."""
    import bench

    prof = {"k_emit": (13.1, 20), "k_tierg": (13.5, 80), "k_walk": (4.0, 40)}
    assert bench.roofline_stage(prof)[0] == "k_emit"
    prof = {"k_emit": (3.0, 20), "k_tierg": (13.5, 80), "k_cutcells": (4.5, 20)}
    assert bench.roofline_stage(prof)[0] == "k_cutcells"
