"""The N > 1 path of bench.py on CPU: ranks are independent replicas (no data-path collective);
the job's time is the slowest rank's and its value counts every rank's work. Two gloo ranks run
the cross-rank step, and two torchrun ranks run the reference arm (rank 0 alone reports)."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r took 1 + r seconds for 100 units
        t, value = bench.combine_over_ranks(1.0 + rank, 100.0, dist, "cpu")
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump({"t": t, "value": value}, f)
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_rank_and_value_counts_all_ranks(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_rank_main, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       start_method="spawn", join=True)
    for r in range(ws):
        got = json.load(open(tmp_path / f"rank{r}.json"))
        assert got["t"] == 2.0                 # max over ranks
        assert got["value"] == 2 * 100.0 / 2.0  # all ranks' units over the job's time


def test_one_rank_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.combine_over_ranks(0.5, 10.0) == (0.5, 20.0)


def test_reference_arm_under_two_ranks_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1",
           "--warmup", "0", "--cpu-seconds", "0.5"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0
