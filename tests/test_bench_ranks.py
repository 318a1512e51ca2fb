"""The multi-rank path of bench.py on CPU (gloo, world size 2): the step time
is the maximum over the ranks, the rate counts the units of every rank, and
the reference arm prints from rank 0 only."""

import os
import socket
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms, rate = bench.whole_job(10.0 + 5.0 * rank, 1000 + rank, dist, "cpu")
    dist.destroy_process_group()
    with open(out + f".{rank}", "w") as f:
        f.write(f"{ms} {rate}\n")


def test_whole_job_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    out = str(tmp_path / "r")
    mp.start_processes(_rank_main, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
    got = [tuple(map(float, open(out + f".{r}").read().split())) for r in range(2)]
    for ms, rate in got:
        assert ms == 15.0                      # max over ranks
        assert abs(rate - 2001 / 0.015) < 1e-6 * rate   # units of both ranks / max time
    assert got[0] == got[1]


def test_whole_job_single_rank():
    sys.path.insert(0, ROOT)
    import bench
    ms, rate = bench.whole_job(20.0, 500, None, "cpu")
    assert ms == 20.0 and abs(rate - 25000.0) < 1e-9


def test_reference_arm_prints_from_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
