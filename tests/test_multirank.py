"""The multi-rank path of bench.py on the CPU (gloo, world size 2): the timing is the slowest rank's on
every rank and the whole-job rate counts all ranks' work; under torchrun the reference arm prints one
line, from rank 0, and every rank exits 0.  The GPU path runs replicas with no data-path collective, so
the timing reduction is the only exchange between ranks."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = bench.max_over_ranks(times[rank], dist, "cpu")
    out[rank] = (ms, bench.whole_job_rate(world, 1000, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_timing_is_the_slowest_rank_and_the_rate_counts_every_rank():
    times = [12.5, 40.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, _free_port(), times, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (40.0, 2 * 1000 / 0.040)


def test_reference_arm_under_torchrun_prints_once():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(_free_port()), os.path.join(ROOT, "bench.py"), "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
