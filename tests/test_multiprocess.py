"""The multi-process paths of bench.py, on the CPU with gloo (world size 2).

Under torchrun the benchmark splits its instance into z slabs (the exchange itself is
covered by tests/test_slab.py, on gloo ranks with oracle slabs) or, with --replicas,
runs independent copies; either way the job reports the particle-steps of all ranks over
the slowest rank's time.  These tests cover the reduction helpers that implement that,
and the reference arm under torchrun (rank 0 times the oracle and prints the one JSON
line, the other ranks exit without work).
"""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world), RANK=str(rank),
                      PIC_BENCH_GLOO="1")
    sys.path.insert(0, ROOT)
    import importlib.util

    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    r, w = bench.dist_init()
    bench.barrier(w)
    res = (r, w, bench.allreduce_max(float(rank + 1), w), bench.allreduce_sum(float(10 * (rank + 1)), w))
    import torch.distributed as dist

    dist.destroy_process_group()
    with open(os.path.join(out, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_bench_reductions_two_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp

    port = free_port()
    mp.spawn(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    for rank in (0, 1):
        r, w, mx, sm = json.load(open(tmp_path / f"rank{rank}.json"))
        assert (r, w) == (rank, 2)
        assert mx == 2.0 and sm == 30.0  # slowest rank's time, all ranks' work


def test_reference_arm_under_torchrun_prints_one_line():
    port = free_port()
    env = dict(os.environ, PIC_BENCH_GLOO="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus",
           "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
