"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): ranks run
independent replicas, the job's time is the maximum over ranks, and the
reference arm under torchrun prints one line from rank 0 while the other
rank exits cleanly."""
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


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    r, w = bench.dist_setup()
    bench.barrier(w)
    m = bench.max_over_ranks(10.0 * (r + 1), w)
    bench.barrier(w)
    dist.destroy_process_group()
    with open(os.path.join(out, "rank%d.json" % r), "w") as fh:
        json.dump({"rank": r, "world": w, "max": m}, fh)


def test_max_over_ranks_with_gloo(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2,
                       join=True, start_method="spawn")
    got = [json.load(open(tmp_path / ("rank%d.json" % r))) for r in range(2)]
    assert [g["world"] for g in got] == [2, 2]
    assert [g["max"] for g in got] == [20.0, 20.0]


def test_reference_arm_under_torchrun():
    port = _free_port()
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run(
        [sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
         "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
         "--master-port", str(port), "bench.py", "--impl", "reference",
         "--gpus", "2", "--steps", "4", "--warmup", "3"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0
