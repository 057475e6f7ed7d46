"""The multi-process path of bench.py on CPU (gloo, world size 2): the
barrier, the max over ranks and the whole-job throughput of independent
replicas, and the reference arm under torch.distributed.run (rank 0 alone
works and prints one line)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    d.init("gloo")
    d.barrier()
    ms = 100.0 + 50.0 * rank  # rank 1 is the slower replica
    value, ms_max = bench.replica_throughput(d, ms, evals_per_step=10**9, steps=4)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"world": d.world, "value": value, "ms_max": ms_max}, f)
    d.barrier()
    d.close()


def test_replicas_take_the_slowest_rank(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r in res:
        assert r["world"] == 2
        assert r["ms_max"] == 150.0
        # 2 ranks x 4 steps x 1e9 evaluations in the slower rank's 0.15 s
        assert abs(r["value"] - 2 * 4 * 1e9 / 0.15 / 1e9) < 1e-9


def test_single_process_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    d.world, d.rank = 1, 0
    d.init("gloo")
    assert d.pg is None
    value, ms_max = bench.replica_throughput(d, 200.0, evals_per_step=5 * 10**8, steps=2)
    assert ms_max == 200.0 and abs(value - 5.0) < 1e-12


def test_reference_arm_prints_one_line_from_rank_0():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "0"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
