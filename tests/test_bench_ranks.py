"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): ranks run
independent channels (weak scaling), the timed region is the slowest rank's,
and only rank 0 prints."""
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


def _worker(rank, ws, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    dist, r, n, local = bench._dist()
    assert (r, n, local) == (rank, ws, rank) and dist.get_backend() == "gloo"
    # rank r took (r + 1) * 10 ms: the job is timed by the slowest rank
    ms_max = bench._max_over_ranks(dist, 10.0 * (rank + 1))
    value = bench._weak_value(n, 1000, 50, ms_max)
    dist.barrier()
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"ms_max": ms_max, "value": value}, fh)
    dist.destroy_process_group()


def test_max_over_ranks_and_weak_value_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    if not torch.distributed.is_available():
        pytest.skip("torch.distributed unavailable")
    ws, port = 2, _free_port()
    mp.spawn(_worker, args=(ws, port, str(tmp_path)), nprocs=ws, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(ws)]
    for r in res:
        assert r["ms_max"] == 20.0
        # two ranks x 1000 nodes x 50 steps in 20 ms
        assert r["value"] == pytest.approx(2 * 1000 * 50 / 0.020 / 1e9)


def test_reference_arm_prints_one_line_under_torchrun():
    pytest.importorskip("torch")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "2", "--warmup", "3"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0
