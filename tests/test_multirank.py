"""The N > 1 path of bench.py, on the CPU: ranks are replicas (each fits its
own image, no collective on the data path); the only collective is the
job-wide aggregation after the timed region (max of the ranks' times, sum of
their work), exercised here with two gloo ranks.  The reference arm under
torchrun prints one line from rank 0; the other ranks exit 0 without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    ws, r, _ = bench.dist_init("gloo")
    # rank r: a step time of 1 + r seconds, 10 (r + 1) units of work
    res = bench.aggregate(1.0 + r, 10.0 * (r + 1), 2.0 + 0.5 * r, ws, device="cpu")
    q.put((r, res, bench.replica_seed(r)))
    torch.distributed.destroy_process_group()


def test_two_gloo_ranks_aggregate_max_time_and_total_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=180) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    by_rank = {r: (res, seed) for r, res, seed in out}
    for r in (0, 1):
        assert by_rank[r][0] == (2.0, 30.0, 2.5)
    assert by_rank[0][1] != by_rank[1][1]        # every rank fits its own image


def test_single_rank_aggregation_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(1.5, 7.0, 2.0, 1, device="cpu") == (1.5, 7.0, 2.0)


def test_reference_arm_under_torchrun_prints_one_line():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
           "--ref-crop", "32"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
