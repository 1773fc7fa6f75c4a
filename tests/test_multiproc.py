"""The N > 1 path of bench.py on CPU: two gloo ranks run the barrier and the
max / sum reductions that turn per-rank timings and counts into the
whole-job value (units all ranks processed / slowest rank's time), every
rank runs its own chain (distinct seeds, no data-path collective), and under
torchrun only rank 0 prints the reference arm's line."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, _ = bench.dist_setup()
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    ms = 100.0 + 50.0 * r          # per-rank timed milliseconds
    accepted = 3 + r                # per-rank accepted updates
    ms_max = bench.allmax(w, ms)
    total = bench.allsum(w, accepted)
    value = total / (ms_max * 1e-3)
    q.put((r, w, ms_max, total, value, bench.SEED + 1 + 1000 * r))
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, m0, t0, v0, s0), (r1, w1, m1, t1, v1, s1) = out
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert m0 == m1 == 150.0 and t0 == t1 == 7.0
    assert v0 == v1 == pytest.approx(7.0 / 0.150)
    assert s0 != s1


def test_reference_arm_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--workload", "4^4", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["cpu_baseline"]["kind"] == "oracle"
