"""The benchmark's multi-rank logic on CPU: two gloo ranks, each with its own
share of work and no data-path collective; the job time is the slowest
rank's time (max over ranks) and the aggregate counts every rank's units."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank), CVS_BENCH_BACKEND="gloo")
    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    # each rank's own timing of its share; rank 1 is the slow one
    local_seconds = 1.5 if rank == 1 else 1.0
    bench.barrier(w)
    t = bench.max_over_ranks(local_seconds, w)
    units_per_rank = 1000
    value = w * units_per_rank / t
    q.put((rank, t, value))
    import torch.distributed as dist
    dist.destroy_process_group()


def test_two_rank_max_and_aggregate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    res = sorted(q.get(timeout=10) for _ in range(2))
    assert [r[1] for r in res] == [1.5, 1.5]          # both see the slowest rank's time
    assert res[0][2] == pytest.approx(2 * 1000 / 1.5)  # units of all ranks / max time


# --------------------------------------------------------------- reference arm
def _reference_cmd(extra=()):
    return [*extra, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
            "--warmup", "1", "--cpu-sample", "256"]


def _json_lines(out: str):
    import json
    return [json.loads(ln) for ln in out.splitlines() if ln.startswith("{")]


def test_reference_arm_line():
    """One rank: one JSON line timing the FP64 CPU oracle on a bounded sample."""
    import subprocess
    r = subprocess.run([sys.executable, *_reference_cmd()], cwd=ROOT, capture_output=True,
                       text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["unit"] == "Gcand/s" and line["value"] > 0
    assert line["higher_is_better"] is True and line["steps"] == 1 and line["warmup"] == 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "Gcand/s",
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_two_ranks_rank0_only():
    """Launched as the multi-GPU runs are (torch.distributed.run, two ranks,
    gloo here): rank 0 alone runs the oracle and prints; the other rank exits 0
    without work."""
    import subprocess
    env = dict(os.environ, CVS_BENCH_BACKEND="gloo")
    cmd = _reference_cmd([sys.executable, "-m", "torch.distributed.run", "--nnodes=1",
                          "--nproc-per-node", "2", "--master-addr", "127.0.0.1",
                          "--master-port", str(_free_port())])
    cmd += ["--gpus", "2"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["impl"] == "reference" and lines[0]["n_gpus"] == 2
