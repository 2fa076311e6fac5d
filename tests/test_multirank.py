"""The host side of a multi-process bench run (one process per GPU, each a
replica of the workload): two gloo ranks on the CPU.  The job's time is
the slowest rank's (an all-reduce MAX over the ranks), the job's work the
sum over ranks, and the rank variables come from the launcher's
environment.  The reference arm prints nothing on ranks other than 0, and on
rank 0 one JSON line with the benchmark's keys."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import sys
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        got_ws, got_rank, got_local = bench._dist()
        t = bench.max_over_ranks(1.5 + rank, got_ws, "cpu")   # rank r took 1.5 + r s
        units = bench.job_units(1000, got_ws)
        out.put((rank, got_ws, got_rank, got_local, t, units))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, got_ws, got_rank, got_local, t, units) in enumerate(res):
        assert (rank, got_ws, got_rank, got_local) == (r, ws, r, r)
        assert t == pytest.approx(1.5 + ws - 1)          # the slowest rank's time on every rank
        assert units == 1000 * ws


def test_single_rank_needs_no_process_group(monkeypatch):
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench._dist() == (1, 0, 0)
    assert bench.max_over_ranks(2.5, 1, "cpu") == 2.5
    assert bench.job_units(7, 1) == 7


def test_reference_arm_silent_off_rank_zero(monkeypatch, capsys):
    import argparse
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(argparse.Namespace(workload="cosmo128", steps=1, warmup=0))
    assert capsys.readouterr().out == ""


def test_reference_arm_json_line():
    """The reference arm (the FP64 oracle on the full workload, no GPU)
    prints one JSON line with the benchmark's keys."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1"],
                         cwd=root, capture_output=True, text=True, check=True, env=env, timeout=600).stdout
    lines = [ln for ln in out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
