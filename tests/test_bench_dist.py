"""The multi-GPU bench path on CPU: replicas on world_size 2 over gloo.

bench.py runs one independent replica per rank (queries do not shard a
search); the only exchange is the whole-job throughput: all ranks' edges over
the slowest rank's time.  The reference arm runs on rank 0 alone."""
import io
import os
import socket
import contextlib

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed (r + 1) * 1e9 edges in 10 * (r + 1) ms
        value, ms = bench.job_throughput((rank + 1) * 1e9, 10.0 * (rank + 1), dist, "cpu")
        out.put((rank, value, ms))
    finally:
        dist.destroy_process_group()


def test_job_throughput_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(out.get(timeout=10) for _ in range(2))
    # 3e9 edges over the slowest rank's 20 ms on every rank
    for rank, value, ms in res:
        assert ms == pytest.approx(20.0)
        assert value == pytest.approx(3e9 / 20e-3 / 1e9)


def test_job_throughput_single_rank():
    value, ms = bench.job_throughput(2e9, 4.0)
    assert ms == 4.0 and value == pytest.approx(500.0)


def test_reference_arm_runs_on_rank_zero_only():
    class Args:
        workload = "er16"
        steps = 1
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args(), 2, 1)
    assert buf.getvalue() == ""


def test_reference_arm_line_on_rank_zero():
    """The reference arm's JSON line carries the contract's keys and times the
    oracle on the host (ER 2^16, one step)."""
    import json

    class Args:
        workload = "er16"
        steps = 2
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(Args(), 1, 0)
    line = json.loads(buf.getvalue().strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["metric"] == "GTEPS" and line["value"] > 0
    assert line["config"]["workload"] == "er16_src0"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
