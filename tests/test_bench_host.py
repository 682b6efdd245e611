"""Host logic of bench.py for a job of several ranks (the replicas of --gpus N), on CPU ranks
with the gloo backend: max-over-ranks timing, and the reference arm that only rank 0 runs."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        out[rank] = bench.max_over_ranks(10.0 * (rank + 1), world, "cpu")
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_with_two_gloo_ranks():
    world, port = 2, _free_port()
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    assert dict(out) == {0: 20.0, 1: 20.0}


def test_max_over_ranks_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun the reference arm (the oracle on the host) runs on rank 0; the other
    ranks return at once without output."""
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    args = bench.parse()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    assert buf.getvalue() == ""


def test_reference_arm_prints_the_contract_line(monkeypatch):
    """Rank 0 of the reference arm prints one JSON line with the contract's keys: the oracle
    timed on the host on the benchmark's workload, cut to a bounded sample."""
    import json
    import bench
    monkeypatch.delenv("RANK", raising=False)
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                                      "--cpu-levels", "3"])
    args = bench.parse()
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)
    lines = [l for l in buf.getvalue().splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "Gdof/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["host"]["nproc"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert "workload" in d["config"]
    # the line states what this arm ran: the FP64 oracle on a cut of the workload
    assert d["config"]["precision"].startswith("FP64")
    assert "cut to" in d["config"]["sample"]


def test_cpu_baseline_legs(monkeypatch):
    """The CPU baseline times the one-thread oracle and the OpenMP build on every host core,
    each with its set-up and solve seconds, and records the host's cores and CPU model."""
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()
    cb = bench.cpu_baseline(args, 3, 4, min_seconds=0.0, max_runs=1)
    assert cb["kind"] == "oracle" and cb["value"] > 0 and cb["cores"] >= 1
    assert cb["host"]["nproc"] >= 1 and isinstance(cb["host"]["cpu_model"], str)
    one, omp = cb["legs"]
    assert one["cores"] == 1 and omp["cores"] >= 1
    assert one["finest"] == "32^3" and omp["finest"] == "64^3"
    for leg in (one, omp):
        assert leg["seconds_assembly"] > 0 and leg["seconds_solve"] > 0


def test_k1_traffic_record_matches_the_byte_model():
    """The ncu figures the bench line reports as K1's `traffic` (profiles/k_pq_float_traffic.json)
    belong to the kernel the bench times: the ring form at the recorded size moves 16 bytes per
    node off the Dirichlet faces (r and p_old in, p and q out), the record's sum is its read plus
    its write, and the measured traffic stays within a few percent of those bytes."""
    import json
    d = json.load(open(os.path.join(ROOT, "profiles", "k_pq_float_traffic.json")))
    n = d["n"]
    assert d["algorithmic_bytes_per_launch"] == 16 * (n - 1) ** 3
    assert abs(d["dram_bytes_per_launch"] - (d["dram_bytes_read"] + d["dram_bytes_write"])) < 1.0
    assert 1.0 <= d["dram_bytes_per_launch"] / d["algorithmic_bytes_per_launch"] < 1.05
    assert os.path.exists(os.path.join(ROOT, "profiles", d["source"]))
