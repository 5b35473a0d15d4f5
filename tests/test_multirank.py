"""bench.py's multi-process path on CPU: two gloo ranks on 127.0.0.1.

Every rank solves its own replica (no data-path collective); the job's time
is the slowest rank's, and the job's value is all ranks' solves over it.
"""
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


def _rank_main(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, l = bench._dist()
        t = bench.max_over_ranks(100.0 + 50.0 * rank, torch.device("cpu"))
        q.put((rank, w, r, l, t, bench.job_rate(w, 5, t)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_the_work():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, PORT[0], q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(ws))
    for rank, w, r, l, t, v in got:
        assert (w, r, l) == (ws, rank, rank)
        assert t == 150.0                      # the slower rank's time on every rank
        assert v == pytest.approx(2 * 5 / 0.150)  # 10 solves in 150 ms


def test_single_process_is_identity():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, torch.device("cpu")) == 12.5
    assert bench.job_rate(1, 3, 1500.0) == pytest.approx(2.0)


PORT = [_free_port()]


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    # under torchrun the oracle arm runs and prints on rank 0 only; other
    # ranks exit 0 without work
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = bench.build_parser().parse_args(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert bench.run_reference(args) == 0
    assert capsys.readouterr().out == ""


def test_gpu_count_must_match_the_launched_ranks(monkeypatch, capsys):
    # `bench.py --gpus 2` started as one process (not through torch.distributed.run)
    # refuses to run rather than report one GPU's rate as two GPUs'; the check
    # comes before any device work, so it runs on the CPU
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    monkeypatch.setenv("LOCAL_RANK", "0")
    args = bench.build_parser().parse_args(["--gpus", "2", "--steps", "1", "--warmup", "0"])
    assert bench.run_ours(args) == 2
    err = capsys.readouterr().err
    assert "--gpus 2" in err and "torch.distributed.run" in err


def test_reference_arm_json_line_contract():
    # the reference arm (the FP64 oracle on host cores) runs without a GPU:
    # one JSON line with the contract's keys, its own cpu_baseline and an e2e
    # entry with zero transfer bytes
    import json
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT,
                         env=dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0"))
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "solves/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


def _sum_main(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        import synth
        W = synth.WORKLOADS["batched"]
        sides, _ = synth.batch_systems(W["seed"], W["nsys"])
        mine = bench.partition_jobs([int(v) ** 2 for v in sides], ws)[rank]
        # each rank counts its own jobs; the job totals come from the sum over ranks
        q.put((rank, sorted(mine), bench.sum_over_ranks(len(mine), torch.device("cpu"))))
    finally:
        dist.destroy_process_group()


def test_batched_partition_over_two_gloo_ranks():
    # the batched workload's 256 systems split over two ranks: disjoint,
    # complete, balanced by size (loads differ by at most the largest
    # system), and the per-rank counts sum to the job total on every rank
    import synth
    sys.path.insert(0, ROOT)
    import bench
    W = synth.WORKLOADS["batched"]
    sides, _ = synth.batch_systems(W["seed"], W["nsys"])
    sizes = [int(v) ** 2 for v in sides]
    for ws in (1, 2, 3, 8):
        parts = bench.partition_jobs(sizes, ws)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) - min(loads) <= max(sizes)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sum_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert set(got[0][1]).isdisjoint(got[1][1])
    assert sorted(got[0][1] + got[1][1]) == list(range(len(sizes)))
    assert got[0][2] == got[1][2] == len(sizes)
